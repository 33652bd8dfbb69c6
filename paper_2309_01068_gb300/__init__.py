"""GB300-native kernel-free boundary integral (KFBI) library.

The compute path is libkfbi.so (hand-written CUDA for sm_103a, C ABI in include/kfbi.h),
built in-tree by `paper_2309_01068_gb300.build.build()`; `paper_2309_01068_gb300.kfbi` is
its thin ctypes binding.
"""
