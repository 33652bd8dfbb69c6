"""CPU oracle for the KFBI hot path (plain, slow, FP64; numpy + scipy.fft).

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the CPU-baseline
leg of bench.py may import this package. The product path (the CUDA library and its
Python binding) never imports, links or executes anything here, and this package
imports nothing from the product.

Modules:
  kfbi    grid, trigonometric interpolant, crossings/classification, jumps,
          corrected five-point right-hand side, DST/DCT solve, jump-corrected
          interpolation, layer-potential apply, BIE operators (Sec. 3, Sec. 4, App. A)
  gmres   restarted GMRES with modified Gram-Schmidt and Givens rotations (Sec. 4)
  thetal  theta-L interface evolution with small-scale decomposition and the
          semi-implicit propagator (Sec. 5); Hele-Shaw and Stefan steps
  mlp     forward/backward of the warm-start multilayer perceptron (not in the paper)
"""
