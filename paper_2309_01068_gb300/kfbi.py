"""Thin Python binding of libkfbi (include/kfbi.h) over ctypes.

Argument marshalling only: tensors are passed as device pointers on torch's current
CUDA stream; every step of the method runs in the library's CUDA kernels. There is no
CPU fallback: if libkfbi.so is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkfbi.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "kfbi.h")

# codes mirrored from include/kfbi.h
OK, ERR_ARG, ERR_CUDA, ERR_OUTSIDE_BOX, ERR_UNDERRESOLVED, ERR_NOT_CONVERGED = 0, 1, 2, 3, 4, 5
OPT_CUDA_GRAPHS, OPT_CLUSTER_GMRES, OPT_LAST_CLUSTER, OPT_PDL, OPT_CLUSTER_SIZE, OPT_COL_PAIRS = 1, 2, 3, 4, 5, 6
OPT_BOX_MATRIX = 7
OPT_FP32_ARNOLDI = 8
OPT_PUSH_REDUCE = 9
OPT_FUSE_INTERP = 10
OPT_FUSE_DFT = 11
OPT_BODY_CAP, OPT_SWEEP_CAP, OPT_COL_REG, OPT_COL_TC, OPT_COL_RADIX4, OPT_FUSE_ROWS = 12, 13, 14, 15, 16, 17
OPT_COL_POINTS = 18
OPT_GRID_IR = 19
MLP_FEATURES, MLP_MODES = 47, 16
ERR_SINGULAR, ERR_TIMEOUT, ERR_STATE, ERR_CAPACITY = 6, 7, 8, 9
BOX_DIRICHLET0, BOX_NEUMANN0, BOX_FREESPACE_DL = 0, 1, 2
FP64, MIXED = 0, 1
SINGLE, DOUBLE = 0, 1
BIE_INTERIOR_DL, BIE_HS_EXTERIOR_MDL, BIE_STEFAN_SL = 0, 1, 2
STEP_HELE_SHAW, STEP_STEFAN = 0, 1
SCHEME_SEMI_IMPLICIT, SCHEME_EXPLICIT = 0, 1


class KfbiError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {_status_string(status)} (status {status})")


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("refinements", ctypes.c_int),
                ("status", ctypes.c_int), ("rel_residual", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class InstanceDesc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
                ("ymin", ctypes.c_double), ("ymax", ctypes.c_double), ("kappa", ctypes.c_double),
                ("boxbc", ctypes.c_int), ("max_nodes", ctypes.c_int)]


class ThetaLParams(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("sigma", ctypes.c_double), ("J", ctypes.c_double),
                ("St", ctypes.c_double), ("eps_c", ctypes.c_double), ("eps_aniso", ctypes.c_double),
                ("eps_v", ctypes.c_double), ("fold", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("restart", ctypes.c_int), ("scheme", ctypes.c_int),
                ("refine_ratio", ctypes.c_double), ("rescale", ctypes.c_int)]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

_SIGNATURES = {
    "kfbi_create": (_I, [_I, _D, _D, _D, _D, _D, _I, _I, _I, ctypes.POINTER(_P)]),
    "kfbi_destroy": (None, [_P]),
    "kfbi_set_stream": (_I, [_P, _P]),
    "kfbi_set_interface": (_I, [_P, _I, _P]),
    "kfbi_apply_layer_potential": (_I, [_P, _I, _P, _P, _P, _P]),
    "kfbi_bie_apply": (_I, [_P, _I, _P, _P, _P]),
    "kfbi_solve_bie": (_I, [_P, _I, _P, _P, _D, _I, _I, _P, ctypes.POINTER(SolveInfo)]),
    "kfbi_grid_solve": (_I, [_P, _P, _P]),
    "kfbi_grid_solve_mixed": (_I, [_P, _P, _P, _I]),
    "kfbi_interp_grid": (_I, [_P, _P, _P]),
    "kfbi_interface_stats": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "kfbi_copy_sides": (_I, [_P, _P]),
    "kfbi_copy_crossings": (_I, [_P, _I, _P, _P]),
    "kfbi_copy_irregular": (_I, [_P, _I, _P]),
    "kfbi_thetal_create": (_I, [_P, _I, _P, _D, ctypes.POINTER(_D), ctypes.POINTER(ThetaLParams),
                                ctypes.POINTER(_P)]),
    "kfbi_thetal_destroy": (None, [_P]),
    "kfbi_step": (_I, [_P, _P, _D, ctypes.POINTER(SolveInfo)]),
    "kfbi_thetal_read": (_I, [_P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(_D)]),
    "kfbi_thetal_write": (_I, [_P, _P, _P, _P, _P, _P, ctypes.POINTER(_D)]),
    "kfbi_status_string": (ctypes.c_char_p, [_I]),
    "kfbi_timing_enable": (_I, [_P, _I]),
    "kfbi_timing_read": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(_I)]),
    "kfbi_launch_count": (_I, [_P, ctypes.POINTER(ctypes.c_longlong)]),
    "kfbi_set_option": (_I, [_P, _I, _I]),
    "kfbi_mlp_create": (_I, [_I, _I, ctypes.POINTER(_P)]),
    "kfbi_mlp_destroy": (None, [_P]),
    "kfbi_mlp_set_stream": (_I, [_P, _P]),
    "kfbi_mlp_param_count": (_I, [_P, ctypes.POINTER(_I)]),
    "kfbi_mlp_set_tensor_cores": (_I, [_P, _I]),
    "kfbi_mlp_tc_error": (_I, [_P, ctypes.POINTER(_I)]),
    "kfbi_mlp_set_params": (_I, [_P, _P]),
    "kfbi_mlp_get_params": (_I, [_P, _P]),
    "kfbi_mlp_forward": (_I, [_P, _P, _I, _P]),
    "kfbi_mlp_gradients": (_I, [_P, _P, _P, _P, _I, _P, ctypes.POINTER(ctypes.c_float)]),
    "kfbi_mlp_train_step": (_I, [_P, _P, _P, _P, _I, ctypes.c_float, ctypes.POINTER(ctypes.c_float)]),
    "kfbi_warmstart_features": (_I, [_P, _P, _P, _P]),
    "kfbi_warmstart_predict": (_I, [_P, _P, _P, _P]),
    "kfbi_batch_create": (_I, [_I, _P, _I, ctypes.POINTER(_P)]),
    "kfbi_batch_destroy": (None, [_P]),
    "kfbi_batch_context": (_I, [_P, _I, ctypes.POINTER(_P)]),
    "kfbi_batch_set_stream": (_I, [_P, _P]),
    "kfbi_batch_solve": (_I, [_P, _I, _P, _P, _D, _I, _I, _P]),
    "kfbi_batch_autotune": (_I, [_P, _I, _P, _D, _I, _I, ctypes.POINTER(_D)]),
    "kfbi_get_option": (_I, [_P, _I, ctypes.POINTER(_I)]),
    "kfbi_grid_solve_noalloc": (_I, [_I, _D, _D, _I, _P, _P, _P]),
    "kfbi_alu_peak": (_I, [_I, ctypes.POINTER(_D), _P]),
    "kfbi_time_column": (_I, [_P, _I, _I, ctypes.POINTER(_D)]),
    "kfbi_tc_gemm": (_I, [_I, _I, _I, _P, ctypes.c_long, _I, _P, ctypes.c_long, _I, _P, ctypes.c_long, _I, _P, _P]),
    "kfbi_thetal_set_warmstart": (_I, [_P, _P]),
    "kfbi_thetal_count": (_I, [_P, ctypes.POINTER(_I)]),
    "kfbi_thetal_training_pair": (_I, [_P, _P, _P]),
}


def header_functions():
    """Names of the functions include/kfbi.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kfbi_\w+)\s*\(", text)))


def load():
    """Load libkfbi.so (built in-tree by build.py) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2309_01068_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _status_string(s):
    try:
        return load().kfbi_status_string(s).decode()
    except Exception:  # noqa: BLE001 - best effort message
        return "status"


def _check(status, where, allow=()):
    if status != OK and status not in allow:
        raise KfbiError(status, where)
    return status


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("libkfbi takes device tensors")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _f64(t, shape):
    if t.dtype != torch.float64 or tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected float64 tensor of shape {shape}, got {t.dtype} {tuple(t.shape)}")
    return _ptr(t)


def _opt_f64(t, shape):
    return None if t is None else _f64(t, shape)


def _f32(t, shape):
    if t.dtype != torch.float32 or tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected float32 tensor of shape {shape}, got {t.dtype} {tuple(t.shape)}")
    return _ptr(t)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Context:
    """kfbi_create / kfbi_destroy and the calls on one grid."""

    def __init__(self, N, box, kappa=0.0, boxbc=BOX_DIRICHLET0, precision=FP64, max_nodes=1024):
        self.lib = load()
        self.N = int(N)
        self.box = tuple(float(b) for b in box)
        self.kappa = float(kappa)
        self.boxbc = int(boxbc)
        self.precision = int(precision)
        self.max_nodes = int(max_nodes)
        self.n = 0
        h = ctypes.c_void_p()
        _check(self.lib.kfbi_create(self.N, *self.box, self.kappa, self.boxbc, self.precision, self.max_nodes,
                                    ctypes.byref(h)), "kfbi_create")
        self.handle = h

    @classmethod
    def borrowed(cls, handle, N, box, kappa, boxbc, precision, max_nodes):
        """A Context view of a context owned elsewhere (a batch instance); close() leaves it."""
        self = cls.__new__(cls)
        self.lib = load()
        self.N, self.box, self.kappa = int(N), tuple(float(b) for b in box), float(kappa)
        self.boxbc, self.precision, self.max_nodes = int(boxbc), int(precision), int(max_nodes)
        self.n = 0
        self.handle = handle
        self._borrowed = True
        return self

    def close(self):
        if getattr(self, "handle", None):
            if not getattr(self, "_borrowed", False):
                self.lib.kfbi_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def _sync_stream(self):
        _check(self.lib.kfbi_set_stream(self.handle, _stream()), "kfbi_set_stream")

    def set_interface(self, xy):
        self._sync_stream()
        n = xy.shape[0]
        _check(self.lib.kfbi_set_interface(self.handle, n, _f64(xy, (n, 2))), "kfbi_set_interface")
        self.n = n

    def apply(self, layer, density, dnormal=False, grid=False):
        self._sync_stream()
        n = self.n
        vals = torch.empty(max(n, 1), dtype=torch.float64, device=density.device)[:n]
        dn = torch.empty(n, dtype=torch.float64, device=density.device) if dnormal else None
        g = torch.empty((self.N, self.N), dtype=torch.float64, device=density.device) if grid else None
        dptr = _f64(density, (n,)) if n > 0 else _ptr(density)  # no interface yet: the library reports it
        _check(self.lib.kfbi_apply_layer_potential(self.handle, layer, dptr, _ptr(vals), _ptr(dn), _ptr(g)),
               "kfbi_apply_layer_potential")
        return vals, dn, g

    def apply_into(self, layer, density, values, dnormal=None, grid=None):
        """The apply into caller buffers, each checked for dtype and shape before the call."""
        self._sync_stream()
        n, N = self.n, self.N
        _check(self.lib.kfbi_apply_layer_potential(self.handle, layer, _f64(density, (n,)), _f64(values, (n,)),
                                                   _opt_f64(dnormal, (n,)), _opt_f64(grid, (N, N))),
               "kfbi_apply_layer_potential")

    def bie_apply(self, kind, x, eps_v=None, out=None):
        self._sync_stream()
        y = out if out is not None else torch.empty_like(x)
        _check(self.lib.kfbi_bie_apply(self.handle, kind, _opt_f64(eps_v, (self.n,)), _f64(x, (self.n,)),
                                       _f64(y, (self.n,))), "kfbi_bie_apply")
        return y

    def solve_bie(self, kind, rhs, density=None, tol=1e-10, max_iter=500, restart=100, eps_v=None):
        """Returns (density, info dict); density is updated in place when given. A solve that
        stops unconverged (ERR_NOT_CONVERGED) or at a loop bound (ERR_TIMEOUT) returns its
        iterate with that status in info["status"]; other errors raise."""
        self._sync_stream()
        x = density if density is not None else torch.zeros_like(rhs)
        info = SolveInfo()
        _check(self.lib.kfbi_solve_bie(self.handle, kind, _ptr(eps_v), _f64(rhs, (self.n,)), float(tol),
                                       int(max_iter), int(restart), _f64(x, (self.n,)), ctypes.byref(info)),
               "kfbi_solve_bie", allow=(ERR_NOT_CONVERGED, ERR_TIMEOUT))
        return x, info.as_dict()

    def grid_solve(self, rhs, out=None):
        self._sync_stream()
        u = out if out is not None else torch.empty_like(rhs)
        # both checked for dtype and shape before the call: the library writes N x N float64
        _check(self.lib.kfbi_grid_solve(self.handle, _f64(rhs, (self.N, self.N)), _f64(u, (self.N, self.N))),
               "kfbi_grid_solve")
        return u

    def grid_solve_mixed(self, rhs, sweeps=2, out=None):
        """kfbi_grid_solve_mixed (KFBI_MIXED contexts): float32 box solves with `sweeps` float64
        residual corrections; `out` must not be `rhs`."""
        self._sync_stream()
        u = out if out is not None else torch.empty_like(rhs)
        _check(self.lib.kfbi_grid_solve_mixed(self.handle, _f64(rhs, (self.N, self.N)), _f64(u, (self.N, self.N)),
                                              int(sweeps)), "kfbi_grid_solve_mixed")
        return u

    def interp_grid(self, grid):
        self._sync_stream()
        v = torch.empty(self.n, dtype=torch.float64, device=grid.device)
        _check(self.lib.kfbi_interp_grid(self.handle, _f64(grid, (self.N, self.N)), _ptr(v)), "kfbi_interp_grid")
        return v

    def stats(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self.lib.kfbi_interface_stats(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "kfbi_interface_stats")
        return dict(crossings=a.value, irregular=b.value, probes=c.value)

    def sides(self):
        self._sync_stream()
        s = torch.empty((self.N, self.N), dtype=torch.uint8, device="cuda")
        _check(self.lib.kfbi_copy_sides(self.handle, _ptr(s)), "kfbi_copy_sides")
        return s

    def crossings(self):
        self._sync_stream()
        cnt = self.stats()["crossings"]
        klf = torch.empty((max(cnt, 1), 3), dtype=torch.int32, device="cuda")
        ax = torch.empty((max(cnt, 1), 2), dtype=torch.float64, device="cuda")
        _check(self.lib.kfbi_copy_crossings(self.handle, cnt, _ptr(klf), _ptr(ax)), "kfbi_copy_crossings")
        return klf[:cnt], ax[:cnt]

    def irregular(self):
        self._sync_stream()
        cnt = self.stats()["irregular"]
        ji = torch.empty((max(cnt, 1), 2), dtype=torch.int32, device="cuda")
        _check(self.lib.kfbi_copy_irregular(self.handle, cnt, _ptr(ji)), "kfbi_copy_irregular")
        return ji[:cnt]

    def timing(self, enable=None):
        """timing(True/False) switches column-kernel event timing; timing() returns
        dict(fp64_ms, fp64_launches, fp32_ms, fp32_launches)."""
        if enable is not None:
            _check(self.lib.kfbi_timing_enable(self.handle, 1 if enable else 0), "kfbi_timing_enable")
            return None
        a, b, c, d = ctypes.c_double(), ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
        _check(self.lib.kfbi_timing_read(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                         ctypes.byref(d)), "kfbi_timing_read")
        return dict(fp64_ms=a.value, fp64_launches=b.value, fp32_ms=c.value, fp32_launches=d.value)

    def time_column(self, fp32=True, reps=200):
        """kfbi_time_column: mean microseconds per column solve, `reps` launches back to back
        (the spectral-grid scratch buffer is overwritten)."""
        self._sync_stream()
        v = ctypes.c_double()
        _check(self.lib.kfbi_time_column(self.handle, 1 if fp32 else 0, int(reps), ctypes.byref(v)),
               "kfbi_time_column")
        return v.value

    def set_option(self, option, value):
        """kfbi_set_option: one of the OPT_* constants (values as the header states)."""
        _check(self.lib.kfbi_set_option(self.handle, int(option), int(value)), "kfbi_set_option")

    def get_option(self, option):
        """kfbi_get_option: the current value of one of the OPT_* constants."""
        v = ctypes.c_int()
        _check(self.lib.kfbi_get_option(self.handle, int(option), ctypes.byref(v)), "kfbi_get_option")
        return v.value

    def warmstart_features(self, rhs):
        """kfbi_warmstart_features: (features [n][47] float32, rms(rhs) [1] float64)."""
        self._sync_stream()
        n = self.n
        feat = torch.empty((max(n, 1), MLP_FEATURES), dtype=torch.float32, device=rhs.device)[:n]
        scale = torch.empty(1, dtype=torch.float64, device=rhs.device)
        _check(self.lib.kfbi_warmstart_features(self.handle, _f64(rhs, (n,)), _ptr(feat), _ptr(scale)),
               "kfbi_warmstart_features")
        return feat, scale

    def warmstart_predict(self, mlp, rhs, out=None):
        """kfbi_warmstart_predict: the network's initial density for rhs."""
        self._sync_stream()
        n = self.n
        d = out if out is not None else torch.empty(n, dtype=torch.float64, device=rhs.device)
        _check(self.lib.kfbi_warmstart_predict(self.handle, mlp.handle, _f64(rhs, (n,)), _f64(d, (n,))),
               "kfbi_warmstart_predict")
        return d

    def launch_count(self):
        v = ctypes.c_longlong()
        _check(self.lib.kfbi_launch_count(self.handle, ctypes.byref(v)), "kfbi_launch_count")
        return v.value


class Mlp:
    """kfbi_mlp_*: the warm-start network (47 -> hidden -> hidden -> 1, bfloat16 weights)."""

    NAMES = ("W1", "b1", "W2", "b2", "w3", "b3")

    def __init__(self, hidden=256, max_rows=4096):
        self.lib = load()
        self.hidden = int(hidden)
        self.max_rows = int(max_rows)
        h = ctypes.c_void_p()
        _check(self.lib.kfbi_mlp_create(self.hidden, self.max_rows, ctypes.byref(h)), "kfbi_mlp_create")
        self.handle = h
        c = ctypes.c_int()
        _check(self.lib.kfbi_mlp_param_count(self.handle, ctypes.byref(c)), "kfbi_mlp_param_count")
        self.count = c.value

    def close(self):
        if getattr(self, "handle", None):
            self.lib.kfbi_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def _sync_stream(self):
        _check(self.lib.kfbi_mlp_set_stream(self.handle, _stream()), "kfbi_mlp_set_stream")

    def tensor_cores(self, enable):
        """kfbi_mlp_set_tensor_cores: the H x H layer on the tensor cores (True) or CUDA cores."""
        self._sync_stream()
        _check(self.lib.kfbi_mlp_set_tensor_cores(self.handle, 1 if enable else 0), "kfbi_mlp_set_tensor_cores")

    def tc_error(self):
        """kfbi_mlp_tc_error: 1 if a tensor-core completion wait gave up, else 0."""
        self._sync_stream()
        v = ctypes.c_int()
        _check(self.lib.kfbi_mlp_tc_error(self.handle, ctypes.byref(v)), "kfbi_mlp_tc_error")
        return v.value

    def _shapes(self):
        H, F = self.hidden, MLP_FEATURES
        return dict(W1=(H, F), b1=(H,), W2=(H, H), b2=(H,), w3=(H,), b3=())

    def flatten(self, params):
        """dict of arrays (W1, b1, W2, b2, w3, b3) -> flat float32 host array in the C layout."""
        import numpy as np

        parts = [np.asarray(params[k], dtype=np.float32).reshape(-1) for k in self.NAMES]
        flat = np.ascontiguousarray(np.concatenate(parts))
        if flat.size != self.count:
            raise ValueError(f"expected {self.count} parameters, got {flat.size}")
        return flat

    def unflatten(self, flat):
        import numpy as np

        out, o = {}, 0
        for k, shp in self._shapes().items():
            sz = int(np.prod(shp)) if shp else 1
            out[k] = flat[o:o + sz].reshape(shp) if shp else float(flat[o])
            o += sz
        return out

    def set_params(self, params):
        self._sync_stream()
        flat = self.flatten(params)
        _check(self.lib.kfbi_mlp_set_params(self.handle, flat.ctypes.data_as(ctypes.c_void_p)), "kfbi_mlp_set_params")

    def get_params(self):
        import numpy as np

        self._sync_stream()
        flat = np.empty(self.count, dtype=np.float32)
        _check(self.lib.kfbi_mlp_get_params(self.handle, flat.ctypes.data_as(ctypes.c_void_p)), "kfbi_mlp_get_params")
        return self.unflatten(flat)

    def forward(self, feat, out=None):
        self._sync_stream()
        rows = feat.shape[0]
        y = out if out is not None else torch.empty(rows, dtype=torch.float32, device=feat.device)
        _check(self.lib.kfbi_mlp_forward(self.handle, _f32(feat, (rows, MLP_FEATURES)), rows, _f32(y, (rows,))),
               "kfbi_mlp_forward")
        return y

    def gradients(self, feat, target, idx=None):
        """(loss, flat gradient tensor) of the mean squared error on rows idx (all rows if None)."""
        self._sync_stream()
        rows = feat.shape[0] if idx is None else idx.shape[0]
        g = torch.empty(self.count, dtype=torch.float32, device=feat.device)
        loss = ctypes.c_float()
        _check(self.lib.kfbi_mlp_gradients(self.handle, _ptr(feat), _ptr(target), _ptr(idx), rows, _ptr(g),
                                           ctypes.byref(loss)), "kfbi_mlp_gradients")
        return loss.value, g

    def train_step(self, feat, target, idx=None, lr=1e-3, want_loss=True):
        self._sync_stream()
        rows = feat.shape[0] if idx is None else idx.shape[0]
        loss = ctypes.c_float()
        _check(self.lib.kfbi_mlp_train_step(self.handle, _ptr(feat), _ptr(target), _ptr(idx), rows, float(lr),
                                            ctypes.byref(loss) if want_loss else None), "kfbi_mlp_train_step")
        return loss.value if want_loss else None


class Batch:
    """kfbi_batch_*: many independent instances solved by one graph launch."""

    def __init__(self, descs, precision=MIXED):
        """descs: list of dict(N, box=(xmin, xmax, ymin, ymax), kappa, boxbc, max_nodes)."""
        self.lib = load()
        self.count = len(descs)
        self.precision = int(precision)
        arr = (InstanceDesc * self.count)()
        for i, d in enumerate(descs):
            x0, x1, y0, y1 = (float(v) for v in d["box"])
            arr[i] = InstanceDesc(int(d["N"]), x0, x1, y0, y1, float(d.get("kappa", 0.0)),
                                  int(d.get("boxbc", BOX_DIRICHLET0)), int(d["max_nodes"]))
        h = ctypes.c_void_p()
        _check(self.lib.kfbi_batch_create(self.count, ctypes.cast(arr, ctypes.c_void_p), self.precision,
                                          ctypes.byref(h)), "kfbi_batch_create")
        self.handle = h
        self.contexts = []
        for i, d in enumerate(descs):
            c = ctypes.c_void_p()
            _check(self.lib.kfbi_batch_context(self.handle, i, ctypes.byref(c)), "kfbi_batch_context")
            self.contexts.append(Context.borrowed(c, d["N"], d["box"], d.get("kappa", 0.0),
                                                  d.get("boxbc", BOX_DIRICHLET0), self.precision, d["max_nodes"]))

    def close(self):
        if getattr(self, "handle", None):
            for c in self.contexts:
                c.handle = None
            self.lib.kfbi_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def _ptrs(self, tensors):
        arr = (ctypes.c_void_p * self.count)()
        for i, t in enumerate(tensors):
            arr[i] = _ptr(t).value
        return arr

    def solve(self, kind, rhs, density, tol=1e-8, max_iter=500, restart=100):
        """rhs, density: lists of device float64 tensors; density holds the guess, gets the
        solution. Returns (status, list of info dicts)."""
        _check(self.lib.kfbi_batch_set_stream(self.handle, _stream()), "kfbi_batch_set_stream")
        infos = (SolveInfo * self.count)()
        rp, dp = self._ptrs(rhs), self._ptrs(density)  # kept alive across the call
        st = self.lib.kfbi_batch_solve(self.handle, int(kind), ctypes.cast(rp, ctypes.c_void_p),
                                       ctypes.cast(dp, ctypes.c_void_p), float(tol), int(max_iter), int(restart),
                                       ctypes.cast(infos, ctypes.c_void_p))
        _check(st, "kfbi_batch_solve", allow=(ERR_NOT_CONVERGED,))
        return st, [infos[i].as_dict() for i in range(self.count)]

    def autotune(self, kind, rhs, tol=1e-8, max_iter=500, restart=100):
        _check(self.lib.kfbi_batch_set_stream(self.handle, _stream()), "kfbi_batch_set_stream")
        ms = ctypes.c_double()
        rp = self._ptrs(rhs)
        _check(self.lib.kfbi_batch_autotune(self.handle, int(kind), ctypes.cast(rp, ctypes.c_void_p),
                                            float(tol), int(max_iter), int(restart), ctypes.byref(ms)),
               "kfbi_batch_autotune")
        return ms.value


def grid_solve_noalloc(rhs, h, kappa=0.0, boxbc=BOX_DIRICHLET0, out=None):
    """kfbi_grid_solve_noalloc: the box solve without any device allocation in the library
    (its scratch is a static device array; N <= 512). `out` may be preallocated (float64,
    N x N, on the device of rhs; it may be rhs itself); anything else raises ValueError before
    the library is called."""
    lib = load()
    N = rhs.shape[0]
    rp = _f64(rhs, (N, N))
    u = out if out is not None else torch.empty_like(rhs)
    up = _f64(u, (N, N))
    if u.device != rhs.device:
        raise ValueError(f"out is on {u.device}, rhs on {rhs.device}")
    _check(lib.kfbi_grid_solve_noalloc(N, float(h), float(kappa), int(boxbc), rp, up, _stream()),
           "kfbi_grid_solve_noalloc")
    return u


class ThetaL:
    """kfbi_thetal_create / kfbi_step / kfbi_thetal_read on a context."""

    def __init__(self, ctx: Context, eta, L, xbar, kind, tol=1e-8, max_iter=500, restart=100, sigma=0.0, J=0.0,
                 St=0.0, eps_c=0.0, eps_aniso=0.0, eps_v=0.0, fold=4, scheme=SCHEME_SEMI_IMPLICIT, refine_ratio=0.0,
                 rescale=False):
        self.ctx = ctx
        self.lib = ctx.lib
        self.n = eta.shape[0]
        p = ThetaLParams(kind=kind, sigma=sigma, J=J, St=St, eps_c=eps_c, eps_aniso=eps_aniso, eps_v=eps_v,
                         fold=fold, tol=tol, max_iter=max_iter, restart=restart, scheme=scheme,
                         refine_ratio=float(refine_ratio), rescale=1 if rescale else 0)
        xb = (ctypes.c_double * 2)(float(xbar[0]), float(xbar[1]))
        h = ctypes.c_void_p()
        ctx._sync_stream()
        _check(self.lib.kfbi_thetal_create(ctx.handle, self.n, _f64(eta, (self.n,)), float(L), xb, ctypes.byref(p),
                                           ctypes.byref(h)), "kfbi_thetal_create")
        self.handle = h

    def step(self, dt):
        self.ctx._sync_stream()
        info = SolveInfo()
        _check(self.lib.kfbi_step(self.ctx.handle, self.handle, float(dt), ctypes.byref(info)), "kfbi_step",
               allow=(ERR_NOT_CONVERGED,))
        c = ctypes.c_int()
        _check(self.lib.kfbi_thetal_count(self.handle, ctypes.byref(c)), "kfbi_thetal_count")
        self.n = c.value          # marker doubling may have grown it
        self.ctx.n = self.n  # the step set the context's interface
        return info.as_dict()

    SCALARS = 20

    def read(self, T=True):
        """State as device tensors plus the host scalars (checkpoint)."""
        self.ctx._sync_stream()
        n, N = self.n, self.ctx.N
        eta = torch.empty(n, dtype=torch.float64, device="cuda")
        xy = torch.empty((n, 2), dtype=torch.float64, device="cuda")
        dens = torch.empty(n, dtype=torch.float64, device="cuda")
        nhat = torch.empty((n // 2 + 1, 2), dtype=torch.float64, device="cuda")
        Tg = torch.empty((N, N), dtype=torch.float64, device="cuda") if T else None
        Tp = torch.empty((N, N), dtype=torch.float64, device="cuda") if T else None
        sc = (ctypes.c_double * self.SCALARS)()
        _check(self.lib.kfbi_thetal_read(self.handle, _ptr(eta), _ptr(xy), _ptr(dens), _ptr(nhat), _ptr(Tg), _ptr(Tp),
                                         sc), "kfbi_thetal_read")
        torch.cuda.current_stream().synchronize()
        return dict(eta=eta, xy=xy, density=dens, nhat=nhat, T=Tg, T_prev=Tp, scalars=list(sc), L=sc[0],
                    Xbar=(sc[1], sc[2]), t=sc[3], steps=int(sc[4]))

    def write(self, eta=None, density=None, nhat=None, T=None, T_prev=None, scalars=None):
        """Restore (part of) the state; arguments are device tensors and a host list."""
        self.ctx._sync_stream()
        sc = None
        if scalars is not None:
            sc = (ctypes.c_double * self.SCALARS)(*[float(v) for v in scalars])
        _check(self.lib.kfbi_thetal_write(self.handle, _ptr(eta), _ptr(density), _ptr(nhat), _ptr(T), _ptr(T_prev),
                                          sc), "kfbi_thetal_write")

    def set_warmstart(self, mlp):
        """kfbi_thetal_set_warmstart: attach a network (Mlp) or detach (None)."""
        self._mlp = mlp  # kept alive while attached
        _check(self.lib.kfbi_thetal_set_warmstart(self.handle, mlp.handle if mlp is not None else None),
               "kfbi_thetal_set_warmstart")

    def training_pair(self):
        """kfbi_thetal_training_pair: (features [n][47] float32, target [n] float32) of the last step."""
        self.ctx._sync_stream()
        feat = torch.empty((self.n, MLP_FEATURES), dtype=torch.float32, device="cuda")
        target = torch.empty(self.n, dtype=torch.float32, device="cuda")
        _check(self.lib.kfbi_thetal_training_pair(self.handle, _ptr(feat), _ptr(target)), "kfbi_thetal_training_pair")
        return feat, target

    def close(self):
        if getattr(self, "handle", None):
            self.lib.kfbi_thetal_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def alu_peak(kind):
    """kfbi_alu_peak: measured FMA throughput in TFLOP/s (kind 0 float32, 1 float64)."""
    lib = load()
    v = ctypes.c_double()
    _check(lib.kfbi_alu_peak(int(kind), ctypes.byref(v), _stream()), "kfbi_alu_peak")
    return v.value


def tc_gemm(A, B, transA=False, transB=False, terms=3):
    """kfbi_tc_gemm: C = A B^T on the tensor cores (float32 device tensors). A is M x K (or K x M
    with transA), B is N x K (or K x N with transB). Returns (C, error flag)."""
    lib = load()
    if A.dtype != torch.float32 or B.dtype != torch.float32 or A.dim() != 2 or B.dim() != 2:
        raise ValueError("tc_gemm takes 2-D float32 tensors")
    M, K = (A.shape[1], A.shape[0]) if transA else (A.shape[0], A.shape[1])
    N, K2 = (B.shape[1], B.shape[0]) if transB else (B.shape[0], B.shape[1])
    if K2 != K:
        raise ValueError(f"inner dimensions differ: {K} and {K2}")
    C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib.kfbi_tc_gemm(M, N, K, _ptr(A), A.shape[1], int(transA), _ptr(B), B.shape[1], int(transB), _ptr(C), N,
                            int(terms), _ptr(err), _stream()), "kfbi_tc_gemm")
    return C, err
