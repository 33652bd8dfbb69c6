"""The register-resident radix-16 column solve, the default float32 column kernel for N >= 32.

- float64 (the radix-16 kernel selected; float64 applies default to the radix-4 kernel): the
  grid solve (rows, columns through the radix-16 kernel, inverse rows) against the
  oracle's fast solve (Sec. 4.2) to 1e-12 for every power of two from 32 to 4096, both box types
  (DST-II and DCT-II columns) and both of the kernel's pair counts, and against the radix-4
  shared-memory kernel (the same arithmetic up to rounding order);
- float32: the apply of a mixed context (16 and 8 points per thread, every pair count) against
  the same apply through the radix-4 kernel (both float32) and against the oracle's float64 apply, for the three boxes (the free-space box leaves
  rows without irregular nodes to the column kernel, which forms them from their box data).
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import kfbi as OK

pytestmark = pytest.mark.gpu

K = pytest.importorskip("paper_2309_01068_gb300.kfbi")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_01068_gb300 import build

    build.build()
    K.load()


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


SIZES = [32, 64, 128, 256, 512, 1024, 2048, 4096]


@pytest.mark.parametrize("N", SIZES)
@pytest.mark.parametrize("boxbc,kappa", [(OK.BOX_DIRICHLET0, 0.0), (OK.BOX_DIRICHLET0, 40.0), (OK.BOX_NEUMANN0, 20.0)])
def test_grid_solve_radix16(N, boxbc, kappa):
    C = np.random.default_rng(N + 7 * boxbc + int(kappa)).standard_normal((N, N))
    ctx = K.Context(N, (-1.0, 1.0, -1.0, 1.0), kappa, boxbc, K.FP64, max_nodes=64)
    assert ctx.get_option(K.OPT_COL_RADIX4) == 2  # default: radix-16 in float32, radix-4 in float64
    ctx.set_option(K.OPT_COL_RADIX4, 0)
    ref = OK.solve_grid(OK.Grid(N, (-1, 1, -1, 1)), C, kappa, boxbc)
    u_def = ctx.grid_solve(dev(C)).cpu().numpy()
    assert rel(u_def, ref) < 1e-12
    # the other pair counts of the kernel (PMIN, and 2 PMIN for N <= 1024)
    for pairs in (1, min(16, 2 * max(1, 512 // N))):
        ctx.set_option(K.OPT_COL_PAIRS, pairs)
        u_alt = ctx.grid_solve(dev(C)).cpu().numpy()
        assert rel(u_alt, ref) < 1e-12, pairs
    ctx.set_option(K.OPT_COL_PAIRS, 0)
    # the radix-4 kernel for float64
    ctx.set_option(K.OPT_COL_RADIX4, 2)
    u_r4 = ctx.grid_solve(dev(C)).cpu().numpy()
    assert rel(u_def, u_r4) < 1e-13
    ctx.close()


BOXES = [(OK.BOX_DIRICHLET0, 0.0, 1.0), (OK.BOX_NEUMANN0, 30.0, 1.0), (OK.BOX_FREESPACE_DL, 0.0, 1.5)]


@pytest.mark.parametrize("N", SIZES[:-1])
@pytest.mark.parametrize("boxbc,kappa,box", BOXES)
def test_float32_apply_radix16(N, boxbc, kappa, box):
    n = max(16, min(N, 256))
    R0 = (0.2, 0.3) if N <= 32 else (0.35, 0.55)
    p = W.random_problem(500 + N, N=N, n=n, kappa=kappa, boxbc=boxbc, box=box, R0=R0)
    ctx = K.Context(p.N, p.box, kappa, boxbc, K.MIXED, max_nodes=p.n)
    ctx.set_interface(dev(p.xy))
    dens = W.random_density(N + 1, p.n, modes=6)
    layers = (K.DOUBLE,) if boxbc == OK.BOX_FREESPACE_DL else (K.DOUBLE, K.SINGLE)
    ref = OK.Kfbi(p.N, p.box, kappa, boxbc).set_interface(p.xy)
    for layer in layers:
        v16, _, _ = ctx.apply(layer, dev(dens))
        ctx.set_option(K.OPT_COL_PAIRS, 1)
        v16b, _, _ = ctx.apply(layer, dev(dens))
        ctx.set_option(K.OPT_COL_PAIRS, min(16, 2 * max(1, 512 // N)))
        v16c, _, _ = ctx.apply(layer, dev(dens))
        ctx.set_option(K.OPT_COL_PAIRS, 0)
        ctx.set_option(K.OPT_COL_POINTS, 8)
        v8, _, _ = ctx.apply(layer, dev(dens))
        ctx.set_option(K.OPT_COL_PAIRS, 1)
        v8b, _, _ = ctx.apply(layer, dev(dens))
        ctx.set_option(K.OPT_COL_PAIRS, 0)
        ctx.set_option(K.OPT_COL_POINTS, 16)
        v16d, _, _ = ctx.apply(layer, dev(dens))
        ctx.set_option(K.OPT_COL_POINTS, 0)
        ctx.set_option(K.OPT_COL_RADIX4, 3)
        v4, _, _ = ctx.apply(layer, dev(dens))
        ctx.set_option(K.OPT_COL_RADIX4, 2)
        a, b, c = v16.cpu().numpy(), v16b.cpu().numpy(), v4.cpu().numpy()
        assert np.isfinite(a).all()
        assert rel(a, c) < 2e-5, (layer, rel(a, c))
        assert rel(b, c) < 2e-5, (layer, rel(b, c))
        assert rel(v16c.cpu().numpy(), c) < 2e-5, layer
        assert rel(v8.cpu().numpy(), c) < 2e-5, layer    # 8 points per thread
        assert rel(v8b.cpu().numpy(), c) < 2e-5, layer
        assert rel(v16d.cpu().numpy(), c) < 2e-5, layer  # 16 points per thread
        rv, _, _ = ref.apply(OK.LAYER_DOUBLE if layer == K.DOUBLE else OK.LAYER_SINGLE, dens)
        assert rel(a, rv) < 2e-4, (layer, rel(a, rv))
    ctx.close()


def test_option_values():
    ctx = K.Context(64, (-1.0, 1.0, -1.0, 1.0), 0.0, OK.BOX_DIRICHLET0, K.MIXED, max_nodes=64)
    assert ctx.get_option(K.OPT_COL_POINTS) == 0
    for v in (8, 16, 0):
        ctx.set_option(K.OPT_COL_POINTS, v)
        assert ctx.get_option(K.OPT_COL_POINTS) == v
    with pytest.raises(K.KfbiError):
        ctx.set_option(K.OPT_COL_POINTS, 4)
    for v in (0, 1, 2, 3):
        ctx.set_option(K.OPT_COL_RADIX4, v)
        assert ctx.get_option(K.OPT_COL_RADIX4) == v
    for bad in (-1, 4):
        with pytest.raises(K.KfbiError):
            ctx.set_option(K.OPT_COL_RADIX4, bad)
    ctx.close()


@pytest.mark.parametrize("N", [64, 256, 1024, 2048])
@pytest.mark.parametrize("boxbc,kappa,box", BOXES)
def test_rows_formed_in_the_column_kernel(N, boxbc, kappa, box):
    """KFBI_OPT_FUSE_ROWS = 1: the float32 apply whose column kernel forms the row transform from
    the arm corrections (one launch fewer) against the same apply with the separate row transform
    (float32 both: rounding order only) and against the oracle's float64 apply."""
    n = max(16, min(N, 512))
    p = W.random_problem(700 + N, N=N, n=n, kappa=kappa, boxbc=boxbc, box=box)
    ctx = K.Context(p.N, p.box, kappa, boxbc, K.MIXED, max_nodes=p.n)
    ctx.set_interface(dev(p.xy))
    assert ctx.get_option(K.OPT_FUSE_ROWS) == 0
    ctx.set_option(K.OPT_FUSE_ROWS, 1)
    dens = W.random_density(N + 3, p.n, modes=8)
    ref = OK.Kfbi(p.N, p.box, kappa, boxbc).set_interface(p.xy)
    layers = (K.DOUBLE,) if boxbc == OK.BOX_FREESPACE_DL else (K.DOUBLE, K.SINGLE)
    for layer in layers:
        l0 = ctx.launch_count()
        vf, _, _ = ctx.apply(layer, dev(dens))
        lf = ctx.launch_count() - l0
        ctx.set_option(K.OPT_FUSE_ROWS, 0)
        l0 = ctx.launch_count()
        vs, _, _ = ctx.apply(layer, dev(dens))
        ls = ctx.launch_count() - l0
        ctx.set_option(K.OPT_FUSE_ROWS, 1)
        assert lf == ls - 1, (lf, ls)
        a, b = vf.cpu().numpy(), vs.cpu().numpy()
        assert np.isfinite(a).all()
        assert rel(a, b) < 2e-5, (layer, rel(a, b))
        rv, _, _ = ref.apply(OK.LAYER_DOUBLE if layer == K.DOUBLE else OK.LAYER_SINGLE, dens)
        assert rel(a, rv) < 2e-4, (layer, rel(a, rv))
    ctx.close()


def test_rows_formed_in_the_column_kernel_follow_the_interface():
    """The arm map is rebuilt with every interface: a second interface on the same context
    (different crossings and irregular nodes) gives the same apply as a fresh context."""
    p1 = W.random_problem(801, N=256, n=256, kappa=0.0, boxbc=OK.BOX_DIRICHLET0)
    p2 = W.random_problem(802, N=256, n=256, kappa=0.0, boxbc=OK.BOX_DIRICHLET0, R0=(0.25, 0.45))
    ctx = K.Context(256, p1.box, 0.0, OK.BOX_DIRICHLET0, K.MIXED, max_nodes=256)
    ctx.set_option(K.OPT_FUSE_ROWS, 1)
    ctx.set_interface(dev(p1.xy))
    dens = W.random_density(5, 256, modes=6)
    ctx.apply(K.DOUBLE, dev(dens))
    ctx.set_interface(dev(p2.xy))
    v2, _, _ = ctx.apply(K.DOUBLE, dev(dens))
    fresh = K.Context(256, p2.box, 0.0, OK.BOX_DIRICHLET0, K.MIXED, max_nodes=256)
    fresh.set_option(K.OPT_FUSE_ROWS, 1)
    fresh.set_interface(dev(p2.xy))
    vf, _, _ = fresh.apply(K.DOUBLE, dev(dens))
    assert np.array_equal(v2.cpu().numpy(), vf.cpu().numpy())
    ctx.close()
    fresh.close()


def test_time_column_leaves_applies_unchanged():
    """kfbi_time_column times the selected column kernel on the context's spectral-grid scratch;
    the next apply rewrites that buffer, so its result is bit-identical to the one before."""
    p = W.random_problem(901, N=256, n=200, kappa=0.0, boxbc=OK.BOX_FREESPACE_DL, box=1.5)
    ctx = K.Context(p.N, p.box, 0.0, OK.BOX_FREESPACE_DL, K.MIXED, max_nodes=p.n)
    ctx.set_interface(dev(p.xy))
    dens = dev(W.random_density(9, p.n, modes=6))
    v1, _, _ = ctx.apply(K.DOUBLE, dens)
    t32 = ctx.time_column(True, 20)
    t64 = ctx.time_column(False, 5)
    assert 0.0 < t32 < 1e4 and 0.0 < t64 < 1e5
    v2, _, _ = ctx.apply(K.DOUBLE, dens)
    assert np.array_equal(v1.cpu().numpy(), v2.cpu().numpy())
    with pytest.raises(K.KfbiError):
        ctx.time_column(True, 0)
    ctx.close()
