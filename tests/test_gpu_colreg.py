"""The float32 column solve with its FFTs in registers (KFBI_OPT_COL_REG, N <= 1024).

The float32 apply of a mixed context with the register kernel is compared with the same apply
through the shared-memory Stockham kernel (both float32: they differ by rounding order only) and
with the oracle's float64 apply, for every grid size the kernel covers, for the three boxes
(Dirichlet DST-II, Neumann DCT-II, free-space box data that exercises the rows the row
transform leaves to the column kernel).
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


BOXES = [(OK.BOX_DIRICHLET0, 0.0, 1.0), (OK.BOX_NEUMANN0, 30.0, 1.0), (OK.BOX_FREESPACE_DL, 0.0, 1.5)]


@pytest.mark.parametrize("N", [16, 32, 64, 128, 256, 512, 1024])
@pytest.mark.parametrize("boxbc,kappa,box", BOXES)
def test_register_column_kernel_apply(N, boxbc, kappa, box):
    n = max(16, min(N, 256))
    R0 = (0.2, 0.3) if N <= 32 else (0.35, 0.55)
    p = W.random_problem(300 + N, N=N, n=n, kappa=kappa, boxbc=boxbc, box=box, R0=R0)
    ctx = K.Context(p.N, p.box, kappa, boxbc, K.MIXED, max_nodes=p.n)
    ctx.set_interface(dev(p.xy))
    ctx.set_option(K.OPT_COL_REG, 1)
    dens = W.random_density(N, p.n, modes=6)
    layers = (K.DOUBLE,) if boxbc == OK.BOX_FREESPACE_DL else (K.DOUBLE, K.SINGLE)
    ref = OK.Kfbi(p.N, p.box, kappa, boxbc).set_interface(p.xy)
    for layer in layers:
        v_reg, _, _ = ctx.apply(layer, dev(dens))
        ctx.set_option(K.OPT_COL_REG, 0)
        v_stk, _, _ = ctx.apply(layer, dev(dens))
        ctx.set_option(K.OPT_COL_REG, 1)
        a, b = v_reg.cpu().numpy(), v_stk.cpu().numpy()
        assert np.isfinite(a).all()
        assert rel(a, b) < 2e-5, (layer, rel(a, b))
        rv, _, _ = ref.apply(OK.LAYER_DOUBLE if layer == K.DOUBLE else OK.LAYER_SINGLE, dens)
        assert rel(a, rv) < 2e-4, (layer, rel(a, rv))
    ctx.close()


@pytest.mark.parametrize("boxbc,kappa,box", BOXES[:2])
def test_register_column_kernel_mixed_solve(boxbc, kappa, box):
    """A mixed solve whose inner applies use the register kernel reaches the float64 tolerance
    and agrees with the oracle's solution."""
    p = W.random_problem(41, N=256, n=200, kappa=kappa, boxbc=boxbc, box=box)
    ctx = K.Context(p.N, p.box, kappa, boxbc, K.MIXED, max_nodes=p.n)
    ctx.set_interface(dev(p.xy))
    ctx.set_option(K.OPT_COL_REG, 1)
    kind = K.BIE_INTERIOR_DL if boxbc == OK.BOX_DIRICHLET0 else K.BIE_STEFAN_SL
    ev = dev(np.full(p.n, 2e-3)) if kind == K.BIE_STEFAN_SL else None
    phi, info = ctx.solve_bie(kind, dev(p.rhs), tol=1e-12, max_iter=400, eps_v=ev)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-12
    ref = OK.Kfbi(p.N, p.box, kappa, boxbc).set_interface(p.xy)
    from oracle.gmres import gmres

    e = np.full(p.n, 2e-3)
    x, _ = gmres(lambda v: ref.bie_matvec(kind, v, eps_v=e), p.rhs, tol=1e-13)
    assert rel(phi.cpu().numpy(), x) < 1e-9
    ctx.close()
