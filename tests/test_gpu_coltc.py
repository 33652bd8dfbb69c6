"""The float32 column solve as two tensor-core contractions (KFBI_OPT_COL_TC, N <= 256).

The transform along y is an N x N matrix (DST-II or DCT-II), the eigenvalue division is the
first contraction's epilogue and the exact inverse (DST-III / DCT-III, weights, 2/N) the second;
both run through kfbi_tc_gemm with split bfloat16 products. The float32 apply of a mixed context
with this path is compared with the same apply through the FFT column kernel (5e-5: both are
float32 forms, each about 3e-5 from the float64 apply) and with the oracle's float64 apply; a mixed solve through it
reaches the float64 tolerance and the oracle's density, and a batch of 128^2 instances with the
option matches the oracle instance by instance.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import kfbi as OK
from oracle.gmres import gmres

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


@pytest.mark.parametrize("N", [16, 64, 128, 256])
@pytest.mark.parametrize("boxbc,kappa,box", [(OK.BOX_DIRICHLET0, 0.0, 1.0), (OK.BOX_NEUMANN0, 30.0, 1.0),
                                             (OK.BOX_FREESPACE_DL, 0.0, 1.5)])
def test_tensor_core_column_solve_apply(N, boxbc, kappa, box):
    n = max(16, min(N, 200))
    R0 = (0.2, 0.3) if N <= 32 else (0.35, 0.55)
    p = W.random_problem(500 + N, N=N, n=n, kappa=kappa, boxbc=boxbc, box=box, R0=R0)
    ctx = K.Context(p.N, p.box, kappa, boxbc, K.MIXED, max_nodes=p.n)
    ctx.set_interface(dev(p.xy))
    dens = W.random_density(N + 1, p.n, modes=6)
    layers = (K.DOUBLE,) if boxbc == OK.BOX_FREESPACE_DL else (K.DOUBLE, K.SINGLE)
    ref = OK.Kfbi(p.N, p.box, kappa, boxbc).set_interface(p.xy)
    for layer in layers:
        v_fft, _, _ = ctx.apply(layer, dev(dens))
        ctx.set_option(K.OPT_COL_TC, 1)
        v_tc, _, _ = ctx.apply(layer, dev(dens))
        ctx.set_option(K.OPT_COL_TC, 0)
        a, b = v_tc.cpu().numpy(), v_fft.cpu().numpy()
        assert np.isfinite(a).all()
        # two float32 forms, each within about 3e-5 of the float64 apply (the float32 sines of the
        # row transform set that): they differ by rounding of that size
        assert rel(a, b) < 5e-5, (layer, rel(a, b))
        rv, _, _ = ref.apply(OK.LAYER_DOUBLE if layer == K.DOUBLE else OK.LAYER_SINGLE, dens)
        assert rel(a, rv) < 2e-4
    ctx.close()


def test_tensor_core_column_solve_mixed_solve_and_capacity():
    p = W.random_problem(43, N=128, n=120)
    ctx = K.Context(p.N, p.box, 0.0, K.BOX_DIRICHLET0, K.MIXED, max_nodes=p.n)
    ctx.set_interface(dev(p.xy))
    ctx.set_option(K.OPT_COL_TC, 1)
    assert ctx.get_option(K.OPT_COL_TC) == 1
    phi, info = ctx.solve_bie(K.BIE_INTERIOR_DL, dev(p.rhs), tol=1e-12, max_iter=400)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-12
    ref = OK.Kfbi(p.N, p.box, 0.0, OK.BOX_DIRICHLET0).set_interface(p.xy)
    x, _ = gmres(lambda v: ref.bie_matvec(OK.BIE_INTERIOR_DL, v), p.rhs, tol=1e-13)
    assert rel(phi.cpu().numpy(), x) < 1e-9
    ctx.close()
    big = K.Context(512, (-1.0, 1.0, -1.0, 1.0), 0.0, K.BOX_DIRICHLET0, K.MIXED, max_nodes=64)
    with pytest.raises(K.KfbiError) as e:
        big.set_option(K.OPT_COL_TC, 1)
    assert e.value.status == K.ERR_CAPACITY
    big.close()


def test_batch_of_small_grids_with_tensor_core_columns():
    """Mixed batch of 128^2 instances with the tensor-core column solve chosen explicitly: per
    instance status and density against the oracle."""
    probs = [W.random_problem(900 + i, N=128, n=int(80 + 10 * i), kappa=[0.0, 10.0][i % 2]) for i in range(4)]
    descs = [dict(N=p.N, box=p.box, kappa=p.kappa, boxbc=K.BOX_DIRICHLET0, max_nodes=p.n) for p in probs]
    b = K.Batch(descs, K.MIXED)
    for c, p in zip(b.contexts, probs):
        c.set_interface(dev(p.xy))
        c.set_option(K.OPT_COL_TC, 1)
    rhs = [dev(p.rhs) for p in probs]
    dens = [torch.zeros(p.n, dtype=torch.float64, device="cuda") for p in probs]
    _, infos = b.solve(K.BIE_INTERIOR_DL, rhs, dens, tol=1e-11, max_iter=400, restart=100)
    for p, d, info in zip(probs, dens, infos):
        assert info["status"] == 0
        ref = OK.Kfbi(p.N, p.box, p.kappa, OK.BOX_DIRICHLET0).set_interface(p.xy)
        x, _ = gmres(lambda v: ref.bie_matvec(OK.BIE_INTERIOR_DL, v), p.rhs, tol=1e-13)
        assert rel(d.cpu().numpy(), x) < 1e-9
    b.close()
