"""Failure detection on the device: the GMRES and refinement loops run out of their bounds.

The solve loops are CUDA-graph WHILE nodes whose condition the device sets; each has a body
cap after which the solve ends with KFBI_ERR_TIMEOUT. These tests lower the caps
(KFBI_OPT_BODY_CAP, KFBI_OPT_SWEEP_CAP) below what a solve needs, check the status and the
returned iterate, and check that the context keeps working afterwards. No wait is starved and
no fault is provoked: the loop test simply reaches its count.
"""
import numpy as np
import pytest
import torch

import workloads as W

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


def residual(ctx, kind, x, rhs):
    y = ctx.bie_apply(kind, x)
    return float(torch.linalg.norm(rhs - y) / torch.linalg.norm(rhs))


@pytest.mark.parametrize("graphs", [1, 0])
def test_gmres_body_cap_returns_timeout(graphs):
    p = W.config_small_laplace(N=128, n=128)
    ctx = K.Context(p.N, p.box, 0.0, K.BOX_DIRICHLET0, K.FP64, max_nodes=p.n)
    ctx.set_option(K.OPT_CUDA_GRAPHS, graphs)
    ctx.set_interface(dev(p.xy))
    rhs = dev(p.rhs)
    ctx.set_option(K.OPT_BODY_CAP, 9)
    assert ctx.get_option(K.OPT_BODY_CAP) == 9
    x = torch.zeros_like(rhs)
    _, info = ctx.solve_bie(K.BIE_INTERIOR_DL, rhs, density=x, tol=1e-14, max_iter=500, restart=4)
    assert info["status"] == K.ERR_TIMEOUT
    assert info["iterations"] <= 9
    assert bool(torch.isfinite(x).all())
    r = residual(ctx, K.BIE_INTERIOR_DL, x, rhs)
    assert 0.0 < r < 1.0          # the iterate of a completed restart cycle, better than zero
    # the bound lifted, the same context converges
    ctx.set_option(K.OPT_BODY_CAP, 0)
    x2 = torch.zeros_like(rhs)
    _, info2 = ctx.solve_bie(K.BIE_INTERIOR_DL, rhs, density=x2, tol=1e-10, max_iter=500, restart=100)
    assert info2["status"] == K.OK and info2["rel_residual"] <= 1e-10
    ctx.close()


@pytest.mark.parametrize("graphs", [1, 0])
def test_refinement_sweep_cap_returns_timeout(graphs):
    p = W.config_small_laplace(N=128, n=128)
    ctx = K.Context(p.N, p.box, 0.0, K.BOX_DIRICHLET0, K.MIXED, max_nodes=p.n)
    ctx.set_option(K.OPT_CUDA_GRAPHS, graphs)
    ctx.set_interface(dev(p.xy))
    rhs = dev(p.rhs)
    ctx.set_option(K.OPT_SWEEP_CAP, 1)
    x = torch.zeros_like(rhs)
    _, info = ctx.solve_bie(K.BIE_INTERIOR_DL, rhs, density=x, tol=1e-13, max_iter=500, restart=100)
    assert info["status"] == K.ERR_TIMEOUT
    assert bool(torch.isfinite(x).all())
    r = residual(ctx, K.BIE_INTERIOR_DL, x, rhs)
    assert 0.0 < r < 1e-3         # one float32 correction sweep was applied
    ctx.set_option(K.OPT_SWEEP_CAP, 0)
    x2 = torch.zeros_like(rhs)
    _, info2 = ctx.solve_bie(K.BIE_INTERIOR_DL, rhs, density=x2, tol=1e-10, max_iter=500, restart=100)
    assert info2["status"] == K.OK and info2["rel_residual"] <= 1e-10
    ctx.close()


def test_cap_options_reject_negative_values():
    ctx = K.Context(64, (-1.0, 1.0, -1.0, 1.0), 0.0, K.BOX_DIRICHLET0, K.FP64, max_nodes=64)
    for opt in (K.OPT_BODY_CAP, K.OPT_SWEEP_CAP):
        with pytest.raises(K.KfbiError):
            ctx.set_option(opt, -1)
    ctx.close()
