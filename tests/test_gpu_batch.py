"""Batched solves (one graph launch for many instances) vs single-instance solves and the
oracle, through the C ABI; the autotuner's choices are valid and keep the results.

Each instance of a batch runs the kernels of kfbi_solve_bie on its own data, so the batch
density equals the single-instance density to rounding (1e-13 relative: the two graphs run
the same kernels, only their interleaving on the GPU differs), and both equal the oracle's
GMRES density to the tolerance of the solve.
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
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def instances(count, seed=7):
    """Uneven small instances: N in {64, 128}, node counts that keep the spacing above h,
    kappa in {0, 10} (interior Dirichlet, data from the exact interior solution)."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed + i)
        N = int(rng.choice([64, 128]))
        n = int(rng.integers(40, 70 if N == 64 else 130))
        kappa = float(rng.choice([0.0, 10.0]))
        out.append(W.random_problem(seed * 100 + i, N=N, n=n, kappa=kappa))
    return out


def make_batch(probs, precision):
    descs = [dict(N=p.N, box=p.box, kappa=p.kappa, boxbc=K.BOX_DIRICHLET0, max_nodes=p.n) for p in probs]
    b = K.Batch(descs, precision)
    for c, p in zip(b.contexts, probs):
        c.set_interface(dev(p.xy))
    return b


@pytest.mark.parametrize("precision,tol", [(0, 1e-13), (1, 1e-10)])
def test_batch_matches_single_solves_and_oracle(precision, tol):
    probs = instances(9)
    b = make_batch(probs, precision)
    rhs = [dev(p.rhs) for p in probs]
    dens = [torch.zeros(p.n, dtype=torch.float64, device="cuda") for p in probs]
    st, infos = b.solve(K.BIE_INTERIOR_DL, rhs, dens, tol=tol, max_iter=400, restart=100)
    assert st == 0 and all(i["status"] == 0 and i["rel_residual"] <= tol for i in infos)
    for c, p, d, inf in zip(b.contexts, probs, dens, infos):
        single, si = c.solve_bie(K.BIE_INTERIOR_DL, dev(p.rhs), tol=tol, max_iter=400, restart=100)
        assert si["iterations"] == inf["iterations"]
        assert rel(d.cpu().numpy(), single.cpu().numpy()) < 1e-13
        ref = OK.Kfbi(p.N, p.box, p.kappa, OK.BOX_DIRICHLET0).set_interface(p.xy)
        rphi, _ = gmres(lambda v: ref.bie_matvec(OK.BIE_INTERIOR_DL, v), p.rhs, tol=1e-13)
        assert rel(d.cpu().numpy(), rphi) < (1e-9 if precision == 0 else 1e-8)
    # the same buffers again: the cached graph, the same answer from the converged start
    st2, infos2 = b.solve(K.BIE_INTERIOR_DL, rhs, dens, tol=tol, max_iter=400, restart=100)
    assert st2 == 0 and all(i["iterations"] <= 1 for i in infos2)


def test_batch_autotune_choices_are_valid_and_results_unchanged():
    probs = instances(6, seed=11)
    b = make_batch(probs, K.MIXED)
    rhs = [dev(p.rhs) for p in probs]
    ms = b.autotune(K.BIE_INTERIOR_DL, rhs, tol=1e-10, max_iter=400, restart=100)
    assert ms > 0.0
    for c in b.contexts:
        assert c.get_option(K.OPT_CLUSTER_GMRES) in (0, 1)
        assert c.get_option(K.OPT_CLUSTER_SIZE) in (0, 8, 16)
        assert c.get_option(K.OPT_COL_PAIRS) in (0, 1, 2, 4)
        assert c.get_option(K.OPT_COL_RADIX4) in (2, 3)
    dens = [torch.zeros(p.n, dtype=torch.float64, device="cuda") for p in probs]
    st, infos = b.solve(K.BIE_INTERIOR_DL, rhs, dens, tol=1e-10, max_iter=400, restart=100)
    assert st == 0
    for p, d in zip(probs, dens):
        ref = OK.Kfbi(p.N, p.box, p.kappa, OK.BOX_DIRICHLET0).set_interface(p.xy)
        rphi, _ = gmres(lambda v: ref.bie_matvec(OK.BIE_INTERIOR_DL, v), p.rhs, tol=1e-13)
        assert rel(d.cpu().numpy(), rphi) < 1e-8


def test_batch_errors():
    probs = instances(2, seed=13)
    descs = [dict(N=p.N, box=p.box, kappa=p.kappa, boxbc=K.BOX_DIRICHLET0, max_nodes=p.n) for p in probs]
    b = K.Batch(descs, K.FP64)
    b.contexts[0].set_interface(dev(probs[0].xy))
    rhs = [dev(p.rhs) for p in probs]
    dens = [torch.zeros(p.n, dtype=torch.float64, device="cuda") for p in probs]
    with pytest.raises(K.KfbiError) as e:
        b.solve(K.BIE_INTERIOR_DL, rhs, dens)
    assert e.value.status == K.ERR_STATE  # instance 1 has no interface
    b.contexts[1].set_interface(dev(probs[1].xy))
    with pytest.raises(K.KfbiError) as e:
        b.solve(K.BIE_STEFAN_SL, rhs, dens)
    assert e.value.status == K.ERR_ARG
