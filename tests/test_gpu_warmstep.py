"""The learned warm start inside the time step (kfbi_thetal_set_warmstart), on the Stefan
single-layer equation.

A network is trained by the library's own kernels on (features, density) pairs that the Stefan
steps themselves produce (kfbi_thetal_training_pair). From one checkpoint the same steps then
run twice: from the previous step's density (the default start) and with the network attached,
where each step starts from whichever of the two guesses has the smaller float64 residual.
GMRES iterates to the same tolerance either way, so the densities and the curves agree to
that tolerance; the test asserts that agreement, that the step took the start with the smaller
residual (by construction never more iterations than a margin for rounding) and reports the
iteration counts of both runs.
"""
import math

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


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def make_stefan(N=256, n=256, dt=1e-4, tol=1e-10):
    p = W.config_stefan(N=N, n=n, box=0.5, dt=dt)
    x = p.extra
    ctx = K.Context(p.N, p.box, p.kappa, K.BOX_NEUMANN0, K.FP64, max_nodes=p.n)
    alpha = 2 * math.pi * np.arange(p.n) / p.n
    st = K.ThetaL(ctx, dev(p.theta - alpha), p.L, p.xy.mean(0), K.STEP_STEFAN, tol=tol, max_iter=2000, restart=150,
                  St=x["St"], eps_c=x["eps_c"], eps_aniso=x["eps_aniso"], eps_v=x["eps_v"], fold=x["fold"])
    return p, ctx, st


def test_learned_warm_start_in_the_step():
    p, ctx, st = make_stefan()
    dt = p.extra["dt"]
    feats, targets = [], []
    for _ in range(30):
        info = st.step(dt)
        assert info["status"] == 0
        f, t = st.training_pair()
        feats.append(f.clone())
        targets.append(t.clone())
    X, T = torch.cat(feats), torch.cat(targets)
    m = K.Mlp(hidden=128, max_rows=max(X.shape[0], p.n))
    m.set_params(W.mlp_init(5, hidden=128))
    g = torch.Generator(device="cpu").manual_seed(1)
    first, _ = m.gradients(X, T)
    for it in range(1500):
        idx = torch.randint(0, X.shape[0], (512,), generator=g, dtype=torch.int32).cuda()
        m.train_step(X, T, idx=idx, lr=1e-3 if it < 1000 else 3e-4, want_loss=False)
    last, _ = m.gradients(X, T)
    assert last < 0.2 * first, (first, last)
    ck = st.read(T=True)
    ck = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in ck.items()}

    def run(with_net):
        st.write(eta=ck["eta"], density=ck["density"], nhat=ck["nhat"], T=ck["T"], T_prev=ck["T_prev"],
                 scalars=ck["scalars"])
        st.set_warmstart(m if with_net else None)
        its, dens = [], []
        for _ in range(6):
            info = st.step(dt)
            assert info["status"] == 0
            its.append(info["iterations"])
            dens.append(st.read(T=False)["density"].clone())
        out = st.read(T=True)
        st.set_warmstart(None)
        return its, dens, out

    its0, d0, o0 = run(False)
    its1, d1, o1 = run(True)
    wins = int(o1["scalars"][14] - ck["scalars"][14])
    print(f"warm start in the Stefan step: iterations previous-step start {its0}, with the network {its1}; "
          f"network start taken in {wins} of 6 steps; training loss {first:.3e} -> {last:.3e}")
    for a, b in zip(d0, d1):
        assert float((a - b).abs().max() / b.abs().max()) < 1e-7
    assert float((o0["eta"] - o1["eta"]).abs().max()) < 1e-9
    assert float((o0["T"] - o1["T"]).abs().max() / o0["T"].abs().max()) < 1e-8
    # the start with the smaller residual never costs more than rounding-level extra iterations
    assert sum(its1) <= sum(its0) + len(its0), (its0, its1)
    st.close()
    ctx.close()
