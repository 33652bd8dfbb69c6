"""kfbi_grid_solve_mixed: the box solve (Delta_h - kappa) u = rhs (Sec. 4.2) as float32 solves
with float64 residual corrections, against the oracle's float64 solve (DST-II / DCT-II by
scipy), and the Stefan step with its two grid solves done that way (KFBI_OPT_GRID_IR) against
the float64 grid solves.

Tolerances: one float32 solve is accurate to ~1e-6 of max |u| (float32 transforms of
length N, float32 sines); every correction multiplies the error by about that factor, down to
the float64 residual's rounding (~1e-16 times the operator's condition number, ~1e-13 for the
largest kappa h^2 ratio used here).
"""
import numpy as np
import pytest
import torch

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


CASES = [(OK.BOX_DIRICHLET0, 0.0, 1.0), (OK.BOX_DIRICHLET0, 40.0, 1.0), (OK.BOX_NEUMANN0, 20.0, 1.0),
         (OK.BOX_NEUMANN0, 3000.0, 2.0)]


@pytest.mark.parametrize("N", [32, 64, 256, 1024])
@pytest.mark.parametrize("boxbc,kappa,half", CASES)
def test_grid_solve_mixed_matches_oracle(N, boxbc, kappa, half):
    rng = np.random.default_rng(N + 11 * boxbc + int(kappa))
    C = rng.standard_normal((N, N))
    ctx = K.Context(N, (-half, half, -half, half), kappa, boxbc, K.MIXED, max_nodes=64)
    ref = OK.solve_grid(OK.Grid(N, (-half, half, -half, half)), C, kappa, boxbc)
    errs = []
    for sweeps in (0, 1, 2, 3):
        u = ctx.grid_solve_mixed(dev(C), sweeps).cpu().numpy()
        assert np.isfinite(u).all()
        errs.append(rel(u, ref))
    assert errs[0] < 1e-4, errs
    assert errs[1] < 1e-8, errs
    assert errs[2] < 1e-11, errs
    assert errs[3] < 1e-11, errs
    # the float64 solve of the same context, for scale
    u64 = ctx.grid_solve(dev(C)).cpu().numpy()
    assert rel(u64, ref) < 1e-12
    ctx.close()


def test_grid_solve_mixed_smooth_rhs_and_arguments():
    """A smooth right-hand side with a jump (the Stefan step's BDF2 data: T = St outside a
    disc, 0 inside), and the argument checks."""
    N, half, kappa = 512, 2.0, 3000.0
    g = OK.Grid(N, (-half, half, -half, half))
    X, Y = np.meshgrid(g.x, g.y)
    T = np.where(X ** 2 + Y ** 2 < 0.3 ** 2, 0.0, -0.5)
    rhs = -3.0 * T / (2 * 5e-4)
    ctx = K.Context(N, (-half, half, -half, half), kappa, OK.BOX_NEUMANN0, K.MIXED, max_nodes=64)
    ref = OK.solve_grid(g, rhs, kappa, OK.BOX_NEUMANN0)
    u = ctx.grid_solve_mixed(dev(rhs), 2).cpu().numpy()
    assert rel(u, ref) < 1e-11
    r = dev(rhs)
    with pytest.raises(K.KfbiError):
        ctx.grid_solve_mixed(r, 2, out=r)  # aliasing
    with pytest.raises(K.KfbiError):
        ctx.grid_solve_mixed(r, 9)
    # a wrong output buffer is refused before the library is called
    for bad in (torch.empty((N, N), dtype=torch.float32, device="cuda"),
                torch.empty((N, N - 1), dtype=torch.float64, device="cuda")):
        with pytest.raises(ValueError):
            ctx.grid_solve_mixed(r, 2, out=bad)
        with pytest.raises(ValueError):
            ctx.grid_solve(r, out=bad)
    assert ctx.get_option(K.OPT_GRID_IR) == 2
    for v in (0, 1, 3, 2):
        ctx.set_option(K.OPT_GRID_IR, v)
        assert ctx.get_option(K.OPT_GRID_IR) == v
    for bad in (-1, 9):
        with pytest.raises(K.KfbiError):
            ctx.set_option(K.OPT_GRID_IR, bad)
    ctx.close()
    c64 = K.Context(64, (-1.0, 1.0, -1.0, 1.0), 1.0, OK.BOX_NEUMANN0, K.FP64, max_nodes=64)
    with pytest.raises(K.KfbiError):
        c64.grid_solve_mixed(dev(np.ones((64, 64))), 2)
    c64.close()


def test_grid_solve_mixed_largest_grid():
    """N = 4096 (the largest grid; the float32 row kernels need more than the default shared
    memory there), Neumann box, kappa = 3000: against the oracle."""
    N, half, kappa = 4096, 2.0, 3000.0
    g = OK.Grid(N, (-half, half, -half, half))
    X, Y = np.meshgrid(g.x, g.y)
    rhs = np.cos(3 * X) * np.exp(-Y * Y) + np.where(X ** 2 + Y ** 2 < 0.25, 1.0, 0.0)
    ctx = K.Context(N, (-half, half, -half, half), kappa, OK.BOX_NEUMANN0, K.MIXED, max_nodes=64)
    ref = OK.solve_grid(g, rhs, kappa, OK.BOX_NEUMANN0)
    u = ctx.grid_solve_mixed(dev(rhs), 2).cpu().numpy()
    assert rel(u, ref) < 1e-11
    ctx.close()


def test_stefan_step_with_mixed_grid_solve():
    """Two mixed Stefan steps (2048^2 grid, 2048 nodes, tol 1e-9) from the same state with the
    two grid solves (T1, and the single layer's grid values T2 from the float64 jumps) by
    KFBI_OPT_GRID_IR = 2 and by float64 solves: temperature, density and angles agree to what
    the 1e-9 solve tolerance leaves."""
    import bench as B
    import workloads as W

    p = W.config_stefan(N=2048, n=2048)
    x = p.extra
    outs = []
    for ir in (2, 0):
        ctx = K.Context(p.N, p.box, p.kappa, K.BOX_NEUMANN0, K.MIXED, max_nodes=p.n)
        ctx.set_option(K.OPT_GRID_IR, ir)
        eta = torch.tensor(p.theta - B.alpha_array(p.n), dtype=torch.float64, device="cuda")
        st = K.ThetaL(ctx, eta, p.L, p.xy.mean(0), K.STEP_STEFAN, tol=1e-9, max_iter=3000, restart=150,
                      St=x["St"], eps_c=x["eps_c"], eps_aniso=x["eps_aniso"], eps_v=x["eps_v"], fold=x["fold"])
        infos = [st.step(x["dt"]) for _ in range(2)]
        assert all(i["status"] == 0 for i in infos)
        r = st.read(T=True)
        outs.append({k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in r.items()})
        st.close()
        ctx.close()
    a, b = outs
    assert rel(a["T"], b["T"]) < 1e-9
    assert rel(a["density"], b["density"]) < 1e-6
    assert np.abs(a["eta"] - b["eta"]).max() < 1e-8


def test_refined_float64_apply_on_the_largest_grid():
    """N = 4096, Dirichlet box, interior double-layer problem in a mixed context: the float64
    applies of the refinement solve their grid by float32 solves with float64 residual sweeps
    (KFBI_OPT_GRID_IR = 2) or by the float64 column solve (0); both meet the 1e-11 residual
    and give the same density to what that residual allows, and match the float64 context."""
    import workloads as W

    rng = np.random.default_rng(17)
    p = W.interior_dirichlet(W.random_star(rng), 4096, 512, kappa=0.0, name="big")
    dens = {}
    for ir in (2, 0):
        ctx = K.Context(p.N, p.box, 0.0, K.BOX_DIRICHLET0, K.MIXED, max_nodes=p.n)
        ctx.set_option(K.OPT_GRID_IR, ir)
        ctx.set_interface(dev(p.xy))
        phi, info = ctx.solve_bie(K.BIE_INTERIOR_DL, dev(p.rhs), tol=1e-11, max_iter=300, restart=100)
        assert info["status"] == 0 and info["rel_residual"] <= 1e-11
        dens[ir] = phi.cpu().numpy()
        ctx.close()
    c64 = K.Context(p.N, p.box, 0.0, K.BOX_DIRICHLET0, K.FP64, max_nodes=p.n)
    c64.set_interface(dev(p.xy))
    phi64, info64 = c64.solve_bie(K.BIE_INTERIOR_DL, dev(p.rhs), tol=1e-11, max_iter=300, restart=100)
    c64.close()
    assert rel(dens[2], dens[0]) < 1e-9
    assert rel(dens[2], phi64.cpu().numpy()) < 1e-9


def test_refined_apply_with_one_sweep_meets_the_tolerance():
    """A mixed solve to 1e-8 on a 4096^2 grid refines its float64 applies' grid solve with one
    correction sweep: the returned density's residual under the float64 context's operator
    (float64 column solve) still meets the tolerance, and the iteration count matches the
    two-sweep form within one."""
    import workloads as W

    rng = np.random.default_rng(23)
    p = W.interior_dirichlet(W.random_star(rng), 4096, 512, kappa=0.0, name="big")
    c64 = K.Context(p.N, p.box, 0.0, K.BOX_DIRICHLET0, K.FP64, max_nodes=p.n)
    c64.set_interface(dev(p.xy))
    b = dev(p.rhs)
    its = {}
    for ir in (2, 0):
        ctx = K.Context(p.N, p.box, 0.0, K.BOX_DIRICHLET0, K.MIXED, max_nodes=p.n)
        ctx.set_option(K.OPT_GRID_IR, ir)
        ctx.set_interface(dev(p.xy))
        phi, info = ctx.solve_bie(K.BIE_INTERIOR_DL, b, tol=1e-8, max_iter=300, restart=100)
        assert info["status"] == 0
        its[ir] = info["iterations"]
        r = b - c64.bie_apply(K.BIE_INTERIOR_DL, phi)
        assert float(r.norm() / b.norm()) <= 1.05e-8, (ir, float(r.norm() / b.norm()))
        ctx.close()
    c64.close()
    assert abs(its[2] - its[0]) <= 1, its
