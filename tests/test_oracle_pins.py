"""Pins for the CPU oracle: each test checks it against something other than itself.

- the DST/DCT solve against a dense five-point matrix built from the stencil;
- the jump formulas (App. A.1) against the exact jumps of two closed-form pieces;
- the corrected scheme (Sec. 4.2) against the local truncation error of the same pieces;
- the 6-point jump-corrected interpolation (Sec. 4.3) against quadratic exactness;
- the double layer of a constant density (Table 2 jump, Gauss: D1 = indicator);
- circle spectra in free space (D e^{ik a} = 0, k != 0) and for the modified Helmholtz
  single layer (-R I_k(cR) K_k(cR), scipy.special);
- second-order convergence of the interior Dirichlet problem with u = e^x sin y;
- GMRES against a dense LU solve of the assembled operator.
"""
import math

import numpy as np
import pytest
import scipy.special as sp

import workloads as W
from oracle import kfbi as K
from oracle.gmres import gmres


# ---------------------------------------------------------------- helpers
def dense_five_point(N, h, kappa, boxbc):
    """The 5-point matrix of (Delta_h - kappa) with ghost cells u_{-1} = -u_0 (Dirichlet-0)
    or u_{-1} = u_0 (Neumann-0), assembled entry by entry."""
    A = np.zeros((N * N, N * N))
    gs = -1.0 if boxbc != K.BOX_NEUMANN0 else 1.0
    for j in range(N):
        for i in range(N):
            r = j * N + i
            A[r, r] += -4.0 / h ** 2 - kappa
            for dj, di in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                jj, ii = j + dj, i + di
                if 0 <= jj < N and 0 <= ii < N:
                    A[r, jj * N + ii] += 1.0 / h ** 2
                else:
                    A[r, r] += gs / h ** 2
    return A


def plain_ellipse_nodes(a, b, n, cx=0.0, cy=0.0):
    t = 2 * math.pi * np.arange(n) / n
    return np.stack([cx + a * np.cos(t), cy + b * np.sin(t)], -1)


def pieces(kappa):
    """Two closed-form solutions of (Delta - kappa) u = 0 with all second derivatives."""
    if kappa == 0.0:
        def up(x, y):
            e = np.exp(x)
            s, c = np.sin(y), np.cos(y)
            return dict(u=e * s, ux=e * s, uy=e * c, uxx=e * s, uyy=-e * s, uxy=e * c)

        def um(x, y):
            z = np.zeros_like(x)
            return dict(u=x * x - y * y, ux=2 * x, uy=-2 * y, uxx=z + 2, uyy=z - 2, uxy=z)
    else:
        a = math.sqrt(kappa + 1.0)
        r = math.sqrt(kappa)

        def up(x, y):
            e = np.exp(a * x)
            s, c = np.sin(y), np.cos(y)
            return dict(u=e * s, ux=a * e * s, uy=e * c, uxx=a * a * e * s, uyy=-e * s, uxy=a * e * c)

        def um(x, y):
            z = np.zeros_like(x)
            return dict(u=np.cosh(r * x), ux=r * np.sinh(r * x), uy=z, uxx=kappa * np.cosh(r * x), uyy=z, uxy=z)
    return up, um


def exact_jump_data(iface, up, um):
    g = iface.node
    P = up(g["x"], g["y"])
    M = um(g["x"], g["y"])
    Phi = P["u"] - M["u"]
    Psi = g["nx"] * (P["ux"] - M["ux"]) + g["ny"] * (P["uy"] - M["uy"])
    return Phi, Psi


# ---------------------------------------------------------------- solver
@pytest.mark.parametrize("N", [12, 16])
@pytest.mark.parametrize("boxbc,kappa", [(K.BOX_DIRICHLET0, 0.0), (K.BOX_DIRICHLET0, 7.5),
                                         (K.BOX_NEUMANN0, 3.0)])
def test_solver_equals_dense_five_point(N, boxbc, kappa):
    grid = K.Grid(N, (-1.0, 1.5, -0.5, 2.0))
    rng = np.random.default_rng(5)
    C = rng.standard_normal((N, N))
    u = K.solve_grid(grid, C, kappa, boxbc)
    A = dense_five_point(N, grid.h, kappa, boxbc)
    ref = np.linalg.solve(A, C.ravel()).reshape(N, N)
    assert np.abs(u - ref).max() <= 1e-12 * np.abs(ref).max()


def test_neumann_laplace_is_singular():
    with pytest.raises(K.Singular):
        K.Kfbi(16, (-1, 1, -1, 1), 0.0, K.BOX_NEUMANN0)


def test_box_data_ghost_rule():
    """Dirichlet data g on a face enters as -2 g / h^2: a linear function is reproduced."""
    N = 16
    grid = K.Grid(N, (-1.0, 1.0, -1.0, 1.0))
    f = lambda x, y: 0.3 + 2.0 * x - 1.5 * y  # harmonic, 5-point exact
    W_, E_, S_, N_ = K.box_face_points(grid)
    C = np.zeros((N, N))
    C = K.add_box_data(grid, C, f(*W_.T), f(*E_.T), f(*S_.T), f(*N_.T))
    u = K.solve_grid(grid, C, 0.0, K.BOX_DIRICHLET0)
    X, Y = np.meshgrid(grid.x, grid.y)
    assert np.abs(u - f(X, Y)).max() < 1e-12


# ---------------------------------------------------------------- interpolant
def test_trig_interpolant_derivatives():
    for n in (15, 16):
        a = 2 * math.pi * np.arange(n) / n
        f = 0.7 + np.cos(3 * a) - 0.4 * np.sin(5 * a)
        T = K.Trig(f)
        t = np.linspace(0.1, 6.0, 37)
        assert np.abs(T.eval(t, 0) - (0.7 + np.cos(3 * t) - 0.4 * np.sin(5 * t))).max() < 1e-13
        assert np.abs(T.eval(t, 1) - (-3 * np.sin(3 * t) - 2.0 * np.cos(5 * t))).max() < 1e-12
        assert np.abs(T.eval(t, 2) - (-9 * np.cos(3 * t) + 10.0 * np.sin(5 * t))).max() < 1e-11
    # Nyquist mode is the real cosine
    n = 8
    a = 2 * math.pi * np.arange(n) / n
    T = K.Trig(np.cos(4 * a))
    t = np.array([0.3, 1.1])
    assert np.abs(T.eval(t, 0) - np.cos(4 * t)).max() < 1e-14
    assert np.abs(T.eval(t, 1) + 4 * np.sin(4 * t)).max() < 1e-13


# ---------------------------------------------------------------- jumps (App. A.1)
@pytest.mark.parametrize("kappa", [0.0, 10.0])
def test_jumps_match_closed_form(kappa):
    iface = K.Interface(plain_ellipse_nodes(0.5, 0.3, 96, 0.05, -0.02))
    up, um = pieces(kappa)
    Phi, Psi = exact_jump_data(iface, up, um)
    alpha = np.concatenate([iface.alpha, np.linspace(0.01, 6.2, 41)])
    J = K.jumps_from_data(iface, alpha, Phi, Psi, kappa)
    g = iface.geom(alpha)
    P = up(g["x"], g["y"])
    M = um(g["x"], g["y"])
    for col, key in enumerate(["u", "ux", "uy", "uxx", "uyy", "uxy"]):
        exact = P[key] - M[key]
        assert np.abs(J[:, col] - exact).max() < 5e-10 * max(1.0, np.abs(exact).max()), key


def test_layer_jump_table():
    """Table 2: D phi has [u] = phi, [du/dn] = 0; S psi has [u] = 0, [du/dn] = -psi."""
    iface = K.Interface(plain_ellipse_nodes(0.5, 0.3, 64))
    dens = W.random_density(3, 64)
    g = iface.node
    Jd = K.jumps(iface, iface.alpha, K.LAYER_DOUBLE, dens, 0.0)
    assert np.abs(Jd[:, 0] - dens).max() < 1e-13
    assert np.abs(g["nx"] * Jd[:, 1] + g["ny"] * Jd[:, 2]).max() < 1e-12
    Js = K.jumps(iface, iface.alpha, K.LAYER_SINGLE, dens, 0.0)
    assert np.abs(Js[:, 0]).max() == 0.0
    assert np.abs(g["nx"] * Js[:, 1] + g["ny"] * Js[:, 2] + dens).max() < 1e-12


# ---------------------------------------------------------------- corrected scheme (Sec. 4.2)
@pytest.mark.parametrize("kappa", [0.0, 10.0])
def test_correction_matches_truncation_error(kappa):
    """(Delta_h - kappa) u - C is O(h) at irregular nodes, while (Delta_h - kappa) u is O(h^-2)."""
    up, um = pieces(kappa)
    res = []
    for N in (64, 128):
        solver = K.Kfbi(N, (-1, 1, -1, 1), kappa, K.BOX_DIRICHLET0)
        solver.set_interface(plain_ellipse_nodes(0.55, 0.35, 128, 0.03, 0.01))
        Phi, Psi = exact_jump_data(solver.iface, up, um)
        Jc = K.jumps_from_data(solver.iface, solver.cr.alpha, Phi, Psi, kappa)
        C = K.correction_rhs(solver.grid, solver.cr, solver.cl, Jc)
        X, Y = np.meshgrid(solver.grid.x, solver.grid.y)
        u = np.where(solver.cl.side == 1, up(X, Y)["u"], um(X, Y)["u"])
        h = solver.grid.h
        L = np.zeros_like(u)
        L[1:-1, 1:-1] = (u[1:-1, 2:] + u[1:-1, :-2] + u[2:, 1:-1] + u[:-2, 1:-1] - 4 * u[1:-1, 1:-1]) / h ** 2
        L -= kappa * u
        irr = solver.cl.irregular.copy()
        irr[[0, -1], :] = False
        irr[:, [0, -1]] = False
        raw = np.abs(L[irr]).max()
        r = np.abs(L[irr] - C[irr]).max()
        assert raw > 50.0 * r
        res.append(r)
    assert res[1] < 0.75 * res[0]


# ---------------------------------------------------------------- interpolation (Sec. 4.3)
def test_interpolation_quadratic_exact():
    solver = K.Kfbi(64, (-1, 1, -1, 1), 0.0, K.BOX_DIRICHLET0)
    solver.set_interface(plain_ellipse_nodes(0.5, 0.4, 80))
    P = lambda x, y: 1.0 + 0.5 * x - 0.25 * y + 0.3 * x * x - 0.7 * x * y + 0.2 * y * y
    Q = lambda x, y: -0.5 + 2.0 * x + 1.0 * y - 0.1 * x * x + 0.4 * x * y + 0.9 * y * y
    X, Y = np.meshgrid(solver.grid.x, solver.grid.y)
    u = np.where(solver.cl.side == 1, P(X, Y), Q(X, Y))
    p = solver.iface.xy
    x, y = p[:, 0], p[:, 1]
    Jn = np.stack([P(x, y) - Q(x, y),
                   (0.5 + 0.6 * x - 0.7 * y) - (2.0 - 0.2 * x + 0.4 * y),
                   (-0.25 - 0.7 * x + 0.4 * y) - (1.0 + 0.4 * x + 1.8 * y),
                   np.full_like(x, 0.6 - (-0.2)), np.full_like(x, 0.4 - 1.8), np.full_like(x, -0.7 - 0.4)], -1)
    g = solver.iface.node
    val, dn = K.interpolate(solver.st, u, Jn, g["nx"], g["ny"])
    assert np.abs(val - 0.5 * (P(x, y) + Q(x, y))).max() < 1e-12
    gx = 0.5 * ((0.5 + 0.6 * x - 0.7 * y) + (2.0 - 0.2 * x + 0.4 * y))
    gy = 0.5 * ((-0.25 - 0.7 * x + 0.4 * y) + (1.0 + 0.4 * x + 1.8 * y))
    assert np.abs(dn - (g["nx"] * gx + g["ny"] * gy)).max() < 1e-10


# ---------------------------------------------------------------- constant density (Table 2, Gauss)
@pytest.mark.parametrize("boxbc,box", [(K.BOX_DIRICHLET0, 1.0), (K.BOX_FREESPACE_DL, 1.5)])
def test_double_layer_of_one_is_indicator(boxbc, box):
    p = W.random_problem(11, N=96, n=96, box=box)
    solver = K.Kfbi(p.N, p.box, 0.0, boxbc).set_interface(p.xy)
    val, dn, u = solver.apply(K.LAYER_DOUBLE, np.ones(p.n), want_dnormal=True)
    assert np.abs(u - solver.cl.side).max() < 1e-12
    assert np.abs(val - 0.5).max() < 1e-12
    assert np.abs(dn).max() < 1e-10


# ---------------------------------------------------------------- circle spectra
def test_free_space_double_layer_circle_spectrum():
    nodes = W.equal_arclength(W.ellipse(1.0, 1.0), 128)
    a = 2 * math.pi * np.arange(128) / 128
    errs = []
    for N in (128, 256):
        s = K.Kfbi(N, (-4, 4, -4, 4), 0.0, K.BOX_FREESPACE_DL).set_interface(nodes["xy"])
        v, _, _ = s.apply(K.LAYER_DOUBLE, np.cos(3 * a) + 0.5)
        errs.append(np.abs(v - 0.25).max())
    assert errs[0] < 2e-3 and errs[1] < 0.35 * errs[0]


def test_modified_helmholtz_single_layer_circle_spectrum():
    R, kap, k = 0.5, 400.0, 3
    c = math.sqrt(kap)
    nodes = W.equal_arclength(W.ellipse(R, R), 128)
    a = 2 * math.pi * np.arange(128) / 128
    exact = -R * sp.ive(k, c * R) * sp.kve(k, c * R) * np.cos(k * a)
    exact0 = -R * sp.ive(0, c * R) * sp.kve(0, c * R)
    errs = []
    for N in (128, 256):
        s = K.Kfbi(N, (-2, 2, -2, 2), kap, K.BOX_NEUMANN0).set_interface(nodes["xy"])
        v, _, _ = s.apply(K.LAYER_SINGLE, np.cos(k * a) + 1.0)
        errs.append(np.abs(v - exact - exact0).max() / abs(exact0))
    assert errs[0] < 4e-2 and errs[1] < 0.35 * errs[0]


# ---------------------------------------------------------------- convergence
def test_interior_dirichlet_second_order():
    errs, hs = [], []
    for N in (32, 64, 128, 256):
        p = W.config_small_laplace(N=N, n=max(64, N))
        s = K.Kfbi(p.N, p.box, 0.0, K.BOX_DIRICHLET0).set_interface(p.xy)
        phi, info = gmres(lambda x: s.bie_matvec(K.BIE_INTERIOR_DL, x), p.rhs, tol=1e-12)
        assert info["converged"]
        _, _, u = s.apply(K.LAYER_DOUBLE, phi)
        X, Y = np.meshgrid(s.grid.x, s.grid.y)
        inside = s.cl.side == 1
        errs.append(np.abs(u - np.exp(X) * np.sin(Y))[inside].max())
        hs.append(s.grid.h)
    slope = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert slope > 1.8, (errs, slope)


# ---------------------------------------------------------------- GMRES
def test_gmres_matches_dense_solve():
    p = W.random_problem(4, N=32, n=40)
    s = K.Kfbi(p.N, p.box, 0.0, K.BOX_DIRICHLET0).set_interface(p.xy)
    A = np.stack([s.bie_matvec(K.BIE_INTERIOR_DL, e) for e in np.eye(p.n)], 1)
    ref = np.linalg.solve(A, p.rhs)
    x, info = gmres(lambda v: A @ v, p.rhs, tol=1e-13, restart=7, max_iter=500)
    assert info["converged"] and info["restarts"] > 0
    assert np.abs(x - ref).max() < 1e-10 * np.abs(ref).max()
    x2, info2 = gmres(lambda v: s.bie_matvec(K.BIE_INTERIOR_DL, v), p.rhs, tol=1e-13)
    assert np.abs(x2 - ref).max() < 1e-10 * np.abs(ref).max()


def test_outside_box_and_underresolved():
    s = K.Kfbi(32, (-1, 1, -1, 1), 0.0, K.BOX_DIRICHLET0)
    with pytest.raises(K.OutsideBox):
        s.set_interface(plain_ellipse_nodes(0.95, 0.5, 64))
    # a star with a very thin arm crosses one arm three times at this resolution
    shape = W.polar(0.5, [(11, 0.45, 0.0)])
    nodes = W.equal_arclength(shape, 256)
    with pytest.raises((K.Underresolved, K.OutsideBox)):
        K.Kfbi(16, (-1, 1, -1, 1), 0.0, K.BOX_DIRICHLET0).set_interface(nodes["xy"])


# ---------------------------------------------------------------- classification edge cases (R3, R4)
def circle_through_node(N, i, j, R, angle_deg, n=256):
    """Nodes of a circle of radius R that passes through grid node (i, j) at the given polar angle."""
    grid = K.Grid(N, (-1.0, 1.0, -1.0, 1.0))
    th = math.radians(angle_deg)
    cx, cy = grid.x[i] - R * math.cos(th), grid.y[j] - R * math.sin(th)
    a = 2 * math.pi * (np.arange(n) + 0.37 / 8) / n + th   # no bracket sample on the grid node
    return np.stack([cx + R * np.cos(a), cy + R * np.sin(a)], -1)


@pytest.mark.parametrize("angle", [-30.0, 150.0, 60.0, -120.0])
def test_node_on_the_curve_is_in_the_closed_interior(angle):
    """A grid node on the curve (to rounding) lies in Omega+ and its row and column
    crossings sit on the arms that leave it toward the outside, whatever the quadrant."""
    N, i, j = 64, 30, 33
    s = K.Kfbi(N, (-1, 1, -1, 1), 0.0, K.BOX_DIRICHLET0).set_interface(circle_through_node(N, i, j, 0.4, angle))
    assert s.cl.side[j, i] == 1
    on = np.abs(s.cr.xi - np.where(s.cr.kind == 0, s.grid.x[i], s.grid.y[j])) == 0.0
    assert on.sum() == 2                            # one row and one column crossing snapped onto it
    v, _, u = s.apply(K.LAYER_DOUBLE, np.ones(s.iface.n))
    assert np.abs(u - s.cl.side).max() < 1e-12      # D1 is still the indicator (Gauss)


def test_arm_crossed_twice_gets_no_correction():
    """A circle whose top rises just above a grid line between two nodes crosses that arm twice;
    both ends are outside, the arm carries no correction and D1 is still the indicator (R4)."""
    N = 64
    h = 2.0 / N
    j = 40
    yl = -1.0 + (j + 0.5) * h
    xc = -1.0 + 20.0 * h                    # the midpoint of the arm (19, j)-(20, j)
    R = 0.5
    a = 2 * math.pi * np.arange(256) / 256
    xy = np.stack([xc + R * np.cos(a), yl - R + 2e-5 + R * np.sin(a)], -1)
    s = K.Kfbi(N, (-1, 1, -1, 1), 0.0, K.BOX_DIRICHLET0).set_interface(xy)
    i = int(np.searchsorted(s.grid.x, xc))
    assert s.cl.hcount[j, i] == 2 and s.cl.hid[j, i] == -1
    assert s.cl.side[j, i - 1] == 0 and s.cl.side[j, i] == 0
    _, _, u = s.apply(K.LAYER_DOUBLE, np.ones(s.iface.n))
    assert np.abs(u - s.cl.side).max() < 1e-12
