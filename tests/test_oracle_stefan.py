"""Pins for the Stefan half of the oracle (Sec. 3.2, Sec. 5.2.2, Sec. 5.3).

Each test checks the oracle against something other than itself:
- the stiff symbols of the small-scale decomposition are the high-mode limit of the linear
  growth rates of a perturbed circle (classical Hele-Shaw stability, and the Stefan rate
  from the closed-form single layer on a circle, scipy.special);
- the propagators e_k integrate the stiff linear equation (an ODE solver, scipy.integrate);
- with the nonlinear term zero the update multiplies each mode by its propagator;
- the single-layer equation eps_V psi - S psi = cos k a on a circle has the closed-form
  solution cos k a / (eps_V + R I_k(cR) K_k(cR)) (the sign of the Stefan operator);
- the grid field of S psi off the circle is -R I_k(c r<) K_k(c r>) cos k theta (the field
  that enters T = T1 - S psi);
- a whole Stefan step on a circle agrees with the radially symmetric reference
  (tests/radial_stefan.py: Bessel functions and a radial Green's function), from the seed
  and from a smooth two-level history (the BDF2 right-hand side, the split T = T1 - S psi,
  the Gibbs-Thomson right-hand side and the length update);
- the time-discrete scheme is second order from a consistent history (radial reference).
"""
import math

import mpmath
import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

import workloads as W
from oracle import kfbi as K
from oracle import thetal as T
from oracle.gmres import gmres
from radial_stefan import RadialStefan


def circle_nodes(R, n):
    a = 2 * math.pi * np.arange(n) / n
    return np.stack([R * np.cos(a), R * np.sin(a)], -1), a


# ---------------------------------------------------------------- stiff symbols (Sec. 5.2)
def test_hele_shaw_symbol_is_high_mode_limit_of_linear_rate():
    """On a circle of radius R (L = 2 pi R), a mode-k perturbation grows at
    J(k-1)/R^2 - sigma k(k^2-1)/R^3; the stiff symbol is the leading term for large k."""
    R, sigma, J, n = 0.8, 1e-3, 1.0, 4096
    L = 2 * math.pi * R
    sym = T.hs_symbol(n, sigma)(L)
    for k in (64, 256, 1024):
        rate = J * (k - 1) / R ** 2 - sigma * k * (k * k - 1) / R ** 3
        assert abs(sym[k] / rate - 1.0) < 4.0 * R / (sigma * k * k), k
        assert sym[k] == sym[n - k]            # symmetric in the sign of k


def test_stefan_symbol_is_high_mode_limit_of_linear_rate():
    """Case I (eps_V > 0): the single-layer equation on a circle gives a mode-k normal velocity
    U_k = -eps_C kappa_k / (eps_V + R I_k(cR) K_k(cR)) with kappa_k = (k^2 - 1)/R^2 per unit
    amplitude; as k grows, R I_k K_k -> 0 and the rate tends to -(eps_C / eps_V) k^2 / R^2,
    the symbol -lambda_1 (2 pi / L)^2 k^2 with lambda_1 = eps_C / eps_V."""
    R, eps_c, eps_v, c, n = 0.3, 3e-3, 1.5e-3, math.sqrt(3000.0), 8192
    L = 2 * math.pi * R
    # lambda_1 as the oracle's step forms it from eps_C and eps_V (one step on a circle)
    nd = W.equal_arclength(W.polar(R, []), 64)
    st = T.state_from_nodes(nd["xy"], nd["theta"], nd["L"])
    T.stefan_step(K.Kfbi(64, (-1, 1, -1, 1), c * c, K.BOX_NEUMANN0), st, 1.5 / (c * c), -0.5, eps_c, 0.0, 4,
                  eps_v, tol=1e-10)
    lam1 = st.last["lam1"]
    sym = T.stefan_symbol(n, lam1)(L)
    prev = None
    for k in (16, 128, 1024, 4000):
        ik_kk = float(mpmath.besseli(k, c * R) * mpmath.besselk(k, c * R))  # scipy overflows at large k
        rate = -eps_c * (k * k - 1) / R ** 2 / (eps_v + R * ik_kk)
        err = abs(sym[k] / rate - 1.0)
        if prev is not None:
            assert err < prev
        prev = err
    assert prev < 2.5e-2       # the single layer fades like R / (2k) against eps_V


# ---------------------------------------------------------------- propagators (Sec. 5.3)
@pytest.mark.parametrize("which", ["hs", "stefan"])
def test_propagators_integrate_the_stiff_equation(which):
    """e_k(t_n, t_{n+1}) and e_k(t_{n-1}, t_{n+1}) are the solution operators of
    d eta_k / dt = s_k(L(t)) eta_k over one and two steps: exactly when L is fixed, to third
    order in dt (trapezoidal rule in time) when L changes linearly."""
    n = 64
    fn = T.hs_symbol(n, 5e-3) if which == "hs" else T.stefan_symbol(n, 1.3)
    k = 9
    for dt, dL in ((2e-3, 0.0), (2e-3, 0.02), (1e-3, 0.01)):
        L0 = 1.7
        Lp, Ln, Lnew = L0 - dL, L0, L0 + dL

        def ode(t, y):
            return [fn(Lp + (t / dt) * dL)[k] * y[0]]

        one = si.solve_ivp(ode, (dt, 2 * dt), [1.0], rtol=1e-13, atol=1e-15, method="DOP853").y[0, -1]
        two = si.solve_ivp(ode, (0.0, 2 * dt), [1.0], rtol=1e-13, atol=1e-15, method="DOP853").y[0, -1]
        e1, e2 = T.st_propagators(fn, dt, Lp, Ln, Lnew)
        tol = 1e-12 if dL == 0.0 else 5.0 * (dt * abs(fn(L0)[k])) ** 3 * (dL / L0) + 1e-12
        assert abs(e1[k] / one - 1.0) < tol
        assert abs(e2[k] / two - 1.0) < tol


@pytest.mark.parametrize("which", ["hs", "stefan"])
def test_update_without_nonlinear_term_is_the_propagator(which):
    """With N^n = N^{n-1} = 0 and L fixed, every Fourier mode of eta after one step is
    exp(dt s_k) times its value: the exact solution of the stiff linear equation."""
    n = 64
    fn = T.hs_symbol(n, 5e-3) if which == "hs" else T.stefan_symbol(n, 1.3)
    rng = np.random.default_rng(3)
    eta = np.fft.fft(rng.standard_normal(n))
    dt, L = 3e-3, 1.9
    e1, e2 = T.st_propagators(fn, dt, L, L, L)
    z = np.zeros(n, dtype=complex)
    out = T.ssd_ab2(eta, z, z, e1, e2, dt)
    for k in range(n):
        exact = si.solve_ivp(lambda t, y: [fn(L)[k] * y[0]], (0.0, dt), [1.0], rtol=1e-13, atol=1e-15,
                             method="DOP853").y[0, -1]
        assert abs(out[k] - exact * eta[k]) <= 1e-12 * abs(eta[k]) + 1e-300


# ---------------------------------------------------------------- single layer on a circle (Sec. 3.2)
@pytest.mark.parametrize("k", [0, 3])
def test_stefan_operator_on_circle_closed_form(k):
    """eps_V psi - S psi = cos k a on a circle of radius R in a box far away (c dist >> 1):
    S e^{ik a} = -R I_k(cR) K_k(cR) e^{ik a} (G_c = -K0(c r)/2 pi), so
    psi = cos k a / (eps_V + R I_k(cR) K_k(cR)); O(h^2) in the grid."""
    R, kap, eps_v, n = 0.5, 900.0, 2e-3, 128
    c = math.sqrt(kap)
    xy, a = circle_nodes(R, n)
    exact = np.cos(k * a) / (eps_v + R * sp.ive(k, c * R) * sp.kve(k, c * R))
    ev = np.full(n, eps_v)
    errs = []
    for N in (128, 256):
        s = K.Kfbi(N, (-2, 2, -2, 2), kap, K.BOX_NEUMANN0).set_interface(xy)
        psi, info = gmres(lambda x: s.bie_matvec(K.BIE_STEFAN_SL, x, eps_v=ev), np.cos(k * a), tol=1e-12)
        assert info["converged"]
        errs.append(np.abs(psi - exact).max() / np.abs(exact).max())
    assert errs[0] < 0.1 and errs[1] < 0.3 * errs[0], errs


@pytest.mark.parametrize("k", [0, 2])
def test_single_layer_grid_field_off_the_circle(k):
    """The grid output of the single-layer apply is S psi = -R I_k(c r<) K_k(c r>) cos k theta
    (r< = min(r, R), r> = max(r, R)) at grid nodes away from the circle; O(h^2)."""
    R, kap, n = 0.5, 400.0, 128
    c = math.sqrt(kap)
    xy, a = circle_nodes(R, n)
    errs = []
    for N in (128, 256):
        s = K.Kfbi(N, (-2, 2, -2, 2), kap, K.BOX_NEUMANN0).set_interface(xy)
        _, _, u = s.apply(K.LAYER_SINGLE, np.cos(k * a))
        X, Y = np.meshgrid(s.grid.x, s.grid.y)
        r = np.hypot(X, Y)
        th = np.arctan2(Y, X)
        rl, rg = np.minimum(r, R), np.maximum(r, R)
        exact = -R * sp.ive(k, c * rl) * sp.kve(k, c * rg) * np.exp(c * (rl - rg)) * np.cos(k * th)
        mask = (np.abs(r - R) > 2 * s.grid.h) & (r < 1.2)
        errs.append(np.abs(u - exact)[mask].max() / np.abs(exact[mask]).max())
    assert errs[0] < 3e-2 and errs[1] < 0.3 * errs[0], errs


# ---------------------------------------------------------------- the whole Stefan step
R0, ST, EPS_C, EPS_V = 0.3, -0.5, 2e-3, 2e-3


def test_stefan_steps_from_seed_match_radial_reference():
    """Three steps from the seed (T = 0 inside, St outside) on a circle: radius, velocity and
    temperature agree with the radial reference to the error of the seed's staircase."""
    tau, N, n = 1e-3, 128, 128
    xy, _ = circle_nodes(R0, n)
    nd = W.equal_arclength(W.polar(R0, []), n)
    st = T.state_from_nodes(nd["xy"], nd["theta"], nd["L"])
    s = K.Kfbi(N, (-1, 1, -1, 1), 1.5 / tau, K.BOX_NEUMANN0)
    rad = RadialStefan(R0, ST, EPS_C, EPS_V)
    X, Y = np.meshgrid(s.grid.x, s.grid.y)
    r = np.hypot(X, Y)
    for _ in range(3):
        R_old = st.L / (2 * math.pi)
        T.stefan_step(s, st, tau, ST, EPS_C, 0.0, 4, EPS_V, tol=1e-12)
        rad.step(tau)
        assert abs(st.L / (2 * math.pi) - rad.R) < 1e-3 * rad.R
        assert abs(st.density.mean() - rad.U_prev) < 2e-2 * abs(rad.U_prev)
        mask = (np.abs(r - R_old) > 3 * s.grid.h) & (r < 0.9)
        assert np.abs(st.T - rad.at(r))[mask].max() < 1e-2 * abs(ST)


def _warm_state(rad, N, n, tau, k0):
    """An oracle state on the circle of the radial reference after k0 steps: temperature levels,
    length history and the previous velocity copied from it."""
    nd = W.equal_arclength(W.polar(rad.R, []), n)
    st = T.state_from_nodes(nd["xy"], nd["theta"], nd["L"])
    s = K.Kfbi(N, (-1, 1, -1, 1), 1.5 / tau, K.BOX_NEUMANN0)
    X, Y = np.meshgrid(s.grid.x, s.grid.y)
    r = np.hypot(X, Y)
    st.T = rad.at(r)
    st.T_prev = np.interp(r, rad.r, rad.T_prev)
    st.M_prev = 2 * math.pi * rad.U_prev
    st.N_prev = np.zeros(n, dtype=complex)
    st.L_prev = st.L
    st.steps = k0
    st.density = np.full(n, rad.U_prev)
    return st, s, r


def test_stefan_steps_from_smooth_history_match_radial_reference():
    """From a smooth two-level history (the radial reference after ten steps) the oracle's
    BDF2 steps agree with the reference at second order in h: velocity errors fall by more
    than 4x from N = 64 to 128 (both levels of the history enter the right-hand side, the
    new temperature is T1 - S psi)."""
    tau, n, k0 = 1e-3, 128, 10
    uerr = []
    for N in (64, 128):
        rad = RadialStefan(R0, ST, EPS_C, EPS_V)
        for _ in range(k0):
            rad.step(tau)
        st, s, r = _warm_state(rad, N, n, tau, k0)
        worst = 0.0
        for _ in range(2):
            R_old = st.L / (2 * math.pi)
            T.stefan_step(s, st, tau, ST, EPS_C, 0.0, 4, EPS_V, tol=1e-12)
            rad.step(tau)
            worst = max(worst, abs(st.density.mean() - rad.U_prev) / abs(rad.U_prev))
            assert abs(st.L / (2 * math.pi) - rad.R) < 1e-3 * rad.R
            mask = (np.abs(r - R_old) > 3 * s.grid.h) & (r < 0.9)
            assert np.abs(st.T - rad.at(r))[mask].max() < 2e-3 * abs(ST)
        uerr.append(worst)
    assert uerr[1] < 1e-2 and uerr[1] < 0.25 * uerr[0], uerr


def test_time_discrete_scheme_is_second_order_from_consistent_history():
    """BDF2 in T with the lagged geometry and AB2 in the radius (the scheme the oracle steps,
    here on the radial reference) converges at second order in tau when started from a
    consistent two-level history (taken from a fine run); the seed's discontinuous
    temperature alone limits the order of a run started at t = 0."""
    tf, ts, span = 1.25e-4, 0.01, 0.008
    fine = RadialStefan(R0, ST, EPS_C, EPS_V, M=20000)
    lv = {0: (fine.R, fine.T.copy(), None)}
    nts = int(round(ts / tf))
    for i in range(nts):
        U = fine.step(tf)
        lv[i + 1] = (fine.R, fine.T.copy(), U)
    res = {}
    for tau in (2e-3, 1e-3, 5e-4, tf):
        b = int(round(tau / tf))
        m = RadialStefan(R0, ST, EPS_C, EPS_V, M=20000)
        # the field computed at level k holds the temperature of level k - 1 (lagged geometry)
        m.R = lv[nts][0]
        m.T = lv[nts - b + 1][1].copy()
        m.T_prev = lv[nts - 2 * b + 1][1].copy()
        m.U_prev = lv[nts - b + 1][2]
        for _ in range(int(round(span / tau))):
            m.step(tau)
        res[tau] = m.R
    e = [abs(res[t] - res[tf]) for t in (2e-3, 1e-3, 5e-4)]
    assert e[0] / e[1] > 3.2 and e[1] / e[2] > 2.8, e


# ---------------------------------------------------------------- case II and the explicit scheme
def test_stefan_case2_symbol_is_high_mode_limit_of_linear_rate():
    """Case II (eps_V = 0): the first-kind equation on a circle gives U_k = -eps_C kappa_k /
    (R I_k(cR) K_k(cR)); R I_k K_k -> R / (2k) for k >> cR, so the rate tends to
    -2 eps_C k^3 / R^3, the symbol -lambda_2 (2 pi / L)^3 |k|^3 with lambda_2 = max |2 eps_C|."""
    R, eps_c, c, n = 0.3, 3e-3, math.sqrt(3000.0), 16384
    L = 2 * math.pi * R
    nd = W.equal_arclength(W.polar(R, []), 64)
    st = T.state_from_nodes(nd["xy"], nd["theta"], nd["L"])
    T.stefan_step(K.Kfbi(64, (-1, 1, -1, 1), c * c, K.BOX_NEUMANN0), st, 1.5 / (c * c), -0.5, eps_c, 0.0, 4, 0.0,
                  tol=1e-10)
    assert "lam2" in st.last and "lam1" not in st.last
    sym = T.stefan_symbol_case2(n, st.last["lam2"])(L)
    prev = None
    for k in (64, 512, 2048, 8000):
        ik_kk = float(mpmath.besseli(k, c * R) * mpmath.besselk(k, c * R))
        rate = -eps_c * (k * k - 1) / R ** 2 / (R * ik_kk)
        err = abs(sym[k] / rate - 1.0)
        if prev is not None:
            assert err < prev
        prev = err
    assert prev < 1e-3


def test_stefan_first_kind_on_circle_closed_form():
    """eps_V = 0: -S psi = cos k a on a circle gives psi = cos k a / (R I_k(cR) K_k(cR))."""
    R, kap, n, k = 0.5, 900.0, 128, 3
    c = math.sqrt(kap)
    xy, a = circle_nodes(R, n)
    exact = np.cos(k * a) / (R * sp.ive(k, c * R) * sp.kve(k, c * R))
    errs = []
    for N in (128, 256):
        s = K.Kfbi(N, (-2, 2, -2, 2), kap, K.BOX_NEUMANN0).set_interface(xy)
        psi, info = gmres(lambda x: s.bie_matvec(K.BIE_STEFAN_SL, x, eps_v=np.zeros(n)), np.cos(k * a), tol=1e-12)
        assert info["converged"]
        errs.append(np.abs(psi - exact).max() / np.abs(exact).max())
    # the first-kind solve carries the grid's O(h^2) error of S without the damping of eps_V
    assert errs[0] < 0.2 and errs[1] < 0.3 * errs[0], errs


def test_stefan_case2_steps_match_radial_reference():
    """eps_V = 0 (Gibbs-Thomson without kinetics): two steps from a smooth history on a circle
    agree with the radial reference."""
    tau, N, n, k0 = 1e-3, 128, 128, 10
    rad = RadialStefan(R0, ST, EPS_C, 0.0)
    for _ in range(k0):
        rad.step(tau)
    st, s, r = _warm_state(rad, N, n, tau, k0)
    for _ in range(2):
        R_old = st.L / (2 * math.pi)
        T.stefan_step(s, st, tau, ST, EPS_C, 0.0, 4, 0.0, tol=1e-12)
        rad.step(tau)
        assert abs(st.density.mean() - rad.U_prev) < 1e-2 * abs(rad.U_prev)
        assert abs(st.L / (2 * math.pi) - rad.R) < 1e-3 * rad.R
        mask = (np.abs(r - R_old) > 3 * s.grid.h) & (r < 0.9)
        assert np.abs(st.T - rad.at(r))[mask].max() < 2e-3 * abs(ST)


def _high_modes(st):
    n = st.eta.shape[0]
    eh = np.fft.fft(st.eta) / n
    return float(np.abs(eh[n // 4: n - n // 4 + 1]).max())


def _stability_run(tau, steps, scheme):
    """The stability test of Sec. 6.2.2 at half its resolution: eps_V = 0, eps_C = 0.05,
    r = 1 + 0.02 cos 4a in (-2, 2)^2 with 64 nodes on a 128^2 grid, St = -0.5. Returns the
    high-mode amplitudes of eta per step, stopping early when the curve stops being
    representable on the grid."""
    nd = W.equal_arclength(W.polar(1.0, [(4, 0.02, 0.0)]), 64)
    st = T.state_from_nodes(nd["xy"], nd["theta"], nd["L"])
    s = K.Kfbi(128, (-2, 2, -2, 2), 1.5 / tau, K.BOX_NEUMANN0)
    amps = []
    for _ in range(steps):
        try:
            T.stefan_step(s, st, tau, -0.5, 0.05, 0.0, 4, 0.0, tol=1e-10, scheme="explicit" if scheme else
                          "semi-implicit")
        except (K.Underresolved, K.OutsideBox):
            amps.append(math.inf)
            break
        amps.append(_high_modes(st))
    return amps


def test_explicit_scheme_is_unstable_above_its_limit_and_semi_implicit_is_not():
    """Third-order stiffness of case II (Sec. 6.2.2): the top mode k = n/2 of the first-kind
    Stefan equation on the circle decays at about 2 eps_C k^2 c / R^2 (c = sqrt(3 / (2 tau)) >> k / R:
    R I_k K_k ~ 1 / (2c)), so Adams-Bashforth without the stiff part needs
    tau 2 eps_C k^2 sqrt(1.5 tau) < 1, tau < 6.4e-5 for k = 32: at 2e-4 the high modes grow
    until the curve breaks within a few steps; at 2.5e-5 they decay; the semi-implicit scheme
    at 1e-2 (160x the explicit limit) keeps them small and bounded."""
    bad = _stability_run(2e-4, 8, True)
    assert bad[-1] == math.inf or bad[-1] > 1.0, bad
    good = _stability_run(2.5e-5, 20, True)
    assert all(np.isfinite(good)) and good[-1] < good[0] and max(good) < 0.1, good
    semi = _stability_run(1e-2, 8, False)
    assert all(np.isfinite(semi)) and max(semi) < 1e-3, semi
