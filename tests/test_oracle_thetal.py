"""Pins for the theta-L oracle (Sec. 5) against invariants and closed forms.

- reconstruction of generator nodes from (eta, L, Xbar);
- equal arclength s_a = L / 2 pi is kept by the tangential velocity (Sec. 5.1);
- Hele-Shaw with injection J: dA/dt = 2 pi J (the modified double layer carries no flux);
- Hele-Shaw with J = 0: area constant, length non-increasing (Sec. 6.1.2);
- Hele-Shaw linear stability of r = R + eps cos k a: eps'/eps = J(k-1)/R^2 - sigma k(k^2-1)/R^3
  (classical result derived from the model of Sec. 2.1, not printed in the paper);
- Stefan: the 4-fold symmetric seed stays 4-fold symmetric (Sec. 6.2.1).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import kfbi as K
from oracle import thetal as T


def mode_amp(X, k, kmax=9):
    r = np.hypot(X[:, 0], X[:, 1])
    ph = np.arctan2(X[:, 1], X[:, 0])
    B = np.stack([np.ones_like(ph)] + [f(m * ph) for m in range(1, kmax + 1) for f in (np.cos, np.sin)], -1)
    c = np.linalg.lstsq(B, r, rcond=None)[0]
    return math.hypot(c[2 * k - 1], c[2 * k])


def test_reconstruction_recovers_nodes():
    for shape, n in ((W.hele_shaw_shape(), 256), (W.ellipse(0.6, 0.4), 128), (W.stefan_shape(), 512)):
        nd = W.equal_arclength(shape, n)
        st = T.state_from_nodes(nd["xy"], nd["theta"], nd["L"])
        X = T.reconstruct(st.eta, st.L, st.Xbar)
        assert np.abs(X - nd["xy"]).max() < 1e-12 * nd["L"]


def test_cumulative_integral_and_derivative():
    n = 64
    a = 2 * math.pi * np.arange(n) / n
    f = 0.3 + np.cos(2 * a) - 0.5 * np.sin(7 * a)
    F = 0.3 * a + 0.5 * np.sin(2 * a) + 0.5 / 7 * (np.cos(7 * a) - 1.0)
    assert np.abs(T.cumulative_integral(f) - F).max() < 1e-13
    assert np.abs(T.spec_deriv(f) - (-2 * np.sin(2 * a) - 3.5 * np.cos(7 * a))).max() < 1e-12


@pytest.fixture(scope="module")
def hs_run():
    nd = W.equal_arclength(W.polar(1.0, [(3, 0.05, 0.0), (5, 0.03, 0.4)]), 128)
    st = T.state_from_nodes(nd["xy"], nd["theta"], nd["L"])
    s = K.Kfbi(192, (-3, 3, -3, 3), 0.0, K.BOX_FREESPACE_DL)
    A0 = T.area(nd["xy"])
    for _ in range(10):
        T.hs_step(s, st, 2e-3, 1e-2, 1.0, tol=1e-11)
    return st, A0


def test_hele_shaw_area_growth(hs_run):
    st, A0 = hs_run
    X = T.reconstruct(st.eta, st.L, st.Xbar)
    growth = T.area(X) - A0
    assert abs(growth - 2 * math.pi * st.t) < 2e-3 * 2 * math.pi * st.t


def test_equal_arclength_kept(hs_run):
    st, _ = hs_run
    X = T.reconstruct(st.eta, st.L, st.Xbar)
    sa = np.hypot(T.spec_deriv(X[:, 0]), T.spec_deriv(X[:, 1]))
    # s_a is constant up to the spectral truncation of this 128-node curve
    assert np.abs(sa - st.L / (2 * math.pi)).max() < 1e-7 * st.L
    assert abs(T.length(X) - st.L) < 1e-12 * st.L


def test_hele_shaw_relaxation_conserves_area_and_shortens():
    nd = W.equal_arclength(W.polar(0.8, [(6, 0.2 / 0.8 * 0.25, 0.0)]), 128)
    st = T.state_from_nodes(nd["xy"], nd["theta"], nd["L"])
    s = K.Kfbi(128, (-1.5, 1.5, -1.5, 1.5), 0.0, K.BOX_FREESPACE_DL)
    A0, L0 = T.area(nd["xy"]), nd["L"]
    Ls = [L0]
    for _ in range(6):
        T.hs_step(s, st, 1e-3, 1e-2, 0.0, tol=1e-11)
        Ls.append(st.L)
    X = T.reconstruct(st.eta, st.L, st.Xbar)
    assert abs(T.area(X) - A0) < 2e-5 * A0
    assert all(b < a for a, b in zip(Ls, Ls[1:]))


@pytest.mark.parametrize("k", [3, 5])
def test_hele_shaw_linear_growth_rate(k):
    R0, sigma, J, eps0 = 1.0, 1e-2, 1.0, 1e-3
    nd = W.equal_arclength(W.polar(R0, [(k, eps0, 0.0)]), 128)
    st = T.state_from_nodes(nd["xy"], nd["theta"], nd["L"])
    s = K.Kfbi(192, (-3, 3, -3, 3), 0.0, K.BOX_FREESPACE_DL)
    a0 = mode_amp(nd["xy"], k)
    for _ in range(12):
        T.hs_step(s, st, 4e-3, sigma, J, tol=1e-11)
    X = T.reconstruct(st.eta, st.L, st.Xbar)
    tt = np.linspace(0.0, st.t, 4001)
    R = np.sqrt(R0 ** 2 + 2 * J * tt)
    pred = np.trapezoid(J * (k - 1) / R ** 2 - sigma * k * (k * k - 1) / R ** 3, tt)
    meas = math.log(mode_amp(X, k) / a0)
    assert abs(meas - pred) < 0.01 * abs(pred)


def test_stefan_four_fold_symmetry():
    p = W.config_stefan(N=128, n=128, box=0.5, dt=1e-3)
    st = T.state_from_nodes(p.xy, p.theta, p.L)
    e = p.extra
    s = K.Kfbi(p.N, p.box, p.kappa, K.BOX_NEUMANN0)
    A0 = T.area(p.xy)
    for _ in range(3):
        T.stefan_step(s, st, e["dt"], e["St"], e["eps_c"], e["eps_aniso"], e["fold"], e["eps_v"], tol=1e-12)
    X = T.reconstruct(st.eta, st.L, st.Xbar)
    n = X.shape[0]
    rot = np.stack([-X[:, 1], X[:, 0]], -1)           # rotate by +90 degrees
    assert np.abs(np.roll(X, -n // 4, axis=0) - rot).max() < 1e-9
    assert T.area(X) > A0                               # undercooled melt: the seed grows
