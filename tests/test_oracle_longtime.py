"""Pins for the long-time Hele-Shaw machinery of the oracle (Sec. 6.1.4): marker doubling and
the rescaled frame.

- doubling the markers keeps the curve (old nodes reproduced, length, area and equal arclength
  unchanged) and a run refined before its first step equals a run started on the fine markers;
- the refinement triggers exactly when L / n exceeds 1.5 h;
- the rescaled run keeps its area at A0 (J = 1) and, mapped back (x = R xb, t = (A0/pi)(e^{2 tb}-1)/2),
  reproduces a run in the physical frame, and the physical area grows as A0 + 2 pi J t.
"""
import math

import numpy as np

import workloads as W
from oracle import kfbi as K
from oracle import thetal as T


def test_refine_markers_keeps_the_curve():
    """The doubled curve passes through the old nodes up to the old curve's own representation
    error (it is rebuilt from cos and sin of the interpolated tangent angle), which falls
    spectrally with n; interpolated functions (the density) are reproduced to rounding."""
    errs = []
    for n in (64, 128):
        nd = W.equal_arclength(W.hele_shaw_shape(), n)
        st = T.state_from_nodes(nd["xy"], nd["theta"], nd["L"])
        st.density = W.random_density(2, n)
        X0 = T.reconstruct(st.eta, st.L, st.Xbar)
        d0 = st.density.copy()
        T.refine_markers(st)
        assert st.eta.shape[0] == 2 * n
        X1 = T.reconstruct(st.eta, st.L, st.Xbar)
        errs.append(np.abs(X1[::2] - X0).max())
        assert np.abs(st.density[::2] - d0).max() < 1e-13
        assert abs(T.area(X1) - T.area(X0)) < 1e-5 * T.area(X0)
        assert abs(T.length(X1) - st.L) < 1e-12 * st.L
    assert errs[1] < 1e-8 and errs[1] < 1e-2 * errs[0], errs


def test_refinement_triggers_at_one_and_a_half_cells():
    nd = W.equal_arclength(W.polar(1.0, [(3, 0.05, 0.0)]), 32)
    st = T.state_from_nodes(nd["xy"], nd["theta"], nd["L"])
    s = K.Kfbi(128, (-3, 3, -3, 3), 0.0, K.BOX_FREESPACE_DL)
    h = s.grid.h
    assert nd["L"] / 64 > 1.5 * h and nd["L"] / 128 <= 1.5 * h
    T.hs_step(s, st, 1e-3, 1e-2, 1.0, tol=1e-11, refine_ratio=1.5)
    assert st.eta.shape[0] == 128               # doubled twice: 32 -> 64 -> 128
    T.hs_step(s, st, 1e-3, 1e-2, 1.0, tol=1e-11, refine_ratio=1.5)
    assert st.eta.shape[0] == 128


def test_refined_run_equals_a_run_on_the_fine_markers():
    shape = W.polar(1.0, [(3, 0.05, 0.0), (5, 0.02, 0.3)])
    coarse = W.equal_arclength(shape, 64)
    fine = W.equal_arclength(shape, 128)
    a = T.state_from_nodes(coarse["xy"], coarse["theta"], coarse["L"])
    T.refine_markers(a)
    b = T.state_from_nodes(fine["xy"], fine["theta"], fine["L"])
    d0 = np.abs(a.eta - b.eta).max()        # the 64-node curve's representation error
    assert d0 < 1e-5
    s = K.Kfbi(192, (-3, 3, -3, 3), 0.0, K.BOX_FREESPACE_DL)
    for _ in range(3):
        T.hs_step(s, a, 2e-3, 1e-2, 1.0, tol=1e-12)
        T.hs_step(s, b, 2e-3, 1e-2, 1.0, tol=1e-12)
    assert abs(a.L - b.L) < 1e-8 * b.L
    assert np.abs(a.eta - b.eta).max() < 5 * d0 + 1e-12


def test_rescaled_run_keeps_its_area_and_maps_to_the_physical_run():
    sigma, J = 1e-2, 1.0
    nd = W.equal_arclength(W.polar(1.0, [(3, 0.05, 0.0)]), 128)
    s = K.Kfbi(192, (-3, 3, -3, 3), 0.0, K.BOX_FREESPACE_DL)
    sc = T.state_from_nodes(nd["xy"], nd["theta"], nd["L"])
    dtb, steps = 5e-3, 10
    for _ in range(steps):
        T.hs_step(s, sc, dtb, sigma, J, tol=1e-12, rescale=True)
    R, t1 = T.scaled_frame(sc)
    Xs = T.reconstruct(sc.eta, sc.L, sc.Xbar)
    assert abs(T.area(Xs) - sc.A0) < 1e-5 * sc.A0
    assert abs(R * R * T.area(Xs) - (sc.A0 + 2 * math.pi * J * t1)) < 1e-4 * sc.A0
    ph = T.state_from_nodes(nd["xy"], nd["theta"], nd["L"])
    for _ in range(steps):
        T.hs_step(s, ph, t1 / steps, sigma, J, tol=1e-12)
    Xp = T.reconstruct(ph.eta, ph.L, ph.Xbar)
    # same curve up to the two runs' time discretisation (their steps differ in physical time)
    rp = np.hypot(Xp[:, 0], Xp[:, 1])
    rs = R * np.hypot(Xs[:, 0], Xs[:, 1])
    assert abs(ph.L - R * sc.L) < 1e-4 * ph.L
    assert np.abs(np.sort(rp) - np.sort(rs)).max() < 1e-4
