"""Pins of the warm-start oracle (oracle/mlp.py) against values fixed by arithmetic and
calculus: bfloat16 rounding of chosen values, a network small enough to evaluate by hand,
central finite differences of the loss, Adam's first step in closed form, and the features
of curves whose curvature is known in closed form."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import kfbi as OK
from oracle import mlp as OM


def test_bf16_rounding_ties_to_even():
    # spacing of bfloat16 at 1 is 2^-7; 1 + 2^-8 is a tie (to the even 1.0), 1 + 3 2^-8 a tie
    # between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -12, -2.5, 0.0])
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7, -2.5, 0.0])
    assert np.array_equal(OM.bf16(vals), want)
    # relative error of bfloat16 rounding is at most 2^-8
    x = np.random.default_rng(0).normal(size=1000) * 10.0
    assert np.max(np.abs(OM.bf16(x) - x) / np.abs(x)) <= 2.0 ** -8


def test_forward_by_hand():
    # y = relu(x0) + relu(-x1) + 0.5 with W1 = [[1, 0], [0, -1]], W2 = I, w3 = (1, 1)
    P = dict(W1=np.array([[1.0, 0.0], [0.0, -1.0]]), b1=np.zeros(2), W2=np.eye(2), b2=np.zeros(2),
             w3=np.ones(2), b3=0.5)
    X = np.array([[2.0, 3.0], [-1.0, -4.0], [0.5, -0.25]])
    y, _ = OM.forward(P, X)
    assert np.allclose(y, [2.0 + 0.0 + 0.5, 0.0 + 4.0 + 0.5, 0.5 + 0.25 + 0.5], atol=0, rtol=0)


def _small(seed, F=5, H=7):
    rng = np.random.default_rng(seed)
    return dict(W1=rng.normal(size=(H, F)), b1=rng.normal(size=H) * 0.1, W2=rng.normal(size=(H, H)) / 2,
                b2=rng.normal(size=H) * 0.1, w3=rng.normal(size=H), b3=0.3)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(1)
    P = _small(2)
    X = rng.normal(size=(11, 5))
    t = rng.normal(size=11)
    loss, G = OM.loss_and_grads(P, X, t, quantize=False)
    eps = 1e-6
    for name in OM.PARAM_NAMES:
        arr = np.atleast_1d(np.asarray(P[name], dtype=np.float64))
        for idx in list(np.ndindex(arr.shape))[:6]:
            Pp = {k: np.array(v, dtype=np.float64, copy=True) for k, v in P.items()}
            Pm = {k: np.array(v, dtype=np.float64, copy=True) for k, v in P.items()}
            if arr.ndim == 1 and np.ndim(P[name]) == 0:
                Pp[name] = P[name] + eps
                Pm[name] = P[name] - eps
                g = G[name]
            else:
                Pp[name][idx] += eps
                Pm[name][idx] -= eps
                g = np.asarray(G[name])[idx]
            fd = (OM.loss_and_grads(Pp, X, t, False)[0] - OM.loss_and_grads(Pm, X, t, False)[0]) / (2 * eps)
            assert abs(fd - g) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, g)


def test_quantised_gradient_is_the_formula_at_rounded_weights():
    rng = np.random.default_rng(3)
    P = _small(4)
    X = rng.normal(size=(9, 5))
    t = rng.normal(size=9)
    lq, Gq = OM.loss_and_grads(P, X, t, quantize=True)
    Pr = dict(P, W1=OM.bf16(P["W1"]), W2=OM.bf16(P["W2"]), w3=OM.bf16(P["w3"]))
    lr_, Gr = OM.loss_and_grads(Pr, X, t, quantize=False)
    assert lq == lr_
    for k in OM.PARAM_NAMES:
        assert np.array_equal(np.asarray(Gq[k]), np.asarray(Gr[k]))


def test_adam_first_step_closed_form():
    # after one step m_hat = g and v_hat = g^2, so theta_1 = theta_0 - lr g / (|g| + eps)
    P = _small(5)
    rng = np.random.default_rng(6)
    G = {k: rng.normal(size=np.shape(P[k])) if np.ndim(P[k]) else float(rng.normal()) for k in OM.PARAM_NAMES}
    P0 = {k: np.array(v, dtype=np.float64, copy=True) for k, v in P.items()}
    M, V = OM.zeros_like(P), OM.zeros_like(P)
    OM.adam_step(P, G, M, V, 1, lr=1e-2, eps=1e-8)
    for k in OM.PARAM_NAMES:
        g = np.asarray(G[k], dtype=np.float64)
        assert np.allclose(P[k], P0[k] - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


def test_adam_fits_a_linear_target():
    # a network with a linear target converges to a small loss (the update direction is right)
    rng = np.random.default_rng(7)
    P = _small(8, F=3, H=16)
    X = rng.normal(size=(64, 3))
    t = X @ np.array([0.5, -1.0, 2.0]) + 0.25
    M, V = OM.zeros_like(P), OM.zeros_like(P)
    l0 = OM.loss_and_grads(P, X, t, False)[0]
    for s in range(1, 1501):
        _, G = OM.loss_and_grads(P, X, t, False)
        OM.adam_step(P, G, M, V, s, lr=1e-2)
    assert OM.loss_and_grads(P, X, t, False)[0] < 1e-3 * l0


def test_features_of_a_circle():
    R, n = 0.7, 64
    a = 2 * math.pi * np.arange(n) / n
    xy = np.stack([0.1 + R * np.cos(a), -0.2 + R * np.sin(a)], 1)
    rhs = np.cos(a)
    F, rms = OM.features(OK.Interface(xy), rhs)
    assert abs(rms - math.sqrt(0.5)) < 1e-14
    assert np.allclose(F[:, 0], 1.0, atol=1e-12)              # khat_0 l = kappa l = 1
    assert np.allclose(F[:, 1:32], 0.0, atol=1e-12)            # no other curvature modes
    assert np.allclose(F[:, 32], 1.0, atol=1e-12)
    assert np.allclose(F[:, 33], np.cos(a), atol=1e-13)
    assert np.allclose(F[:, 34], np.sin(a), atol=1e-13)
    assert np.allclose(F[:, 35], np.arange(n) / n, atol=1e-13)  # uniform speed
    assert np.allclose(F[:, 36], rhs / math.sqrt(0.5), atol=1e-13)
    assert np.allclose(F[:, 37], np.cos(a), atol=1e-12)
    assert np.allclose(F[:, 38], np.sin(a), atol=1e-12)
    # data cos(alpha): only the k = 1 mode, ghat_1 = 1/2, rotated: (1/2) e^{i alpha} / rms
    assert np.allclose(F[:, 39:41], 0.0, atol=1e-13)
    assert np.allclose(F[:, 41], 0.5 * np.cos(a) / math.sqrt(0.5), atol=1e-13)
    assert np.allclose(F[:, 42], 0.5 * np.sin(a) / math.sqrt(0.5), atol=1e-13)
    assert np.allclose(F[:, 43:47], 0.0, atol=1e-13)


def test_curvature_of_an_ellipse():
    # x = a cos t, y = b sin t at t_j = alpha_j: kappa = a b / (a^2 sin^2 t + b^2 cos^2 t)^{3/2}
    A, B, n = 0.6, 0.4, 48
    t = 2 * math.pi * np.arange(n) / n
    xy = np.stack([A * np.cos(t), B * np.sin(t)], 1)
    iface = OK.Interface(xy)
    kap = OM.curvature(iface.node)
    want = A * B / (A * A * np.sin(t) ** 2 + B * B * np.cos(t) ** 2) ** 1.5
    assert np.allclose(kap, want, rtol=1e-12, atol=0)
    F, _ = OM.features(iface, np.ones(n))
    L = np.sum(iface.node["sa"]) * 2 * math.pi / n
    # the rotated modes sum to the curvature (all modes of this curvature above 15 are tiny)
    k_from_modes = np.zeros(n)
    for k in range(OM.MODES):
        w = 1.0 if k == 0 else 2.0
        k_from_modes += w * F[:, 2 * k]
    assert np.max(np.abs(k_from_modes * 2 * math.pi / L - kap)) < 1e-3 * np.max(kap)


def test_warmstart_problem_data_is_harmonic():
    # the boundary data generator is a harmonic function (five-point Laplacian ~ h^2)
    u = W.random_harmonic(11)
    h = 1e-3
    x, y = np.array([0.1, -0.3, 0.4]), np.array([0.2, 0.05, -0.35])
    lap = (u(x + h, y) + u(x - h, y) + u(x, y + h) + u(x, y - h) - 4 * u(x, y)) / (h * h)
    assert np.max(np.abs(lap)) < 1e-4 * max(1.0, np.max(np.abs(u(x, y))))


@pytest.mark.parametrize("seed", [1, 2])
def test_mlp_init_shapes_and_scale(seed):
    P = W.mlp_init(seed, features=OM.FEATURES)
    assert P["W1"].shape == (256, OM.FEATURES) and P["W2"].shape == (256, 256) and P["w3"].shape == (256,)
    assert abs(np.std(P["W2"]) - math.sqrt(2.0 / 256)) < 0.01
