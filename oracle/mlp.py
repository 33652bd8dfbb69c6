"""Oracle for the learned warm start of GMRES: features, MLP forward/backward, Adam (FP64).

TEST INFRASTRUCTURE ONLY: imported by tests/ and bench.py's CPU legs, never by the product
path.

The paper solves every boundary integral equation by GMRES from a given initial density
(Sec. 4); it has no learned component. The warm start here follows the reading recorded
with the build: a small multilayer perceptron maps per-node interface features to the
density, the prediction only seeds GMRES, and GMRES still iterates to the same tolerance,
so the solution does not depend on it.

Features of node j (FEATURES = 47), with l = L / (2 pi) the mean radius of the curve:
  0..31  Re, Im of khat_k e^{i k alpha_j} l, k = 0..15, khat_k = (1/n) sum_m kappa_m e^{-i k alpha_m}
         (the curvature's Fourier modes rotated to the node)
  32     kappa_j l
  33, 34 outward unit normal (n_x, n_y)
  35     s_j / L, arclength from node 0 by the trapezoidal rule
  36     g_j / rms(g)   (the node's right-hand side; rms over the nodes)
  37, 38 (x_j - mean x) / l, (y_j - mean y) / l
  39..46 Re, Im of ghat_k e^{i k alpha_j} / rms(g), k = 0..3, ghat_k = (1/n) sum_m g_m e^{-i k alpha_m}
         (the data's low modes rotated to the node: the density depends on the data
         globally, e.g. on its mean, not only on g_j)
Target: phi_j / rms(g). The equation is linear, so a prediction y_j gives phi_j = rms(g) y_j.

Network: 47 -> H -> H -> 1 with ReLU, weights rounded to bfloat16 (round to nearest even)
where they are used, biases, activations and accumulation in full precision here (float32
on the device). Loss: mean squared error. Gradients are taken with the rounded weights and
applied to the unrounded (master) weights. Adam: Kingma & Ba (2015), bias-corrected.
"""
from __future__ import annotations

import math

import numpy as np

FEATURES = 47
MODES = 16
DATA_MODES = 4


# ----------------------------------------------------------------------------- features
def curvature(g):
    """kappa = (x_a y_aa - y_a x_aa) / s_a^3 from the derivatives of a parametrisation."""
    return (g["xa"] * g["yaa"] - g["ya"] * g["xaa"]) / g["sa"] ** 3


def features(iface, rhs):
    """Per-node features (n x FEATURES) of an oracle Interface and its right-hand side."""
    n = iface.n
    g = iface.node
    kap = curvature(g)
    L = float(np.sum(g["sa"])) * 2.0 * math.pi / n
    ell = L / (2.0 * math.pi)
    alpha = iface.alpha
    F = np.zeros((n, FEATURES))
    for k in range(MODES):
        khat = np.sum(kap * np.exp(-1j * k * alpha)) / n
        rot = khat * np.exp(1j * k * alpha) * ell
        F[:, 2 * k] = rot.real
        F[:, 2 * k + 1] = rot.imag
    F[:, 32] = kap * ell
    F[:, 33] = g["nx"]
    F[:, 34] = g["ny"]
    s = np.zeros(n)
    s[1:] = np.cumsum(0.5 * (g["sa"][:-1] + g["sa"][1:])) * 2.0 * math.pi / n
    F[:, 35] = s / L
    rhs = np.asarray(rhs, dtype=np.float64)
    rms = math.sqrt(float(np.mean(rhs * rhs)))
    F[:, 36] = rhs / rms if rms > 0 else 0.0
    F[:, 37] = (g["x"] - np.mean(g["x"])) / ell
    F[:, 38] = (g["y"] - np.mean(g["y"])) / ell
    for k in range(DATA_MODES):
        ghat = np.sum(rhs * np.exp(-1j * k * alpha)) / n
        rot = ghat * np.exp(1j * k * alpha) / rms if rms > 0 else 0.0 * alpha
        F[:, 39 + 2 * k] = np.real(rot)
        F[:, 40 + 2 * k] = np.imag(rot)
    return F, rms


# ----------------------------------------------------------------------------- bfloat16
def bf16(a):
    """Round to bfloat16 (nearest, ties to even) through float32; returned as float64."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    bits = a32.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64).reshape(a32.shape)


# ----------------------------------------------------------------------------- network
def _weights(P, quantize):
    q = bf16 if quantize else (lambda w: np.asarray(w, dtype=np.float64))
    return q(P["W1"]), q(P["W2"]), q(P["w3"])


def forward(P, X, quantize=True):
    """y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 per row of X; returns (y, cache)."""
    W1, W2, w3 = _weights(P, quantize)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + P["b3"]
    return y, dict(X=X, z1=z1, h1=h1, z2=z2, h2=h2, W2=W2, w3=w3)


def loss_and_grads(P, X, t, quantize=True):
    """Mean squared error and its gradient with respect to every parameter (chain rule
    through the two ReLU layers, written out by hand)."""
    y, c = forward(P, X, quantize)
    R = y.shape[0]
    r = y - np.asarray(t, dtype=np.float64)
    loss = float(np.mean(r * r))
    dy = 2.0 * r / R
    G = {}
    G["w3"] = c["h2"].T @ dy
    G["b3"] = float(np.sum(dy))
    dz2 = np.outer(dy, c["w3"]) * (c["z2"] > 0.0)
    G["W2"] = dz2.T @ c["h1"]
    G["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ c["W2"]) * (c["z1"] > 0.0)
    G["W1"] = dz1.T @ c["X"]
    G["b1"] = dz1.sum(axis=0)
    return loss, G


PARAM_NAMES = ("W1", "b1", "W2", "b2", "w3", "b3")


def adam_step(P, G, M, V, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of every parameter in place; `step` counts from 1."""
    for k in PARAM_NAMES:
        g = np.asarray(G[k], dtype=np.float64)
        M[k] = beta1 * np.asarray(M[k]) + (1.0 - beta1) * g
        V[k] = beta2 * np.asarray(V[k]) + (1.0 - beta2) * g * g
        mh = M[k] / (1.0 - beta1 ** step)
        vh = V[k] / (1.0 - beta2 ** step)
        P[k] = np.asarray(P[k], dtype=np.float64) - lr * mh / (np.sqrt(vh) + eps)
    return P


def zeros_like(P):
    return {k: np.zeros_like(np.asarray(P[k], dtype=np.float64)) for k in PARAM_NAMES}
