"""Seeded synthetic inputs for the KFBI tests and the benchmark.

This module is the only code shared by the CPU oracle and the CUDA path. It holds
none of the method's arithmetic: it draws interface shapes, places nodes at equal
arclength on them, and evaluates closed-form boundary data. Every generator is
deterministic for a given seed (numpy PCG64).

Workload shapes follow the paper's experiments (Sec. 6): star-shaped perturbations
of circles r(t) = R0 (1 + sum_k a_k cos(k t + phi_k)), ellipses, and the Stefan seed
r(t) = 0.1 (1 + 0.2 cos 4t).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MASTER_SEED = 20230901

# box boundary modes and layer / equation codes, mirrored by include/kfbi.h
BOX_DIRICHLET0, BOX_NEUMANN0, BOX_FREESPACE_DL = 0, 1, 2
LAYER_SINGLE, LAYER_DOUBLE = 0, 1
BIE_INTERIOR_DL, BIE_HS_EXTERIOR_MDL, BIE_STEFAN_SL = 0, 1, 2


# --------------------------------------------------------------------------- shapes
@dataclasses.dataclass
class Shape:
    """A closed CCW curve X(t), t in [0, 2pi), with first and second derivatives."""

    kind: str
    params: dict

    def eval(self, t):
        t = np.asarray(t, dtype=np.float64)
        if self.kind == "ellipse":
            a, b = self.params["a"], self.params["b"]
            cx, cy = self.params.get("cx", 0.0), self.params.get("cy", 0.0)
            X = np.stack([cx + a * np.cos(t), cy + b * np.sin(t)], -1)
            Xt = np.stack([-a * np.sin(t), b * np.cos(t)], -1)
            Xtt = np.stack([-a * np.cos(t), -b * np.sin(t)], -1)
            return X, Xt, Xtt
        if self.kind == "polar":
            r, rt, rtt = self._radius(t)
            c, s = np.cos(t), np.sin(t)
            cx, cy = self.params.get("cx", 0.0), self.params.get("cy", 0.0)
            X = np.stack([cx + r * c, cy + r * s], -1)
            Xt = np.stack([rt * c - r * s, rt * s + r * c], -1)
            Xtt = np.stack([rtt * c - 2 * rt * s - r * c, rtt * s + 2 * rt * c - r * s], -1)
            return X, Xt, Xtt
        raise ValueError(self.kind)

    def _radius(self, t):
        """r(t) = R0 (1 + sum_m A_m cos(k_m t + phi_m)) and its t-derivatives."""
        R0 = self.params["R0"]
        r = np.ones_like(t)
        rt = np.zeros_like(t)
        rtt = np.zeros_like(t)
        for k, A, ph in self.params["modes"]:
            arg = k * t + ph
            r = r + A * np.cos(arg)
            rt = rt - A * k * np.sin(arg)
            rtt = rtt - A * k * k * np.cos(arg)
        return R0 * r, R0 * rt, R0 * rtt


def ellipse(a, b, cx=0.0, cy=0.0):
    return Shape("ellipse", dict(a=a, b=b, cx=cx, cy=cy))


def polar(R0, modes, cx=0.0, cy=0.0):
    """modes: list of (k, amplitude, phase) for r = R0 (1 + sum A cos(k t + phase))."""
    return Shape("polar", dict(R0=R0, modes=[tuple(m) for m in modes], cx=cx, cy=cy))


def random_star(rng, R0_range=(0.3, 0.6), kmin=2, kmax=8, amp=0.15):
    """r = R0 (1 + sum_{k=kmin..kmax} a_k cos(k t + phi_k)), |a_k| <= amp/k, uniform phases."""
    R0 = rng.uniform(*R0_range)
    modes = []
    for k in range(kmin, kmax + 1):
        modes.append((k, rng.uniform(-amp / k, amp / k), rng.uniform(0.0, 2 * math.pi)))
    return polar(R0, modes)


# --------------------------------------------------------------------------- nodes
_GL8_X, _GL8_W = np.polynomial.legendre.leggauss(8)


def equal_arclength(shape: Shape, n: int, fine: int | None = None):
    """Nodes at equal arclength on `shape`, plus the tangent angle and length there.

    Returns dict(xy=(n,2), theta=(n,), L=float, t=(n,)). theta is the tangent angle
    unwrapped so that theta - 2*pi*j/n is periodic, theta[0] in (-pi, pi].
    The arclength s(t) is integrated spectrally on a fine grid and refined with
    8-point Gauss-Legendre on each fine cell, then inverted by Newton's method.
    """
    M = fine or max(16 * n, 8192)
    tf = 2 * math.pi * np.arange(M) / M
    _, Xt, _ = shape.eval(tf)
    speed = np.hypot(Xt[:, 0], Xt[:, 1])
    sh = np.fft.fft(speed) / M
    L = 2 * math.pi * sh[0].real
    k = np.fft.fftfreq(M, 1.0 / M)
    with np.errstate(divide="ignore", invalid="ignore"):
        g = np.where(k != 0, sh / (1j * k), 0.0)
    # s(t_m) = sh0 * t_m + sum_{k!=0} sh_k (e^{ik t_m} - 1)/(ik)
    s_fine = sh[0].real * tf + (np.fft.ifft(g) * M).real - g.sum().real

    def s_of(t):
        m = np.floor(t / (2 * math.pi) * M).astype(np.int64)
        m = np.clip(m, 0, M - 1)
        a = tf[m]
        half = 0.5 * (t - a)
        mid = 0.5 * (t + a)
        acc = np.zeros_like(t)
        for xg, wg in zip(_GL8_X, _GL8_W):
            _, d, _ = shape.eval(mid + half * xg)
            acc += wg * np.hypot(d[..., 0], d[..., 1])
        return s_fine[m] + half * acc

    target = L * np.arange(n) / n
    t = 2 * math.pi * np.arange(n) / n
    for _ in range(50):
        _, d, _ = shape.eval(t)
        sp = np.hypot(d[:, 0], d[:, 1])
        dt = (s_of(t) - target) / sp
        t = t - dt
        if np.max(np.abs(dt)) < 1e-15:
            break
    X, Xt, _ = shape.eval(t)
    theta = np.unwrap(np.arctan2(Xt[:, 1], Xt[:, 0]))
    theta = theta - 2 * math.pi * np.round((theta[0]) / (2 * math.pi))
    return dict(xy=np.ascontiguousarray(X), theta=theta, L=float(L), t=t)


# --------------------------------------------------------------------------- data
def exact_interior(kappa: float):
    """A solution of (Delta - kappa) u = 0: e^x sin y (kappa=0) or e^{ax} sin y, a^2 = kappa + 1."""
    a = math.sqrt(kappa + 1.0)

    def u(x, y):
        return np.exp(a * x) * np.sin(y)

    def grad(x, y):
        e = np.exp(a * x)
        return a * e * np.sin(y), e * np.cos(y)

    return u, grad


@dataclasses.dataclass
class Problem:
    """One interface problem: grid, box, operator and interface nodes."""

    name: str
    N: int
    box: tuple
    kappa: float
    boxbc: int
    xy: np.ndarray
    theta: np.ndarray
    L: float
    rhs: np.ndarray | None = None
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self):
        return self.xy.shape[0]


def interior_dirichlet(shape, N, n, box=(-1.0, 1.0, -1.0, 1.0), kappa=0.0, name="interior"):
    """Interior Dirichlet problem with boundary data from the closed-form solution."""
    nodes = equal_arclength(shape, n)
    u, _ = exact_interior(kappa)
    rhs = u(nodes["xy"][:, 0], nodes["xy"][:, 1])
    return Problem(name, N, box, kappa, BOX_DIRICHLET0, nodes["xy"], nodes["theta"], nodes["L"], rhs)


def config_small_laplace(N=128, n=128):
    """Ellipse 0.6 x 0.4 in [-1,1]^2, interior Dirichlet Laplace, data e^x sin y."""
    return interior_dirichlet(ellipse(0.6, 0.4), N, n, name=f"ellipse_laplace_{N}x{N}_n{n}")


def hele_shaw_shape():
    return polar(1.0, [(3, 0.1, 0.0), (5, 0.05, -math.pi / 2)])  # 1 + .1 cos3t + .05 sin5t


def config_hele_shaw(N=1024, n=1024, box=4.0):
    """Hele-Shaw bubble r = 1 + 0.1 cos 3t + 0.05 sin 5t in [-4,4]^2, free-space box data."""
    nodes = equal_arclength(hele_shaw_shape(), n)
    return Problem(f"hele_shaw_{N}x{N}_n{n}", N, (-box, box, -box, box), 0.0, BOX_FREESPACE_DL,
                   nodes["xy"], nodes["theta"], nodes["L"],
                   extra=dict(sigma=1e-3, J=1.0, dt=1e-3))


def stefan_shape():
    return polar(0.1, [(4, 0.2, 0.0)])


def config_stefan(N=2048, n=2048, box=2.0, dt=5e-4):
    """Stefan seed r = 0.1 (1 + 0.2 cos 4t) in [-2,2]^2, undercooling -0.5, Neumann box."""
    nodes = equal_arclength(stefan_shape(), n)
    return Problem(f"stefan_{N}x{N}_n{n}", N, (-box, box, -box, box), 3.0 / (2.0 * dt), BOX_NEUMANN0,
                   nodes["xy"], nodes["theta"], nodes["L"],
                   extra=dict(St=-0.5, eps_c=2e-3, eps_aniso=0.05, fold=4, eps_v=2e-3, dt=dt))


def config_batched(count=256, seed=MASTER_SEED):
    """Uneven interior Dirichlet instances: N in {128,256,512}, n in [64,512], kappa in {0,10,100}."""
    out = []
    for idx in range(count):
        rng = np.random.default_rng(seed + idx)
        N = int(rng.choice([128, 256, 512]))
        n = int(rng.integers(64, 513))
        kappa = float(rng.choice([0.0, 10.0, 100.0]))
        shape = random_star(rng)
        out.append(interior_dirichlet(shape, N, n, kappa=kappa, name=f"batch_{idx}"))
    return out


def random_problem(seed, N=64, n=64, kappa=0.0, boxbc=BOX_DIRICHLET0, box=1.0, R0=(0.35, 0.55)):
    """A small random star problem for parity tests (data e^x sin y style)."""
    rng = np.random.default_rng(seed)
    shape = random_star(rng, R0_range=R0)
    nodes = equal_arclength(shape, n)
    u, _ = exact_interior(kappa)
    rhs = u(nodes["xy"][:, 0], nodes["xy"][:, 1])
    return Problem(f"random_{seed}", N, (-box, box, -box, box), kappa, boxbc,
                   nodes["xy"], nodes["theta"], nodes["L"], rhs)


def random_density(seed, n, modes=8):
    """A smooth random periodic density sampled at alpha_j = 2 pi j / n."""
    rng = np.random.default_rng(seed)
    a = 2 * math.pi * np.arange(n) / n
    f = np.full(n, rng.normal())
    for k in range(1, modes + 1):
        f += rng.normal() / k ** 2 * np.cos(k * a) + rng.normal() / k ** 2 * np.sin(k * a)
    return f


def random_grid(seed, N, smooth=True):
    """A grid right-hand side for plain solver tests."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((N, N))
    return np.ascontiguousarray(g)


# ----------------------------------------------------------------------------- learned warm start
def random_harmonic(seed):
    """A random harmonic function u(x, y) for the boundary data of interior Laplace problems:
    a sum of e^{k x'} cos(k y' + b) terms in randomly rotated coordinates (each harmonic) plus a
    random harmonic quadratic a (x^2 - y^2) + c x y + d."""
    rng = np.random.default_rng(seed)
    terms = []
    for _ in range(int(rng.integers(1, 4))):
        th = rng.uniform(0.0, 2.0 * math.pi)
        k = rng.uniform(0.3, 2.5)
        terms.append((math.cos(th), math.sin(th), k, rng.uniform(0.0, 2.0 * math.pi), rng.normal()))
    a, c, d = rng.normal(), rng.normal(), rng.normal()

    def u(x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        out = a * (x * x - y * y) + c * x * y + d
        for ct, st, k, b, w in terms:
            xr, yr = ct * x + st * y, -st * x + ct * y
            out = out + w * np.exp(k * xr) * np.cos(k * yr + b)
        return out

    return u


def warmstart_problem(seed, N=256, n=None):
    """An interior Dirichlet Laplace problem for warm-start training and tests: a random star
    (config-4 shape family) in [-1, 1]^2 with random harmonic boundary data; n nodes
    (default: uniform in [64, 320], so that on the 256^2 grid the node spacing stays above
    the cell width, where GMRES converges fast)."""
    rng = np.random.default_rng(seed)
    shape = random_star(rng)
    if n is None:
        n = int(rng.integers(64, 321))
    nodes = equal_arclength(shape, n)
    u = random_harmonic(seed + 7919)
    rhs = u(nodes["xy"][:, 0], nodes["xy"][:, 1])
    return Problem(f"warmstart_{seed}", N, (-1.0, 1.0, -1.0, 1.0), 0.0, BOX_DIRICHLET0, nodes["xy"], nodes["theta"],
                   nodes["L"], rhs)


def mlp_init(seed, features=47, hidden=256):
    """Initial weights of the warm-start network (He-normal scaling by fan-in, zero biases),
    float32; drawn on the host so both the device path and the oracle start from them."""
    rng = np.random.default_rng(seed)
    return dict(
        W1=rng.normal(0.0, math.sqrt(2.0 / features), (hidden, features)).astype(np.float32),
        b1=np.zeros(hidden, dtype=np.float32),
        W2=rng.normal(0.0, math.sqrt(2.0 / hidden), (hidden, hidden)).astype(np.float32),
        b2=np.zeros(hidden, dtype=np.float32),
        w3=rng.normal(0.0, math.sqrt(1.0 / hidden), hidden).astype(np.float32),
        b3=np.float32(0.0),
    )
