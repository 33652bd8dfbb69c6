"""theta-L interface evolution with small-scale decomposition (Sec. 5), plain FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

State: eta = theta - alpha at the nodes (Sec. 5.3 remark), length L, mean position
Xbar, and the Adams-Bashforth history (M, Q, N-hat, L at the previous level).

Readings where the paper is silent or its printed formulas are in error (the CUDA path takes the same ones):
  T1  L_t = + int theta_a U da (Sec. 5.1); the sign printed in the Adams-Bashforth
      formula of Sec. 5.3 and its missing factor 1/2 are taken as typos:
      L^{n+1} = L^n + (tau/2)(3 M^n - M^{n-1}), M = int theta_a U da; same for Xbar.
  T2  theta_t = (2 pi / L)(theta_a V - U_a) (Sec. 5.1); N = that minus the stiff part.
  T3  Hele-Shaw stiff part L2 with lambda_2 = sigma (Sec. 5.2.1): symbol -sigma (2pi/L)^3 |k|^3.
      Stefan case I (eps_V > 0) stiff part L1, lambda_1 = max |eps_C / eps_V| (Sec. 5.3):
      symbol -lambda_1 (2pi/L)^2 k^2. Stefan case II (eps_V = 0, the first-kind equation of
      Sec. 5.2.2) stiff part L2, lambda_2 = max |2 eps_C|: symbol -lambda_2 (2pi/L)^3 |k|^3.
      The explicit Adams-Bashforth scheme of the stability test (Sec. 6.2.2) is the same update
      with no stiff part (symbol 0: both propagators 1, N the whole right-hand side).
  T4  first step: the history equals the current level (M^{-1} = M^0, ...).
  T5  reconstruction: X_a = (L/2pi)(cos theta, sin theta) with its mean removed (closure),
      integrated spectrally, shifted so that the node mean is Xbar; Nyquist mode dropped.
  T6  Stefan step with lagged geometry: T^{n+1} is solved with interface conditions on
      Gamma^n, its psi is U^n; BDF2 from the first step with T^{-1} = T^0 so that the
      operator (Delta - 3/(2 tau)) never changes; T^0 = 0 in the seed, St outside.
  T7  anisotropic surface tension eps_C = eps (1 - a cos(m (theta - pi/2))), the angle of
      the outward normal (sin theta, -cos theta) being theta - pi/2.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import kfbi as K
from .gmres import gmres

TWO_PI = 2.0 * math.pi


def wavenumbers(n):
    return np.fft.fftfreq(n, 1.0 / n)


def spec_deriv(f, d=1):
    """d-th derivative at the nodes; for even n the Nyquist mode of odd derivatives is zero."""
    n = f.shape[0]
    k = wavenumbers(n)
    mult = (1j * k) ** d
    if n % 2 == 0 and d % 2 == 1:
        mult[n // 2] = 0.0
    return np.fft.ifft(np.fft.fft(f) * mult).real


def cumulative_integral(f):
    """int_0^{alpha_j} f(a) da for the trigonometric interpolant of f."""
    n = f.shape[0]
    c = np.fft.fft(f) / n
    k = wavenumbers(n)
    g = np.zeros(n, dtype=complex)
    mask = k != 0
    if n % 2 == 0:
        mask[n // 2] = False
    g[mask] = c[mask] / (1j * k[mask])
    alpha = TWO_PI * np.arange(n) / n
    per = (np.fft.ifft(g) * n).real
    return c[0].real * alpha + per - g.sum().real


def reconstruct(eta, L, Xbar):
    """Nodes of the curve from (eta, L, Xbar) (T5)."""
    n = eta.shape[0]
    alpha = TWO_PI * np.arange(n) / n
    th = alpha + eta
    Xa = (L / TWO_PI) * np.stack([np.cos(th), np.sin(th)], -1)
    c = np.fft.fft(Xa, axis=0)
    k = wavenumbers(n)
    Xh = np.zeros_like(c)
    mask = k != 0
    if n % 2 == 0:
        mask[n // 2] = False
    Xh[mask] = c[mask] / (1j * k[mask])[:, None]
    Xh[0] = np.asarray(Xbar) * n
    return np.ascontiguousarray(np.fft.ifft(Xh, axis=0).real)


@dataclasses.dataclass
class State:
    eta: np.ndarray
    L: float
    Xbar: np.ndarray
    t: float = 0.0
    steps: int = 0
    M_prev: float = 0.0
    Q_prev: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(2))
    N_prev: np.ndarray | None = None
    L_prev: float = 0.0
    density: np.ndarray | None = None
    T: np.ndarray | None = None
    T_prev: np.ndarray | None = None
    A0: float | None = None          # scaled-frame area (rescaled Hele-Shaw runs)
    last: dict = dataclasses.field(default_factory=dict)


def state_from_nodes(xy, theta, L):
    """theta-L state from equal-arclength nodes and their tangent angles."""
    n = xy.shape[0]
    alpha = TWO_PI * np.arange(n) / n
    return State(eta=np.asarray(theta, float) - alpha, L=float(L), Xbar=xy.mean(0))


def _advance(st: State, U, dt, stiff_symbol_fn):
    """Semi-implicit update of (eta, L, Xbar) from the normal velocity U (Sec. 5.3)."""
    n = st.eta.shape[0]
    alpha = TWO_PI * np.arange(n) / n
    th = alpha + st.eta
    th_a = 1.0 + spec_deriv(st.eta)
    L = st.L
    thU = th_a * U
    M = TWO_PI * thU.mean()
    V = (alpha / TWO_PI) * M - cumulative_integral(thU)
    s_vec = np.stack([np.cos(th), np.sin(th)], -1)
    n_vec = np.stack([np.sin(th), -np.cos(th)], -1)
    Q = (U[:, None] * n_vec + V[:, None] * s_vec).mean(0)
    U_a = spec_deriv(U)
    rhs = (TWO_PI / L) * (th_a * V - U_a)
    eta_h = np.fft.fft(st.eta)
    sym_n = stiff_symbol_fn(L)
    N_h = np.fft.fft(rhs) - sym_n * eta_h
    if st.steps == 0:
        M_prev, Q_prev, N_prev, L_prev = M, Q, N_h, L
    else:
        M_prev, Q_prev, N_prev, L_prev = st.M_prev, st.Q_prev, st.N_prev, st.L_prev
    L_new = L + 0.5 * dt * (3.0 * M - M_prev)
    e1, e2 = st_propagators(stiff_symbol_fn, dt, L_prev, L, L_new)
    eta_h_new = ssd_ab2(eta_h, N_h, N_prev, e1, e2, dt)
    Xbar_new = st.Xbar + 0.5 * dt * (3.0 * Q - Q_prev)
    st.M_prev, st.Q_prev, st.N_prev, st.L_prev = M, Q, N_h, L
    st.eta = np.fft.ifft(eta_h_new).real
    st.L = L_new
    st.Xbar = Xbar_new
    st.t += dt
    st.steps += 1
    st.last.update(M=M, Q=Q, U=U, V=V)
    return st


def ssd_ab2(eta_h, N_h, N_prev, e1, e2, dt):
    """The semi-implicit update of Sec. 5.3 in Fourier space: the stiff part is integrated
    exactly by the propagators e1 = e_k(t_n, t_{n+1}), e2 = e_k(t_{n-1}, t_{n+1}), the
    remainder N by second-order Adams-Bashforth:
    eta^{n+1} = e1 eta^n + (dt/2)(3 e1 N^n - e2 N^{n-1})."""
    return e1 * eta_h + 0.5 * dt * (3.0 * e1 * N_h - e2 * N_prev)


def st_propagators(stiff_symbol_fn, dt, L_prev, L, L_new):
    """e_k(t_n, t_{n+1}) and e_k(t_{n-1}, t_{n+1}) of Sec. 5.3 from the stiff symbol.

    The symbol is -lam (2 pi / L)^p |k|^p, so the exponents are trapezoidal sums of
    the symbol over the levels: e1 = exp(dt/2 (s(L^n) + s(L^{n+1}))),
    e2 = exp(dt (s(L^{n-1})/2 + s(L^n) + s(L^{n+1})/2)).
    """
    sp, sn, snew = stiff_symbol_fn(L_prev), stiff_symbol_fn(L), stiff_symbol_fn(L_new)
    e1 = np.exp(0.5 * dt * (sn + snew))
    e2 = np.exp(dt * (0.5 * sp + sn + 0.5 * snew))
    return e1, e2


def hs_symbol(n, sigma):
    k = np.abs(wavenumbers(n))
    return lambda L: -sigma * (TWO_PI / L) ** 3 * k ** 3


def stefan_symbol(n, lam1):
    k = wavenumbers(n)
    return lambda L: -lam1 * (TWO_PI / L) ** 2 * k ** 2


def stefan_symbol_case2(n, lam2):
    """Case II (eps_V = 0): third-order stiffness -lam2 (2 pi / L)^3 |k|^3 (Sec. 5.2.2, 5.3)."""
    k = np.abs(wavenumbers(n))
    return lambda L: -lam2 * (TWO_PI / L) ** 3 * k ** 3


def no_symbol(n):
    """The explicit scheme: no stiff part is split off."""
    return lambda L: np.zeros(n)


def _pad_spectrum(F):
    """Unnormalised DFT of length n of a trigonometric interpolant (R2) -> the DFT of length 2n of
    the same interpolant: modes |k| < n/2 kept, the Nyquist cosine split between +-n/2, times 2."""
    n = F.shape[0]
    m = 2 * n
    G = np.zeros(m, dtype=complex)
    K = (n - 1) // 2
    G[:K + 1] = F[:K + 1]
    if K > 0:
        G[m - K:] = F[n - K:]
    if n % 2 == 0:
        G[n // 2] = 0.5 * F[n // 2]
        G[m - n // 2] = 0.5 * F[n // 2]
    return 2.0 * G


def upsample(f):
    """Values at alpha = 2 pi j / (2n) of the trigonometric interpolant of f_j (j < n)."""
    return np.fft.ifft(_pad_spectrum(np.fft.fft(f))).real


def refine_markers(st: State):
    """Doubles the marker count (Sec. 6.1.4: markers are refined once their spacing exceeds
    1.5 h): eta, the density and the Adams-Bashforth history N-hat are carried over as the same
    trigonometric interpolants on twice as many equally spaced parameters; L, Xbar and the
    scalar history are unchanged, so the curve and its equal-arclength parametrisation are kept."""
    st.eta = upsample(st.eta)
    if st.density is not None:
        st.density = upsample(st.density)
    if st.N_prev is not None:
        st.N_prev = _pad_spectrum(st.N_prev)
    return st


def scaled_frame(st: State):
    """(R, physical time) of a rescaled run at scaled time st.t (see hs_step)."""
    return math.exp(st.t), (st.A0 / math.pi) * (math.exp(2.0 * st.t) - 1.0) / 2.0


def hs_step(solver: K.Kfbi, st: State, dt, sigma, J, tol=1e-8, restart=100, max_iter=500, refine_ratio=0.0,
            rescale=False):
    """One Hele-Shaw time step (Sec. 3.1 BIE, Sec. 5.2.1 SSD, Sec. 5.3 scheme).

    p = v + w, v = -J ln|x|; -1/2 phi + D phi + int phi = -sigma kappa - v on Gamma;
    U = -dp/dn from the oil side = J x.n/|x|^2 - dn(D phi) (the double layer's normal
    derivative is continuous across Gamma).

    refine_ratio > 0: the markers are doubled first while L / n > refine_ratio h (Sec. 6.1.4).
    rescale: the step is taken in the scaled frame of the long-time computation (Sec. 6.1.4, the
    rescaling is cited there, not printed; reading): x = R(tb) xb with R = e^{tb}, physical time
    dt/dtb = (A0/pi) R^2, A0 the scaled area at the start. The scaled problem is the same BIE with
    surface tension sigma / R, and the scaled normal velocity is (A0/pi) U - xb.n, which keeps the
    scaled area at A0 when J = 1. st.t is the scaled time (scaled_frame gives R and t).
    """
    if refine_ratio > 0.0:
        while st.L / st.eta.shape[0] > refine_ratio * solver.grid.h:
            refine_markers(st)
    n = st.eta.shape[0]
    alpha = TWO_PI * np.arange(n) / n
    X = reconstruct(st.eta, st.L, st.Xbar)
    solver.set_interface(X)
    th = alpha + st.eta
    th_a = 1.0 + spec_deriv(st.eta)
    curv = (TWO_PI / st.L) * th_a
    r2 = X[:, 0] ** 2 + X[:, 1] ** 2
    sig = sigma
    if rescale:
        if st.A0 is None:
            st.A0 = area(X)
        sig = sigma / math.exp(st.t)
    rhs = -sig * curv + J * 0.5 * np.log(r2)
    x0 = st.density if st.density is not None else np.zeros(n)
    phi, info = gmres(lambda x: solver.bie_matvec(K.BIE_HS_EXTERIOR_MDL, x), rhs, x0=x0,
                      tol=tol, restart=restart, max_iter=max_iter)
    _, dn, _ = solver.apply(K.LAYER_DOUBLE, phi, want_dnormal=True)
    nx, ny = np.sin(th), -np.cos(th)
    U = J * (X[:, 0] * nx + X[:, 1] * ny) / r2 - dn
    lam = sig
    if rescale:
        c = st.A0 / math.pi
        U = c * U - (X[:, 0] * nx + X[:, 1] * ny)
        lam = c * sig
    st.density = phi
    st.last.update(info=info, X=X, rhs=rhs, phi=phi)
    return _advance(st, U, dt, hs_symbol(n, lam))


def stefan_eps_c(theta, eps, aniso, fold):
    return eps * (1.0 - aniso * np.cos(fold * (theta - 0.5 * math.pi)))


def stefan_step(solver: K.Kfbi, st: State, dt, St, eps_c, eps_aniso, fold, eps_v,
                tol=1e-8, restart=100, max_iter=500, scheme="semi-implicit"):
    """One Stefan time step (Sec. 3.2 split T = T1 + T2, Sec. 5.2.2 cases I and II, Sec. 5.3).

    (Delta_h - c^2) T1 = (T^{n-1} - 4 T^n)/(2 tau) in the Neumann box;
    eps_V psi - S psi = -eps_C kappa - T1 on Gamma; U = psi; T^{n+1} = T1 - (S psi)_h.
    eps_V > 0: case I stiff part; eps_V = 0: case II (first-kind equation, third-order stiff part).
    scheme "explicit": the Adams-Bashforth scheme without the stiff part (Sec. 6.2.2).
    """
    n = st.eta.shape[0]
    alpha = TWO_PI * np.arange(n) / n
    X = reconstruct(st.eta, st.L, st.Xbar)
    solver.set_interface(X)
    grid = solver.grid
    if st.T is None:
        T0 = np.where(solver.cl.side == 1, 0.0, St).astype(np.float64)
        st.T, st.T_prev = T0, T0.copy()
    T1 = K.solve_grid(grid, (st.T_prev - 4.0 * st.T) / (2.0 * dt), solver.kappa, K.BOX_NEUMANN0)
    T1n = solver.interp_smooth(T1)
    th = alpha + st.eta
    th_a = 1.0 + spec_deriv(st.eta)
    curv = (TWO_PI / st.L) * th_a
    ec = stefan_eps_c(th, eps_c, eps_aniso, fold)
    ev = np.full(n, eps_v)
    rhs = -ec * curv - T1n
    x0 = st.density if st.density is not None else np.zeros(n)
    psi, info = gmres(lambda x: solver.bie_matvec(K.BIE_STEFAN_SL, x, eps_v=ev), rhs, x0=x0,
                      tol=tol, restart=restart, max_iter=max_iter)
    _, _, Sgrid = solver.apply(K.LAYER_SINGLE, psi)
    T_new = T1 - Sgrid
    st.T_prev, st.T = st.T, T_new
    st.density = psi
    if eps_v > 0.0:
        lam1 = float(np.max(np.abs(ec / ev)))
        sym = stefan_symbol(n, lam1)
        st.last.update(lam1=lam1)
    else:
        lam2 = float(np.max(np.abs(2.0 * ec)))
        sym = stefan_symbol_case2(n, lam2)
        st.last.update(lam2=lam2)
    if scheme == "explicit":
        sym = no_symbol(n)
    elif scheme != "semi-implicit":
        raise ValueError(scheme)
    st.last.update(info=info, X=X, rhs=rhs, psi=psi)
    return _advance(st, psi, dt, sym)


def area(X):
    """Enclosed area (1/2) int x . n ds of the trigonometric interpolant (Sec. 6.1.1)."""
    xa = spec_deriv(X[:, 0])
    ya = spec_deriv(X[:, 1])
    return 0.5 * np.mean(X[:, 0] * ya - X[:, 1] * xa) * TWO_PI


def length(X):
    xa = spec_deriv(X[:, 0])
    ya = spec_deriv(X[:, 1])
    return np.mean(np.hypot(xa, ya)) * TWO_PI
