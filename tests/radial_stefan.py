"""Radially symmetric reference for the Stefan time step (Sec. 3.2, Sec. 5.3), for the pins.

Independent of oracle/: a circle of radius R in an isotropic material stays a circle, so one
step of the time-discrete Stefan problem reduces to an ordinary differential equation in r
that has a closed-form homogeneous part (modified Bessel functions, scipy.special) and a
particular part given by the radial Green's function:

  (1/r)(r T')' - c^2 T = g(r),  g = (T^{n-1} - 4 T^n) / (2 tau),  c^2 = 3 / (2 tau)
  T_p(r) = -K0(cr) int_0^r I0(cs) g(s) s ds - I0(cr) int_r^inf K0(cs) g(s) s ds
  T = T_p + a I0(cr) (r < R),  T = T_p + b K0(cr) (r > R)

with the interface conditions of the step on the current circle: T continuous, the
Gibbs-Thomson relation T(R) = -eps_C / R - eps_V U (curvature 1/R of a CCW circle) and the
Stefan condition U = T'(R-) - T'(R+) (the jump inside minus outside across the outward
normal). The radius then moves by second-order Adams-Bashforth in the normal velocity,
R^{n+1} = R^n + (tau/2)(3 U^n - U^{n-1}) (the length equation L_t = int theta_a U da of
Sec. 5.1 for a circle, L = 2 pi R), with U^{-1} = U^0 on the first step. The first step uses
T^{-1} = T^0; the seed is T = 0 inside and St outside (Sec. 2.2).

Integrals are taken on a fine uniform grid in r by the trapezoidal rule with exponentially
scaled Bessel functions (scipy.special.ive / kve), so nothing overflows.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.signal as ss
import scipy.special as sp


class RadialStefan:
    def __init__(self, R0, St, eps_c, eps_v, rmax=1.5, M=60000):
        self.r = np.linspace(0.0, rmax, M + 1)
        self.dr = self.r[1] - self.r[0]
        self.R = float(R0)
        self.T = np.where(self.r < R0, 0.0, St)
        self.T_prev = self.T.copy()
        self.eps_c, self.eps_v = eps_c, eps_v
        self.U_prev = None
        self.history = []

    def particular(self, g, c):
        r, dr = self.r, self.dr
        x = c * r
        iv = sp.ive(0, x)
        kv = np.where(r > 0, sp.kve(0, np.maximum(x, 1e-300)), 0.0)
        e = math.exp(-c * dr)
        fa = iv * g * r
        fb = kv * g * r
        ua = np.zeros_like(r)
        ua[1:] = 0.5 * dr * (fa[1:] + e * fa[:-1])
        A = ss.lfilter([1.0], [1.0, -e], ua)
        ub = np.zeros_like(r)
        ub[:-1] = 0.5 * dr * (fb[:-1] + e * fb[1:])
        B = ss.lfilter([1.0], [1.0, -e], ub[::-1])[::-1]
        return -(kv * A + iv * B)

    def velocity_and_field(self, tau):
        c = math.sqrt(1.5 / tau)
        g = (self.T_prev - 4.0 * self.T) / (2.0 * tau)
        Tp = self.particular(g, c)
        R = self.R
        x = c * R
        i0, i1, k0, k1 = sp.iv(0, x), sp.iv(1, x), sp.kv(0, x), sp.kv(1, x)
        q = c * (i1 / i0 + k1 / k0)              # U = q v, v = a I0(cR) = b K0(cR)
        v = (-self.eps_c / R - float(np.interp(R, self.r, Tp))) / (1.0 + self.eps_v * q)
        rr = np.maximum(self.r, 1e-300)
        hom = np.where(self.r < R, v * sp.iv(0, c * self.r) / i0, v * sp.kv(0, c * rr) / k0)
        return v * q, Tp + hom

    def step(self, tau):
        U, T_new = self.velocity_and_field(tau)
        self.T_prev, self.T = self.T, T_new
        Up = U if self.U_prev is None else self.U_prev
        self.R = self.R + 0.5 * tau * (3.0 * U - Up)
        self.U_prev = U
        self.history.append(dict(R=self.R, U=U, T=T_new))
        return U

    def at(self, radii):
        return np.interp(radii, self.r, self.T)
