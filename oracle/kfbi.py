"""Oracle for the kernel-free boundary integral (KFBI) apply: plain FP64 on the CPU.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the CPU
baseline of bench.py, never by the product path.

Each function restates one step of the method of Zhou, Li & Ying, "A Cartesian
grid-based boundary integral method for moving interface problems":

  Sec. 4.1, Table 2     jumps of the single/double layer: S psi -> (Phi, Psi) = (0, -psi),
                        D phi -> (phi, 0)
  App. A.1              [u] = Phi; 2x2 system for [u_x],[u_y]; 3x3 system for second jumps
  Sec. 4.2              corrected five-point scheme: C_ij = -(1/h^2){[u] + d[u_x] + d^2/2 [u_xx]}
                        at an irregular node, fast DST/DCT solve (matrix unchanged)
  Sec. 4.1 (box data)   free-space problems: Dirichlet box data = D phi by the trapezoidal rule
  Sec. 4.3              one-sided limits by 6-point Taylor interpolation with jump corrections;
                        boundary operator = average of the one-sided limits
  Sec. 3                boundary integral operators of the three BIEs

Readings where the paper is silent or garbled (the CUDA path takes the same ones):
  R1  cell-centred grid x_i = xmin + (i + 1/2) h (the paper's Sec. 4.2 is node-centred);
      Dirichlet-0 box -> DST-II, Neumann-0 box -> DCT-II, both exact for the 5-point matrix.
  R2  interface functions use the global trigonometric interpolant through the nodes at
      alpha_j = 2 pi j / n (Sec. 5 remark: spectral interface operations); for even n the
      Nyquist mode is the real term c cos(n alpha / 2).
  R3  crossings: bracket sign changes of (coordinate - line) on 8 sub-samples per node
      interval, Newton with bisection safeguard until |step| <= 1e-15. A crossing within
      1e-10 h of a grid node is placed on the node and on the arm that leaves the node toward
      the outside of the curve: a node on the curve is in the closed interior.
  R4  a node is in Omega+ iff an odd number of its row's crossings lie strictly left of
      it; an arm with two crossings (the curve dips between two same-side nodes) gets no
      correction; three or more crossings on an arm, or a vertical arm whose crossing
      count disagrees with the row classification, is an under-resolved interface.
  R5  correction sign for every arm pattern: C += -J/h^2 at an Omega+ node, +J/h^2 at an
      Omega- node, J = [u] + d[u_s] + d^2/2 [u_ss], d = (neighbour - crossing) along the arm.
  R6  Sec. 4.2 writes [u_yy] where [u_xx] is meant; the C(p) in Sec. 4.3 is C(q_m).
  R7  interior problems use a zero-Dirichlet box (the paper does not state it).
  R8  free-space box data is D phi only; the constant integral of phi of the modified
      double layer (Sec. 3.1) is added to the boundary operator after interpolation.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft as sfft

TWO_PI = 2.0 * math.pi

BOX_DIRICHLET0, BOX_NEUMANN0, BOX_FREESPACE_DL = 0, 1, 2
LAYER_SINGLE, LAYER_DOUBLE = 0, 1
BIE_INTERIOR_DL, BIE_HS_EXTERIOR_MDL, BIE_STEFAN_SL = 0, 1, 2

SUBSAMPLES = 8          # R3
NEWTON_TOL = 1e-15      # R3
SNAP_TOL = 1e-10        # R3 tie-break, in cells
NEWTON_MAXIT = 60
BOX_MARGIN_CELLS = 3.0  # the interface must stay this many cells inside the box


class KfbiError(Exception):
    pass


class OutsideBox(KfbiError):
    pass


class Underresolved(KfbiError):
    pass


class Singular(KfbiError):
    pass


# ============================================================================ grid
class Grid:
    """Cell-centred N x N grid on a square box (R1). Arrays are indexed [j, i] = [y, x]."""

    def __init__(self, N, box):
        xmin, xmax, ymin, ymax = (float(v) for v in box)
        self.N = int(N)
        self.xmin, self.xmax, self.ymin, self.ymax = xmin, xmax, ymin, ymax
        self.h = (xmax - xmin) / N
        hy = (ymax - ymin) / N
        if abs(hy - self.h) > 1e-12 * self.h:
            raise KfbiError("square cells required")
        idx = np.arange(self.N, dtype=np.float64)
        self.x = xmin + (idx + 0.5) * self.h
        self.y = ymin + (idx + 0.5) * self.h


# ============================================================================ interpolant
class Trig:
    """Trigonometric interpolant through samples f_j at alpha_j = 2 pi j / n (R2).

    f(alpha) = sum_{|k| <= K} c_k e^{i k alpha} + [n even] c_{n/2} cos(n alpha / 2),
    K = floor((n - 1) / 2), c_k = (1/n) sum_j f_j e^{-i k alpha_j}.
    """

    def __init__(self, f):
        f = np.asarray(f, dtype=np.float64)
        self.n = f.shape[0]
        c = np.fft.fft(f, axis=0) / self.n
        K = (self.n - 1) // 2
        self.k = np.arange(-K, K + 1)
        self.ck = c[self.k % self.n]
        self.nyq = c[self.n // 2].real if self.n % 2 == 0 else None

    def eval(self, alpha, d=0, chunk=256):
        """d-th derivative (d = 0, 1, 2) of the interpolant at the points alpha."""
        alpha = np.asarray(alpha, dtype=np.float64)
        fac = (1j * self.k) ** d
        outs = []
        for s in range(0, alpha.shape[0], chunk):
            a = alpha[s:s + chunk]
            E = np.exp(1j * np.outer(a, self.k)) * fac
            out = (E @ self.ck).real
            if self.nyq is not None:
                m = self.n // 2
                if d == 0:
                    t = np.cos(m * a)
                elif d == 1:
                    t = -m * np.sin(m * a)
                else:
                    t = -m * m * np.cos(m * a)
                out = out + (np.multiply.outer(t, self.nyq) if np.ndim(self.nyq) else t * self.nyq)
            outs.append(out)
        if not outs:
            return np.zeros((0,) + self.ck.shape[1:])
        return np.concatenate(outs, axis=0)


class Interface:
    """A closed CCW curve through the nodes X_j (App. A: normal n = (y_a, -x_a) / s_a)."""

    def __init__(self, xy):
        self.xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float64))
        self.n = self.xy.shape[0]
        self.alpha = TWO_PI * np.arange(self.n) / self.n
        self.X = Trig(self.xy)
        self.node = self.geom(self.alpha)

    def geom(self, alpha):
        P = self.X.eval(alpha, 0)
        D1 = self.X.eval(alpha, 1)
        D2 = self.X.eval(alpha, 2)
        g = dict(x=P[:, 0], y=P[:, 1], xa=D1[:, 0], ya=D1[:, 1], xaa=D2[:, 0], yaa=D2[:, 1])
        g["sa"] = np.hypot(g["xa"], g["ya"])
        g["nx"] = g["ya"] / g["sa"]
        g["ny"] = -g["xa"] / g["sa"]
        return g


# ============================================================================ crossings (R3)
class Crossings:
    """Intersections of the curve with grid lines.

    kind 0: horizontal line y = y_line, `xi` is the x of the crossing;
    kind 1: vertical line x = x_line, `xi` is the y of the crossing.
    `first` = index of the first grid node along the line with coordinate > xi,
    so the crossing lies on the arm (first - 1, first).
    """

    def __init__(self, kind, line, alpha, xi, first):
        self.kind, self.line, self.alpha, self.xi, self.first = kind, line, alpha, xi, first

    def __len__(self):
        return self.alpha.shape[0]


def _roots(trig_col, axis, lo, hi, lv, pos_lo):
    """Newton's method with a bisection safeguard on brackets [lo, hi] (R3)."""
    lo = lo.copy()
    hi = hi.copy()
    t = 0.5 * (lo + hi)
    active = np.ones(t.shape[0], dtype=bool)
    for _ in range(NEWTON_MAXIT):
        idx = np.nonzero(active)[0]
        if idx.size == 0:
            break
        tt = t[idx]
        f = trig_col.eval(tt, 0)[:, axis] - lv[idx]
        fp = trig_col.eval(tt, 1)[:, axis]
        same = (f >= 0.0) == pos_lo[idx]
        lo[idx] = np.where(same, tt, lo[idx])
        hi[idx] = np.where(same, hi[idx], tt)
        with np.errstate(divide="ignore", invalid="ignore"):
            tn = tt - f / fp
        bad = ~np.isfinite(tn) | (tn <= lo[idx]) | (tn >= hi[idx])
        tn = np.where(bad, 0.5 * (lo[idx] + hi[idx]), tn)
        done = np.abs(tn - tt) <= NEWTON_TOL
        t[idx] = tn
        active[idx[done]] = False
    return t


def find_crossings(iface: Interface, grid: Grid):
    """All crossings of the curve with the lines y = y_j and x = x_i."""
    n = iface.n
    M = SUBSAMPLES * n
    a = TWO_PI * np.arange(M) / M
    P = iface.X.eval(a, 0)
    h = grid.h
    m = BOX_MARGIN_CELLS * h
    if (P[:, 0].min() < grid.xmin + m or P[:, 0].max() > grid.xmax - m
            or P[:, 1].min() < grid.ymin + m or P[:, 1].max() > grid.ymax - m):
        raise OutsideBox("interface closer than 3h to the box")
    kinds, lines, alphas, xis, firsts = [], [], [], [], []
    for kind, axis, lines_v, along_v in ((0, 1, grid.y, grid.x), (1, 0, grid.x, grid.y)):
        c = P[:, axis]
        pos = c[:, None] >= lines_v[None, :]
        chg = pos != np.roll(pos, -1, axis=0)
        seg, li = np.nonzero(chg)
        lo = a[seg]
        hi = lo + TWO_PI / M
        t = _roots(iface.X, axis, lo, hi, lines_v[li], pos[seg, li])
        xi = iface.X.eval(t, 0)[:, 1 - axis]
        first = np.searchsorted(along_v, xi, side="right")
        # tie-break: a crossing within SNAP_TOL h of a node lies on the node, on the arm toward
        # the outside (outward normal (y_a, -x_a): +x on a horizontal line when y_a > 0, +y on a
        # vertical line when x_a < 0), so the node is in the closed interior
        lo_along = grid.xmin if kind == 0 else grid.ymin
        l = np.clip(np.rint((xi - lo_along) / h - 0.5).astype(np.int64), 0, grid.N - 1)
        near = np.abs(xi - along_v[l]) <= SNAP_TOL * h
        if np.any(near):
            d = iface.X.eval(t, 1)[:, axis]
            out_plus = d > 0.0 if kind == 0 else d < 0.0
            xi = np.where(near, along_v[l], xi)
            first = np.where(near, np.where(out_plus, l + 1, l), first)
        kinds.append(np.full(t.shape, kind))
        lines.append(li)
        alphas.append(t)
        xis.append(xi)
        firsts.append(first)
    cr = Crossings(*(np.concatenate(v) for v in (kinds, lines, alphas, xis, firsts)))
    if np.any(cr.first <= 0) or np.any(cr.first >= grid.N):
        raise OutsideBox("crossing outside the node range")
    return cr


# ============================================================================ classification (R4)
class Classification:
    """Node sides (1 = Omega+), crossings per arm and the irregular nodes (R4).

    hcount[j, i] / hid[j, i]: number of crossings on the arm (i-1, j)-(i, j) and, when
    there is exactly one, its index (else -1); vcount / vid likewise for the arm
    (i, j-1)-(i, j). An arm with two crossings joins two nodes on the same side: the
    curve dips between them and back, the five-point stencil sees no jump there and the
    arm gets no correction. Three or more crossings on one arm is under-resolved.
    """

    def __init__(self, cr: Crossings, grid: Grid):
        N = grid.N
        hcount = np.zeros((N, N), dtype=np.int64)
        vcount = np.zeros((N, N), dtype=np.int64)
        hid = -np.ones((N, N), dtype=np.int64)
        vid = -np.ones((N, N), dtype=np.int64)
        for c in range(len(cr)):
            line, first = int(cr.line[c]), int(cr.first[c])
            if cr.kind[c] == 0:
                hcount[line, first] += 1
                hid[line, first] = c
            else:
                vcount[first, line] += 1
                vid[first, line] = c
        if hcount.max(initial=0) >= 3 or vcount.max(initial=0) >= 3:
            raise Underresolved("three or more crossings on one arm")
        hid[hcount != 1] = -1
        vid[vcount != 1] = -1
        side = np.cumsum(hcount % 2, axis=1) % 2
        vdiff = side[1:, :] != side[:-1, :]
        if np.any(vdiff != (vcount[1:, :] % 2 == 1)):
            raise Underresolved("vertical arms disagree with the row classification")
        self.side = side.astype(np.uint8)
        self.hcount, self.vcount, self.hid, self.vid = hcount, vcount, hid, vid
        irr = np.zeros((N, N), dtype=bool)
        hd = side[:, 1:] != side[:, :-1]
        irr[:, 1:] |= hd
        irr[:, :-1] |= hd
        irr[1:, :] |= vdiff
        irr[:-1, :] |= vdiff
        self.irregular = irr

    def crossed_arms(self):
        """(kind, j, i, crossing) for every arm with exactly one crossing, kind 0 = horizontal."""
        hj, hi = np.nonzero(self.hid >= 0)
        vj, vi = np.nonzero(self.vid >= 0)
        kind = np.concatenate([np.zeros(hj.size, np.int64), np.ones(vj.size, np.int64)])
        j = np.concatenate([hj, vj])
        i = np.concatenate([hi, vi])
        c = np.concatenate([self.hid[hj, hi], self.vid[vj, vi]])
        return kind, j, i, c


# ============================================================================ jumps (App. A.1)
def jumps(iface: Interface, alpha, layer, density, kappa):
    """Jumps ([u], [u_x], [u_y], [u_xx], [u_yy], [u_xy]) of a layer potential at alpha.

    Table 2: double layer Phi = phi, Psi = 0; single layer Phi = 0, Psi = -psi.
    """
    n = iface.n
    zero = np.zeros(n)
    if layer == LAYER_DOUBLE:
        return jumps_from_data(iface, alpha, density, zero, kappa)
    return jumps_from_data(iface, alpha, zero, -np.asarray(density, dtype=np.float64), kappa)


def jumps_from_data(iface: Interface, alpha, Phi_nodes, Psi_nodes, kappa, f_jump=0.0):
    """Jumps of u for [u] = Phi, [du/dn] = Psi on the curve (App. A.1).

    [u] = Phi;  x_a [u_x] + y_a [u_y] = Phi_a;  y_a [u_x] - x_a [u_y] = s_a Psi;
    x_a^2 [u_xx] + y_a^2 [u_yy] + 2 x_a y_a [u_xy] = Phi_aa - x_aa [u_x] - y_aa [u_y];
    x_a y_a [u_xx] - x_a y_a [u_yy] + (y_a^2 - x_a^2) [u_xy]
        = s_aa Psi + s_a Psi_a - y_aa [u_x] + x_aa [u_y];
    [u_xx] + [u_yy] = c^2 Phi + [f].
    Phi and Psi are given at the nodes and enter through their trigonometric interpolants.
    """
    alpha = np.asarray(alpha, dtype=np.float64)
    g = iface.geom(alpha)
    m = alpha.shape[0]
    P, S = Trig(Phi_nodes), Trig(Psi_nodes)
    Phi, Phi_a, Phi_aa = P.eval(alpha, 0), P.eval(alpha, 1), P.eval(alpha, 2)
    Psi, Psi_a = S.eval(alpha, 0), S.eval(alpha, 1)
    xa, ya, xaa, yaa, sa = g["xa"], g["ya"], g["xaa"], g["yaa"], g["sa"]
    saa = (xa * xaa + ya * yaa) / sa
    A2 = np.empty((m, 2, 2))
    A2[:, 0, 0], A2[:, 0, 1] = xa, ya
    A2[:, 1, 0], A2[:, 1, 1] = ya, -xa
    b2 = np.stack([Phi_a, sa * Psi], -1)
    g1 = np.linalg.solve(A2, b2[..., None])[..., 0]
    ux, uy = g1[:, 0], g1[:, 1]
    A3 = np.empty((m, 3, 3))
    A3[:, 0, :] = np.stack([xa * xa, ya * ya, 2 * xa * ya], -1)
    A3[:, 1, :] = np.stack([xa * ya, -xa * ya, ya * ya - xa * xa], -1)
    A3[:, 2, :] = np.stack([np.ones(m), np.ones(m), np.zeros(m)], -1)
    b3 = np.stack([Phi_aa - xaa * ux - yaa * uy,
                   saa * Psi + sa * Psi_a - yaa * ux + xaa * uy,
                   kappa * Phi + f_jump], -1)
    g2 = np.linalg.solve(A3, b3[..., None])[..., 0]
    return np.stack([Phi, ux, uy, g2[:, 0], g2[:, 1], g2[:, 2]], -1)


# ============================================================================ corrected RHS (Sec. 4.2)
def correction_rhs(grid: Grid, cr: Crossings, cl: Classification, J):
    """Right-hand side of the corrected five-point scheme from the crossing jumps J (R5)."""
    N, h = grid.N, grid.h
    C = np.zeros((N, N))
    inv_h2 = 1.0 / (h * h)
    kind, aj, ai, ac = cl.crossed_arms()
    for a in range(kind.shape[0]):
        j, i, c = int(aj[a]), int(ai[a]), int(ac[a])
        xi = cr.xi[c]
        u0, ux, uy, uxx, uyy, _ = J[c]
        if kind[a] == 0:          # horizontal arm (i-1, j)-(i, j)
            d1, d2, along = ux, uxx, grid.x
            ends = [((j, i - 1), i), ((j, i), i - 1)]
        else:                     # vertical arm (i, j-1)-(i, j)
            d1, d2, along = uy, uyy, grid.y
            ends = [((j - 1, i), j), ((j, i), j - 1)]
        for (jj, ii), nb in ends:
            d = along[nb] - xi
            Jv = u0 + d * d1 + 0.5 * d * d * d2
            sgn = -1.0 if cl.side[jj, ii] == 1 else 1.0
            C[jj, ii] += sgn * Jv * inv_h2
    return C


def box_face_points(grid: Grid):
    """Midpoints of the outer faces of the boundary cells: west, east, south, north."""
    N = grid.N
    W = np.stack([np.full(N, grid.xmin), grid.y], -1)
    E = np.stack([np.full(N, grid.xmax), grid.y], -1)
    S = np.stack([grid.x, np.full(N, grid.ymin)], -1)
    Nn = np.stack([grid.x, np.full(N, grid.ymax)], -1)
    return W, E, S, Nn


def double_layer_direct(iface: Interface, phi, pts):
    """D phi at off-curve points by the composite trapezoidal rule (Sec. 4.1 box data).

    D phi(p) = int phi(y) d/dn_y G0(y - p) ds_y, G0 = ln|x| / (2 pi):
             ~ (1/n) sum_l phi_l (X_l - p) . (y_a, -x_a)_l / |X_l - p|^2.
    """
    g = iface.node
    out = np.empty(pts.shape[0])
    for s in range(0, pts.shape[0], 512):
        p = pts[s:s + 512]
        dx = iface.xy[None, :, 0] - p[:, None, 0]
        dy = iface.xy[None, :, 1] - p[:, None, 1]
        num = dx * g["ya"][None, :] - dy * g["xa"][None, :]
        out[s:s + 512] = (phi[None, :] * num / (dx * dx + dy * dy)).sum(1) / iface.n
    return out


def add_box_data(grid: Grid, C, gW, gE, gS, gN):
    """Inhomogeneous Dirichlet data g on a face: ghost u = 2g - u_0, so RHS -= 2 g / h^2."""
    f = 2.0 / (grid.h * grid.h)
    C[:, 0] -= f * gW
    C[:, -1] -= f * gE
    C[0, :] -= f * gS
    C[-1, :] -= f * gN
    return C


# ============================================================================ fast solve (Sec. 4.2)
def solve_grid(grid: Grid, C, kappa, boxbc):
    """(Delta_h - kappa) u = C with the box condition, by DST-II / DCT-II (R1).

    1-D eigenvalues: Dirichlet-0 (DST-II mode k = 0..N-1): (2 cos(pi (k+1)/N) - 2)/h^2;
    Neumann-0 (DCT-II mode k): (2 cos(pi k / N) - 2)/h^2, evaluated through the identity
    2 cos t - 2 = -4 sin^2(t/2), which keeps full relative precision for small t.
    """
    N, h = grid.N, grid.h
    k = np.arange(N, dtype=np.float64)
    if boxbc == BOX_NEUMANN0:
        if kappa == 0.0:
            raise Singular("Neumann box with kappa = 0")
        lam = -4.0 * np.sin(0.5 * np.pi * k / N) ** 2 / (h * h)
        F = sfft.dctn(C, type=2, norm="ortho")
        return sfft.idctn(F / (lam[:, None] + lam[None, :] - kappa), type=2, norm="ortho")
    lam = -4.0 * np.sin(0.5 * np.pi * (k + 1.0) / N) ** 2 / (h * h)
    F = sfft.dstn(C, type=2, norm="ortho")
    return sfft.idstn(F / (lam[:, None] + lam[None, :] - kappa), type=2, norm="ortho")


# ============================================================================ interpolation (Sec. 4.3)
STENCIL = ((0, 0), (1, 0), (0, 1), (0, -1), (-1, 0))


class Stencils:
    """Six interpolation points per interface node: closest node, its four neighbours
    and the diagonal (d1, d2) (Sec. 4.3)."""

    def __init__(self, iface: Interface, grid: Grid, side):
        p = iface.xy
        h = grid.h
        i0 = np.floor((p[:, 0] - grid.x[0]) / h + 0.5).astype(np.int64)
        j0 = np.floor((p[:, 1] - grid.y[0]) / h + 0.5).astype(np.int64)
        d1 = np.where(p[:, 0] > grid.x[i0], 1, -1)
        d2 = np.where(p[:, 1] > grid.y[j0], 1, -1)
        r = np.stack([np.full_like(i0, a) for a, _ in STENCIL] + [d1], -1)
        s = np.stack([np.full_like(j0, b) for _, b in STENCIL] + [d2], -1)
        self.qi = i0[:, None] + r
        self.qj = j0[:, None] + s
        if self.qi.min() < 0 or self.qj.min() < 0 or self.qi.max() >= grid.N or self.qj.max() >= grid.N:
            raise OutsideBox("interpolation stencil leaves the grid")
        self.dx = grid.x[self.qi] - p[:, 0:1]
        self.dy = grid.y[self.qj] - p[:, 1:2]
        dx, dy = self.dx, self.dy
        self.M = np.stack([np.ones_like(dx), dx, dy, 0.5 * dx * dx, dx * dy, 0.5 * dy * dy], -1)
        self.minus = side[self.qj, self.qi] == 0


def interpolate(st: Stencils, u, Jn, nx=None, ny=None):
    """One-sided values at the nodes from the grid function u (Sec. 4.3).

    Row m: v(q_m) + [q_m in Omega-] C(q_m) = v+ + dx v+_x + dy v+_y + dx^2/2 v+_xx
    + dx dy v+_xy + dy^2/2 v+_yy, C(q_m) = [v] + dx.[grad v] + dx^T [Hess v] dx / 2.
    Returns the average (v+ + v-)/2 = v+ - [v]/2 and, if the normal is given,
    n . (grad v+ + grad v-)/2.
    """
    dx, dy = st.dx, st.dy
    j0, jx, jy, jxx, jyy, jxy = (Jn[:, k:k + 1] for k in range(6))
    Cq = j0 + dx * jx + dy * jy + 0.5 * dx * dx * jxx + dx * dy * jxy + 0.5 * dy * dy * jyy
    b = u[st.qj, st.qi] + np.where(st.minus, Cq, 0.0)
    a = np.linalg.solve(st.M, b[..., None])[..., 0]
    val = a[:, 0] - 0.5 * Jn[:, 0]
    if nx is None:
        return val, None
    gx = a[:, 1] - 0.5 * Jn[:, 1]
    gy = a[:, 2] - 0.5 * Jn[:, 2]
    return val, nx * gx + ny * gy


# ============================================================================ the apply
class Kfbi:
    """Layer-potential apply on one grid (Sec. 4): density -> boundary operator values."""

    def __init__(self, N, box, kappa=0.0, boxbc=BOX_DIRICHLET0):
        self.grid = Grid(N, box)
        self.kappa = float(kappa)
        self.boxbc = int(boxbc)
        if self.boxbc == BOX_FREESPACE_DL and self.kappa != 0.0:
            raise KfbiError("free-space box data is for the Laplace double layer")
        if self.boxbc == BOX_NEUMANN0 and self.kappa == 0.0:
            raise Singular("Neumann box with kappa = 0")

    def set_interface(self, xy):
        self.iface = Interface(xy)
        self.cr = find_crossings(self.iface, self.grid)
        self.cl = Classification(self.cr, self.grid)
        self.st = Stencils(self.iface, self.grid, self.cl.side)
        return self

    def jumps_all(self, layer, density):
        """Jumps at every crossing and at every node."""
        Jc = jumps(self.iface, self.cr.alpha, layer, density, self.kappa)
        Jn = jumps(self.iface, self.iface.alpha, layer, density, self.kappa)
        return Jc, Jn

    def rhs(self, layer, density, Jc=None):
        if Jc is None:
            Jc = jumps(self.iface, self.cr.alpha, layer, density, self.kappa)
        C = correction_rhs(self.grid, self.cr, self.cl, Jc)
        if self.boxbc == BOX_FREESPACE_DL:
            if layer != LAYER_DOUBLE:
                raise KfbiError("free-space box data is for the double layer")
            faces = box_face_points(self.grid)
            gs = [double_layer_direct(self.iface, density, f) for f in faces]
            C = add_box_data(self.grid, C, *gs)
        return C

    def apply(self, layer, density, want_dnormal=False):
        """Returns (values, dnormal or None, grid solution u)."""
        density = np.asarray(density, dtype=np.float64)
        Jc, Jn = self.jumps_all(layer, density)
        C = self.rhs(layer, density, Jc)
        u = solve_grid(self.grid, C, self.kappa, self.boxbc)
        g = self.iface.node
        if want_dnormal:
            val, dn = interpolate(self.st, u, Jn, g["nx"], g["ny"])
        else:
            val, dn = interpolate(self.st, u, Jn)
        return val, dn, u

    def interp_smooth(self, u):
        """Values of a smooth grid function at the nodes (zero jumps)."""
        val, _ = interpolate(self.st, u, np.zeros((self.iface.n, 6)))
        return val

    def arclength_integral(self, f):
        """int_Gamma f ds by the trapezoidal rule in alpha."""
        return float((f * self.iface.node["sa"]).sum() * TWO_PI / self.iface.n)

    def bie_matvec(self, kind, x, eps_v=None):
        """The three boundary integral operators (Sec. 3).

        interior double layer:  (1/2) phi + D phi                      (R7)
        Hele-Shaw exterior:     -(1/2) phi + D phi + int phi ds        (Sec. 3.1)
        Stefan single layer:    eps_V psi - S psi                      (Sec. 3.2)
        """
        if kind == BIE_INTERIOR_DL:
            v, _, _ = self.apply(LAYER_DOUBLE, x)
            return 0.5 * x + v
        if kind == BIE_HS_EXTERIOR_MDL:
            v, _, _ = self.apply(LAYER_DOUBLE, x)
            return -0.5 * x + v + self.arclength_integral(x)
        if kind == BIE_STEFAN_SL:
            v, _, _ = self.apply(LAYER_SINGLE, x)
            return eps_v * x - v
        raise KfbiError("unknown BIE kind")


def irregular_list(cl: Classification):
    """Irregular nodes in row-major order as (j, i) pairs."""
    j, i = np.nonzero(cl.irregular)
    return np.stack([j, i], -1)
