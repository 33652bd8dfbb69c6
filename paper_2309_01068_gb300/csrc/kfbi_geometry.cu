// Interface geometry on the device (kfbi_set_interface): trigonometric interpolant of the
// nodes, crossings of the curve with the grid lines, node classification, irregular nodes
// with their crossed arms (Sec. 4.2) and the 6-point interpolation stencils (Sec. 4.3).
#include <cmath>

#include "kfbi_fft.cuh"
#include "kfbi_internal.cuh"

namespace kfbi {

// --------------------------------------------------------------------------- interpolant
// Real function f(alpha) = c_0 + 2 sum_{k=1}^{K} Re(c_k e^{ik alpha}) + nyq cos(n alpha / 2)
// with K = (n-1)/2 and nyq = c_{n/2} for even n. A warp evaluates f, f', f'' at one
// alpha: lane l sums the modes [k0_l, k0_l + chunk) (k0_l = 1 + l chunk) from its start
// e^{i k0_l alpha}; all lanes return the full sums. The float64 pipe has a long latency,
// so the rotation runs as four interleaved recurrences (phases k0 + q, q = 0..3, advanced
// by e^{4 i alpha}) instead of one.
struct TrigSums {
  double f, f1, f2;
};

// e^{i k0_l alpha} of this lane, e^{i alpha} and e^{i n alpha / 2}
struct TrigStart {
  double2 e0, s1, q;
};

__device__ __forceinline__ int trig_k0(int n, int lane) {
  const int K = (n - 1) / 2;
  return 1 + lane * ((K + 31) / 32);
}

// starts from sincos at an arbitrary alpha
__device__ __forceinline__ TrigStart trig_start(int n, double alpha, int lane) {
  TrigStart t;
  double sn, cs;
  sincos((double)trig_k0(n, lane) * alpha, &sn, &cs);
  t.e0 = make_double2(cs, sn);
  sincos(alpha, &sn, &cs);
  t.s1 = make_double2(cs, sn);
  sincos(0.5 * (double)n * alpha, &sn, &cs);
  t.q = make_double2(cs, sn);
  return t;
}

// starts at alpha = 2 pi s / M from the table tw[m] = e^{2 pi i m / M} (exact index arithmetic)
__device__ __forceinline__ TrigStart trig_start_table(const double2* tw, int M, long s, int n, int lane) {
  TrigStart t;
  t.e0 = tw[((long)trig_k0(n, lane) * s) % M];
  t.s1 = tw[s % M];
  t.q = tw[((long)(n / 2) * s) % M];
  return t;
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ TrigSums trig_sums(const double2* c, int n, const TrigStart& st, int lane, bool d2) {
  const int K = (n - 1) / 2;
  const int chunk = (K + 31) / 32;
  const int k0 = 1 + lane * chunk;
  const int k1 = min(K + 1, k0 + chunk);
  double f[4] = {0.0, 0.0, 0.0, 0.0}, g[4] = {0.0, 0.0, 0.0, 0.0}, h[4] = {0.0, 0.0, 0.0, 0.0};
  if (k0 < k1) {
    const double2 s1 = st.s1;
    const double2 s2 = zmul(s1, s1);
    const double2 s3 = zmul(s2, s1);
    const double2 s4 = zmul(s2, s2);
    double2 e[4] = {st.e0, zmul(st.e0, s1), zmul(st.e0, s2), zmul(st.e0, s3)};
    for (int k = k0; k < k1; k += 4) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int kk = k + q;
        if (kk < k1) {
          const double2 ck = c[kk];
          const double re = ck.x * e[q].x - ck.y * e[q].y;
          const double im = ck.x * e[q].y + ck.y * e[q].x;
          f[q] += re;
          g[q] -= (double)kk * im;
          if (d2) h[q] -= (double)kk * (double)kk * re;
          e[q] = zmul(e[q], s4);
        }
      }
    }
  }
  double F = 2.0 * warp_sum((f[0] + f[1]) + (f[2] + f[3]));
  double F1 = 2.0 * warp_sum((g[0] + g[1]) + (g[2] + g[3]));
  double F2 = d2 ? 2.0 * warp_sum((h[0] + h[1]) + (h[2] + h[3])) : 0.0;
  F += c[0].x;
  if ((n & 1) == 0) {
    const double m = 0.5 * n;
    const double nyq = c[n / 2].x;
    F += nyq * st.q.x;
    F1 -= m * nyq * st.q.y;
    if (d2) F2 -= m * m * nyq * st.q.x;
  }
  return TrigSums{F, F1, F2};
}

__device__ __forceinline__ TrigSums trig_warp(const double2* c, int n, double alpha, int lane, bool d2) {
  return trig_sums(c, n, trig_start(n, alpha, lane), lane, d2);
}

// fine-grid twiddles e^{2 pi i m / M}
__global__ void k_twiddles_M(int M, double2* tw) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  double s, c;
  sincospi(2.0 * (double)m / (double)M, &s, &c);
  tw[m] = make_double2(c, s);
}

// twiddles e^{2 pi i m / n} in float64 and float32
__global__ void k_twiddles_n(int n, double2* tw, float2* tw_f) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  double s, c;
  sincospi(2.0 * (double)m / (double)n, &s, &c);
  tw[m] = make_double2(c, s);
  tw_f[m] = make_float2((float)c, (float)s);
}

// c_k = (1/n) sum_j f_j e^{-2 pi i k j / n}, k = 0..n/2, for `nf` functions stored with
// stride `stride` (function q at f[j*stride + q]); one warp per (function, k).
__global__ void k_dft_real(const double* f, int stride, int nf, int n, const double2* tw, double2* coef) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  int nk = n / 2 + 1;
  if (warp >= nk * nf) return;
  int q = warp / nk, k = warp - q * nk;
  // twiddle index k j mod n advanced by k 32 mod n (no division in the loop); two
  // accumulator pairs shorten the float64 dependency chains
  int idx = (int)(((long)k * lane) % n);
  const int step = (int)(((long)k * 32) % n);
  double re0 = 0.0, im0 = 0.0, re1 = 0.0, im1 = 0.0;
  int j = lane;
  for (; j + 32 < n; j += 64) {
    const double v0 = f[(long)j * stride + q], v1 = f[(long)(j + 32) * stride + q];
    const double2 w0 = tw[idx];
    idx += step;
    if (idx >= n) idx -= n;
    const double2 w1 = tw[idx];
    idx += step;
    if (idx >= n) idx -= n;
    re0 += v0 * w0.x;
    im0 -= v0 * w0.y;
    re1 += v1 * w1.x;
    im1 -= v1 * w1.y;
  }
  if (j < n) {
    const double v = f[(long)j * stride + q];
    const double2 w = tw[idx];
    re0 += v * w.x;
    im0 -= v * w.y;
  }
  const double re = warp_sum(re0 + re1);
  const double im = warp_sum(im0 + im1);
  if (lane == 0) coef[q * nk + k] = make_double2(re / n, im / n);
}

// fine samples X(alpha_s), alpha_s = 2 pi s / M; flags samples closer than 3h to the box
__global__ void k_fine_samples(const double2* coef, int n, int M, const double2* twM, double* fine, double xlo,
                               double xhi, double ylo, double yhi, int* flags) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= M) return;
  int nk = n / 2 + 1;
  const TrigStart st = trig_start_table(twM, M, warp, n, lane);
  TrigSums x = trig_sums(coef, n, st, lane, false);
  TrigSums y = trig_sums(coef + nk, n, st, lane, false);
  if (lane == 0) {
    fine[2 * warp] = x.f;
    fine[2 * warp + 1] = y.f;
    if (x.f < xlo || x.f > xhi || y.f < ylo || y.f > yhi) atomicOr(flags, FLAG_OUTSIDE);
  }
}

// The same fine samples for a power-of-two n from eight inverse FFTs of length n (block r):
// with C_k = cx_k + i cy_k over k in [-K, K] (c_{-k} = conj c_k) the curve is
// x + i y = sum_k C_k e^{i k alpha} + (nx + i ny) cos(n alpha / 2), and at
// alpha = 2 pi (8 q + r) / (8 n)
//   X(alpha_{8q+r}) = sum_k [C_k e^{2 pi i k r / (8n)}] e^{2 pi i k q / n}
//                     + (nx + i ny) cos(pi r / 8) (-1)^q,
// an inverse DFT of length n over q once the Nyquist term sits at index n/2. twn[m] =
// e^{2 pi i m / n} gives the FFT's staged twiddles, twM[m] = e^{2 pi i m / (8n)} the shifts.
// Shared memory: A[n] | B[n] | staged twiddles[n] (complex float64).
__global__ void k_fine_fft(const double2* coef, int n, int logn, const double2* twn, const double2* twM, double* fine,
                           double xlo, double xhi, double ylo, double yhi, int* flags) {
  extern __shared__ double2 fsm[];
  V2<double>* A = (V2<double>*)fsm;
  V2<double>* B = A + n;
  V2<double>* stw = B + n;
  const int r = blockIdx.x, M = 8 * n, nk = n / 2 + 1, K = (n - 1) / 2;
  const double2* cx = coef;
  const double2* cy = coef + nk;
  stage_twiddles_from_roots(twn, stw, n, logn);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    V2<double> v{0.0, 0.0};
    if (k == 0) {
      v = V2<double>{cx[0].x, cy[0].x};
    } else if (k <= K) {
      const double2 a = cx[k], b = cy[k];
      const double2 e = twM[((long)k * r) % M];
      const V2<double> ck{a.x - b.y, a.y + b.x};
      v = cmul(ck, V2<double>{e.x, e.y});
    } else if (k >= n - K) {
      const int kk = n - k;  // mode -kk
      const double2 a = cx[kk], b = cy[kk];
      const double2 e = twM[((long)kk * r) % M];
      const V2<double> ck{a.x + b.y, b.x - a.y};
      v = cmul(ck, V2<double>{e.x, -e.y});
    } else {
      // k = n/2 (even n): the Nyquist term
      const double cr = twM[((long)(n / 2) * r) % M].x;  // cos(pi r / 8)
      v = V2<double>{cx[n / 2].x * cr, cy[n / 2].x * cr};
    }
    A[k] = v;
  }
  __syncthreads();
  const V2<double>* X = fft_stockham<double>(A, B, 1, n, logn, stw, true);
  bool out = false;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const V2<double> z = X[q];
    const long s = 8L * q + r;
    fine[2 * s] = z.x;
    fine[2 * s + 1] = z.y;
    out |= z.x < xlo || z.x > xhi || z.y < ylo || z.y > yhi;
  }
  if (out) atomicOr(flags, FLAG_OUTSIDE);
}

kfbi_status geometry_setup_attributes() {
  KFBI_TRY(cudaFuncSetAttribute(k_fine_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FINE_FFT_SMEM));
  return KFBI_OK;
}

// per fine segment s -> s+1 (cyclic) and kind: number of grid lines crossed.
// kind 0 = horizontal lines y = y_l (coordinate y), kind 1 = vertical lines x = x_l.
__global__ void k_seg_count(const double* fine, int M, double xmin, double ymin, double h, int N,
                            int* seg_count) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * M) return;
  int kind = t / M, s = t - kind * M;
  int s1 = (s + 1 == M) ? 0 : s + 1;
  int ax = kind == 0 ? 1 : 0;
  double lo = kind == 0 ? ymin : xmin;
  int c0 = count_le(lo, h, N, fine[2 * s + ax]);
  int c1 = count_le(lo, h, N, fine[2 * s1 + ax]);
  seg_count[t] = abs(c0 - c1);
}

// exclusive scan of `len` ints by one block; out[len] = total
__global__ void k_scan(const int* in, int* out, int len) {
  __shared__ int part[1024];
  int tid = threadIdx.x, nt = blockDim.x;
  int per = (len + nt - 1) / nt;
  int b = tid * per, e = min(len, b + per);
  int s = 0;
  for (int i = b; i < e; ++i) s += in[i];
  part[tid] = s;
  __syncthreads();
  for (int o = 1; o < nt; o <<= 1) {
    int v = tid >= o ? part[tid - o] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  int run = tid == 0 ? 0 : part[tid - 1];
  for (int i = b; i < e; ++i) {
    out[i] = run;
    run += in[i];
  }
  if (tid == nt - 1) out[len] = part[nt - 1];
}

__global__ void k_emit_pairs(const double* fine, int M, double xmin, double ymin, double h, int N,
                             const int* seg_off, int* cr_kind, int* cr_line, int* cr_seg) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * M) return;
  int kind = t / M, s = t - kind * M;
  int s1 = (s + 1 == M) ? 0 : s + 1;
  int ax = kind == 0 ? 1 : 0;
  double lo = kind == 0 ? ymin : xmin;
  int c0 = count_le(lo, h, N, fine[2 * s + ax]);
  int c1 = count_le(lo, h, N, fine[2 * s1 + ax]);
  int a = min(c0, c1), b = max(c0, c1);
  int off = seg_off[t];
  for (int l = a; l < b; ++l) {
    int slot = off + (l - a);
    cr_kind[slot] = kind;
    cr_line[slot] = l;
    cr_seg[slot] = s;
  }
}

// Newton's method with a bisection safeguard on [alpha_s, alpha_s + 2 pi / M] for
// coordinate(alpha) = line; then the coordinate along the line and the first node past it.
__global__ void k_newton(const double2* coef, int n, int M, const double* fine, double xmin, double ymin,
                         double h, int N, int ncr, const int* cr_kind, const int* cr_line, const int* cr_seg,
                         int* cr_first, double* cr_alpha, double* cr_xi, int* flags) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= ncr) return;
  int nk = n / 2 + 1;
  int kind = cr_kind[warp], line = cr_line[warp], seg = cr_seg[warp];
  int ax = kind == 0 ? 1 : 0;
  const double2* cc = coef + ax * nk;      // coordinate compared with the line
  const double2* co = coef + (1 - ax) * nk;  // coordinate along the line
  double lv = grid_coord(kind == 0 ? ymin : xmin, h, line);
  double lo = (TWO_PI * (double)seg) / (double)M;
  double hi = lo + TWO_PI / (double)M;
  const int seg1 = seg + 1 == M ? 0 : seg + 1;
  const double flo = fine[2 * seg + ax], fhi = fine[2 * seg1 + ax];
  bool pos_lo = flo >= lv;
  // start from the secant through the bracketing fine samples (the midpoint if degenerate)
  double t = lo + (lv - flo) / (fhi - flo) * (hi - lo);
  if (!(t > lo && t < hi)) t = 0.5 * (lo + hi);
  double prev = 1.0;
  double fp_last = 0.0;  // derivative of the compared coordinate at the last iterate
  for (int it = 0; it < NEWTON_MAXIT; ++it) {
    TrigSums v = trig_warp(cc, n, t, lane, false);
    double f = v.f - lv, fp = v.f1;
    fp_last = fp;
    if (f == 0.0) break;  // exactly on the line: t is the root (no step, no bisection)
    bool same = (f >= 0.0) == pos_lo;
    if (same) lo = t; else hi = t;
    double tn = t - f / fp;
    // a Newton step within the tolerance ends the iteration before the bracket test (a
    // rounding-level step may land just outside a bracket whose other end is still far)
    if (isfinite(tn) && fabs(tn - t) <= NEWTON_TOL) {
      if (tn > lo && tn < hi) t = tn;
      break;
    }
    if (!isfinite(tn) || tn <= lo || tn >= hi) tn = 0.5 * (lo + hi);
    // converged, or in the rounding-noise regime (a step below 1e-12 that no longer shrinks)
    const double step = fabs(tn - t);
    bool done = step <= NEWTON_TOL || (step < 1e-12 && step >= 0.5 * prev);
    prev = step;
    t = tn;
    if (done) break;
  }
  TrigSums o = trig_warp(co, n, t, lane, false);
  if (lane == 0) {
    const double lo0 = kind == 0 ? xmin : ymin;
    double xi = o.f;
    int first = count_le(lo0, h, N, xi);
    // tie-break: a crossing on a grid node (within SNAP_TOL h) is placed on the node and on the
    // arm toward the outside, so that the node is in the closed interior. The outward normal
    // (y_a, -x_a) points to +x on a horizontal line when y_a > 0, to +y on a vertical line
    // when x_a < 0.
    int l = (int)rint((xi - lo0) / h - 0.5);
    l = l < 0 ? 0 : (l > N - 1 ? N - 1 : l);
    const double gc = grid_coord(lo0, h, l);
    if (fabs(xi - gc) <= SNAP_TOL * h) {
      xi = gc;
      const bool out_plus = kind == 0 ? fp_last > 0.0 : fp_last < 0.0;
      first = out_plus ? l + 1 : l;
    }
    cr_alpha[warp] = t;
    cr_xi[warp] = xi;
    cr_first[warp] = first;
    if (first <= 0 || first >= N) atomicOr(flags, FLAG_OUTSIDE);
  }
}

__global__ void k_arm_count(int ncr, int N, const int* cr_kind, const int* cr_line, const int* cr_first,
                            int* hcount, int* vcount, int* hid, int* vid) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncr) return;
  int line = cr_line[c], first = cr_first[c];
  if (first <= 0 || first >= N) return;
  if (cr_kind[c] == 0) {
    long a = (long)line * N + first;
    atomicAdd(&hcount[a], 1);
    atomicExch(&hid[a], c);
  } else {
    long a = (long)first * N + line;
    atomicAdd(&vcount[a], 1);
    atomicExch(&vid[a], c);
  }
}

// one warp per row: side = parity of horizontal-arm crossings left of the node
__global__ void k_classify(int N, const int* hcount, uint8_t* side, int* flags) {
  int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (j >= N) return;
  int per = N / 32 > 0 ? N / 32 : 1;
  int b = lane * per, e = min(N, b + per);
  const int* row = hcount + (long)j * N;
  int par = 0, bad = 0;
  for (int i = b; i < e; ++i) {
    int c = row[i];
    par ^= (c & 1);
    bad |= (c >= 3);
  }
  int incl = par;
  for (int o = 1; o < 32; o <<= 1) {
    int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl ^= v;
  }
  int run = incl ^ par;  // exclusive prefix parity
  for (int i = b; i < e; ++i) {
    run ^= (row[i] & 1);
    side[(long)j * N + i] = (uint8_t)run;
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flags, FLAG_UNDERRES);
}

__device__ __forceinline__ bool is_irregular(const uint8_t* side, int N, int i, int j) {
  uint8_t s = side[(long)j * N + i];
  if (i > 0 && side[(long)j * N + i - 1] != s) return true;
  if (i < N - 1 && side[(long)j * N + i + 1] != s) return true;
  if (j > 0 && side[(long)(j - 1) * N + i] != s) return true;
  if (j < N - 1 && side[(long)(j + 1) * N + i] != s) return true;
  return false;
}

// one warp per row: count irregular nodes; check vertical arms against the sides
__global__ void k_irr_count(int N, const uint8_t* side, const int* vcount, int* rowcnt, int* flags) {
  int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (j >= N) return;
  int cnt = 0, bad = 0;
  for (int i = lane; i < N; i += 32) {
    cnt += is_irregular(side, N, i, j) ? 1 : 0;
    if (j >= 1) {
      int vc = vcount[(long)j * N + i];
      bool diff = side[(long)j * N + i] != side[(long)(j - 1) * N + i];
      if (vc >= 3 || diff != ((vc & 1) == 1)) bad = 1;
    }
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) rowcnt[j] = cnt;
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flags, FLAG_UNDERRES);
}

__global__ void k_irr_emit(int N, double xmin, double ymin, double h, const uint8_t* side, const int* hcount,
                           const int* vcount, const int* hid, const int* vid, const double* cr_xi,
                           const int* row_ptr, IrrNode* irr) {
  int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (j >= N) return;
  int base = row_ptr[j];
  for (int i0 = 0; i0 < N; i0 += 32) {
    int i = i0 + lane;
    bool irr_here = i < N && is_irregular(side, N, i, j);
    unsigned mask = __ballot_sync(0xffffffffu, irr_here);
    if (irr_here) {
      int slot = base + __popc(mask & ((1u << lane) - 1u));
      IrrNode node;
      node.i = i;
      node.j = j;
      node.sign = side[(long)j * N + i] ? -1.0 : 1.0;
      for (int a = 0; a < 4; ++a) {
        node.target[a] = -1;
        node.d[a] = 0.0;
      }
      long r = (long)j * N;
      if (i >= 1 && hcount[r + i] == 1) {  // west arm (i-1,j)-(i,j)
        int c = hid[r + i];
        node.target[0] = c;
        node.d[0] = grid_coord(xmin, h, i - 1) - cr_xi[c];
      }
      if (i + 1 <= N - 1 && hcount[r + i + 1] == 1) {  // east arm (i,j)-(i+1,j)
        int c = hid[r + i + 1];
        node.target[1] = c;
        node.d[1] = grid_coord(xmin, h, i + 1) - cr_xi[c];
      }
      if (j >= 1 && vcount[r + i] == 1) {  // south arm (i,j-1)-(i,j)
        int c = vid[r + i];
        node.target[2] = c;
        node.d[2] = grid_coord(ymin, h, j - 1) - cr_xi[c];
      }
      if (j + 1 <= N - 1 && vcount[r + N + i] == 1) {  // north arm (i,j)-(i,j+1)
        int c = vid[r + N + i];
        node.target[3] = c;
        node.d[3] = grid_coord(ymin, h, j + 1) - cr_xi[c];
      }
      for (int a = 0; a < 4; ++a) node.df[a] = (float)node.d[a];
      node.signf = (float)node.sign;
      node.pad = 0;
      irr[slot] = node;
    }
    base += __popc(mask);
  }
}

// The per-arm correction map of the float32 applies whose column kernel forms the row
// transform itself: for irregular node t, 2 i + 1 (column factor of its sines), and for each
// crossed arm a, the code 4 t + a and (d, sign / h^2) filed under the crossing (at most two
// arms cut one crossing: the two ends of its grid segment)
__global__ void k_arm_map(int nirr, const IrrNode* irr, float inv_h2, int* rev, float2* coef, int* ci) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nirr) return;
  const IrrNode& q = irr[t];
  ci[t] = 2 * q.i + 1;
  const float sc = q.signf * inv_h2;
  for (int a = 0; a < 4; ++a) {
    const int cr = q.target[a];
    if (cr < 0) continue;
    const int code = 4 * t + a;
    const int k = atomicCAS(&rev[2 * cr], -1, code) == -1 ? 0 : 1;
    if (k == 1) rev[2 * cr + 1] = code;
    coef[2 * cr + k] = make_float2(q.df[a], sc);
  }
}

// geometry at every target (crossings, then nodes) and the inverse 3x3 jump matrix
// Also stores, per target, the twiddle starts of the per-apply density evaluation: lane l's
// e^{i k0_l alpha} (k0_l = 1 + l chunk, chunk = ceil(K / 32)), then e^{i alpha} and
// e^{i n alpha / 2}, in float64 and float32.
// Targets [t_begin, t_end) of the ncr + n (crossings, then nodes), one warp each.
__global__ void k_target_geo(const double2* coef, int n, int ncr, int t_begin, int t_end, const double* cr_alpha,
                             const double2* twn, TargetGeo* tg, TargetGeoF* tg_f, double2* tstart, float2* tstart_f) {
  int warp = t_begin + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  int lane = threadIdx.x & 31;
  if (warp >= t_end) return;
  int nk = n / 2 + 1;
  double a = warp < ncr ? cr_alpha[warp] : (TWO_PI * (double)(warp - ncr)) / (double)n;
  // crossings: sincos at alpha; nodes alpha_j = 2 pi j / n: the node twiddle table
  const TrigStart st = warp < ncr ? trig_start(n, a, lane) : trig_start_table(twn, n, warp - ncr, n, lane);
  TrigSums x = trig_sums(coef, n, st, lane, true);
  TrigSums y = trig_sums(coef + nk, n, st, lane, true);
  {
    long base = (long)warp * TSTART_STRIDE;
    tstart[base + lane] = st.e0;
    tstart_f[base + lane] = make_float2((float)st.e0.x, (float)st.e0.y);
    if (lane == 0) {
      tstart[base + 32] = st.s1;
      tstart_f[base + 32] = make_float2((float)st.s1.x, (float)st.s1.y);
      tstart[base + 33] = st.q;
      tstart_f[base + 33] = make_float2((float)st.q.x, (float)st.q.y);
    }
  }
  if (lane != 0) return;
  TargetGeo g;
  g.alpha = a;
  g.xa = x.f1;
  g.ya = y.f1;
  g.xaa = x.f2;
  g.yaa = y.f2;
  g.sa = sqrt(g.xa * g.xa + g.ya * g.ya);
  g.saa = (g.xa * g.xaa + g.ya * g.yaa) / g.sa;
  double A[9] = {g.xa * g.xa, g.ya * g.ya, 2.0 * g.xa * g.ya,
                 g.xa * g.ya, -g.xa * g.ya, g.ya * g.ya - g.xa * g.xa,
                 1.0, 1.0, 0.0};
  double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
  double c10 = A[2] * A[7] - A[1] * A[8], c11 = A[0] * A[8] - A[2] * A[6], c12 = A[1] * A[6] - A[0] * A[7];
  double c20 = A[1] * A[5] - A[2] * A[4], c21 = A[2] * A[3] - A[0] * A[5], c22 = A[0] * A[4] - A[1] * A[3];
  double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  double id = 1.0 / det;
  g.A3i[0] = c00 * id; g.A3i[1] = c10 * id; g.A3i[2] = c20 * id;
  g.A3i[3] = c01 * id; g.A3i[4] = c11 * id; g.A3i[5] = c21 * id;
  g.A3i[6] = c02 * id; g.A3i[7] = c12 * id; g.A3i[8] = c22 * id;
  tg[warp] = g;
  TargetGeoF f;
  f.alpha = (float)g.alpha;
  f.xa = (float)g.xa; f.ya = (float)g.ya; f.xaa = (float)g.xaa; f.yaa = (float)g.yaa;
  f.sa = (float)g.sa; f.saa = (float)g.saa;
  for (int q = 0; q < 9; ++q) f.A3i[q] = (float)g.A3i[q];
  tg_f[warp] = f;
}

// 6-point stencil per node: closest node, d1/d2, sides, scaled 6x6 LU -> inverse rows 0..2
__global__ void k_stencil(int n, const double* xy, double xmin, double ymin, double h, int N, const uint8_t* side,
                          const TargetGeo* tg_nodes, Stencil* st, int* probe_mark, int* flags) {
  // (the float32 copy is written by k_stencil_map once the probe ids are final)
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double px = xy[2 * p], py = xy[2 * p + 1];
  double x0 = grid_coord(xmin, h, 0), y0 = grid_coord(ymin, h, 0);
  int i0 = (int)floor(__dadd_rn(__ddiv_rn(__dsub_rn(px, x0), h), 0.5));
  int j0 = (int)floor(__dadd_rn(__ddiv_rn(__dsub_rn(py, y0), h), 0.5));
  int d1 = (i0 >= 0 && i0 < N && px > grid_coord(xmin, h, i0)) ? 1 : -1;
  int d2 = (j0 >= 0 && j0 < N && py > grid_coord(ymin, h, j0)) ? 1 : -1;
  const int rr[6] = {0, 1, 0, 0, -1, d1};
  const int ss[6] = {0, 0, 1, -1, 0, d2};
  Stencil S;
  double M[6][6];
  bool ok = true;
  for (int m = 0; m < 6; ++m) {
    int qi = i0 + rr[m], qj = j0 + ss[m];
    if (qi < 0 || qj < 0 || qi >= N || qj >= N) {
      ok = false;
      qi = 0;
      qj = 0;
    }
    S.q[m] = qj * N + qi;
    S.probe[m] = qj * N + qi;  // the flat grid index until the probes are numbered
    S.minus[m] = side[(long)qj * N + qi] == 0 ? 1 : 0;
    S.dx[m] = __dsub_rn(grid_coord(xmin, h, qi), px);
    S.dy[m] = __dsub_rn(grid_coord(ymin, h, qj), py);
    double a = S.dx[m] / h, b = S.dy[m] / h;
    M[m][0] = 1.0; M[m][1] = a; M[m][2] = b;
    M[m][3] = 0.5 * a * a; M[m][4] = a * b; M[m][5] = 0.5 * b * b;
  }
  if (!ok) atomicOr(flags, FLAG_OUTSIDE);
  // rows r of inv(M) solve M^T z = e_r; LU of M^T with partial pivoting
  double A[6][6];
  int piv[6];
  for (int r = 0; r < 6; ++r)
    for (int c = 0; c < 6; ++c) A[r][c] = M[c][r];
  for (int k = 0; k < 6; ++k) {
    int pr = k;
    double best = fabs(A[k][k]);
    for (int r = k + 1; r < 6; ++r)
      if (fabs(A[r][k]) > best) { best = fabs(A[r][k]); pr = r; }
    piv[k] = pr;
    if (pr != k)
      for (int c = 0; c < 6; ++c) { double t = A[k][c]; A[k][c] = A[pr][c]; A[pr][c] = t; }
    double d = A[k][k];
    for (int r = k + 1; r < 6; ++r) {
      double l = A[r][k] / d;
      A[r][k] = l;
      for (int c = k + 1; c < 6; ++c) A[r][c] -= l * A[k][c];
    }
  }
  for (int row = 0; row < 3; ++row) {
    double z[6] = {0, 0, 0, 0, 0, 0};
    z[row] = 1.0;
    for (int k = 0; k < 6; ++k) {
      int pr = piv[k];
      if (pr != k) { double t = z[k]; z[k] = z[pr]; z[pr] = t; }
    }
    for (int r = 1; r < 6; ++r)
      for (int c = 0; c < r; ++c) z[r] -= A[r][c] * z[c];
    for (int r = 5; r >= 0; --r) {
      for (int c = r + 1; c < 6; ++c) z[r] -= A[r][c] * z[c];
      z[r] /= A[r][r];
    }
    double scale = row == 0 ? 1.0 : 1.0 / h;
    for (int m = 0; m < 6; ++m) {
      double v = z[m] * scale;
      if (row == 0) S.r0[m] = v; else if (row == 1) S.r1[m] = v; else S.r2[m] = v;
    }
  }
  const TargetGeo& g = tg_nodes[p];
  S.nx = g.ya / g.sa;
  S.ny = -g.xa / g.sa;
  S.w = g.sa * TWO_PI / (double)n;
  st[p] = S;
  if (ok)
    for (int m = 0; m < 6; ++m) probe_mark[S.probe[m]] = 1;
}

__global__ void k_probe_count(int N, const int* probe_mark, int* cnt) {
  int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (j >= N) return;
  int c = 0;
  for (int i = lane; i < N; i += 32) c += probe_mark[(long)j * N + i] != 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) cnt[j] = c;
}

__global__ void k_probe_emit(int N, int* probe_mark, const int* prow_ptr, int* probe_i, int* probe_j) {
  int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (j >= N) return;
  int base = prow_ptr[j];
  for (int i0 = 0; i0 < N; i0 += 32) {
    int i = i0 + lane;
    bool on = i < N && probe_mark[(long)j * N + i] != 0;
    unsigned mask = __ballot_sync(0xffffffffu, on);
    if (on) {
      int slot = base + __popc(mask & ((1u << lane) - 1u));
      probe_i[slot] = i;
      probe_j[slot] = j;
      probe_mark[(long)j * N + i] = slot + 1;
    }
    base += __popc(mask);
  }
}

__global__ void k_stencil_map(int n, const int* probe_mark, Stencil* st, StencilF* stf) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  Stencil S = st[p];
  StencilF F;
  for (int m = 0; m < 6; ++m) {
    S.probe[m] = probe_mark[S.probe[m]] - 1;
    F.q[m] = S.q[m];
    F.probe[m] = S.probe[m];
    F.minus[m] = S.minus[m];
    F.dx[m] = (float)S.dx[m];
    F.dy[m] = (float)S.dy[m];
    F.r0[m] = (float)S.r0[m];
    F.r1[m] = (float)S.r1[m];
    F.r2[m] = (float)S.r2[m];
  }
  F.nx = (float)S.nx;
  F.w = (float)S.w;
  F.ny = (float)S.ny;
  st[p] = S;
  stf[p] = F;
}

// packed node data (x, y, y_a, -x_a) for the free-space box quadrature
__global__ void k_npack(int n, const double* xy, const TargetGeo* tg_nodes, double4_32a* np, float4* np_f) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double4_32a v;
  v.x = xy[2 * p];
  v.y = xy[2 * p + 1];
  v.z = tg_nodes[p].ya;
  v.w = -tg_nodes[p].xa;
  np[p] = v;
  np_f[p] = make_float4((float)v.x, (float)v.y, (float)v.z, (float)v.w);
}

// rows that hold at least one interpolation probe, in order; count in *cnt (one warp)
__global__ void k_prow_list(int N, const int* prow_cnt, int* list, int* cnt) {
  int lane = threadIdx.x & 31;
  int base = 0;
  for (int j0 = 0; j0 < N; j0 += 32) {
    int j = j0 + lane;
    bool on = j < N && prow_cnt[j] > 0;
    unsigned mask = __ballot_sync(0xffffffffu, on);
    if (on) list[base + __popc(mask & ((1u << lane) - 1u))] = j;
    base += __popc(mask);
  }
  if (lane == 0) *cnt = base;
}

// --------------------------------------------------------------------------- host driver
kfbi_status set_interface_impl(kfbi_ctx* c, int n, const double* xy_in) {
  cudaStream_t s = c->stream;
  const int N = c->N;
  const double h = c->h;
  const int M = SUBSAMPLES * n;
  const int nk = n / 2 + 1;
  c->have_iface = false;
  KFBI_CHECK(box_table_join(c, s));  // the previous table may still read the node data

  KFBI_TRY(cudaMemcpyAsync(c->xy, xy_in, sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice, s));
  KFBI_TRY(cudaMemsetAsync(c->flags, 0, sizeof(int), s));
  size_t NN = (size_t)N * N;
  KFBI_TRY(cudaMemsetAsync(c->hcount, 0, NN * sizeof(int), s));
  KFBI_TRY(cudaMemsetAsync(c->vcount, 0, NN * sizeof(int), s));
  KFBI_TRY(cudaMemsetAsync(c->probe_mark, 0, NN * sizeof(int), s));

  k_twiddles_n<<<cdiv(n, 256), 256, 0, s>>>(n, (double2*)c->twn, (float2*)c->twn_f);
  k_twiddles_M<<<cdiv(M, 256), 256, 0, s>>>(M, (double2*)c->twM);
  launched(c, 6);
  k_dft_real<<<cdiv((long)2 * nk * 32, 256), 256, 0, s>>>(c->xy, 2, 2, n, (const double2*)c->twn,
                                                          (double2*)c->icoef);
  double mg = BOX_MARGIN * h;
  const int logn = ilog2_exact(n);
  const size_t fsm = 3 * sizeof(double2) * (size_t)n;
  if (logn >= 4 && fsm <= FINE_FFT_SMEM && SUBSAMPLES == 8)
    k_fine_fft<<<SUBSAMPLES, 256, fsm, s>>>((const double2*)c->icoef, n, logn, (const double2*)c->twn,
                                            (const double2*)c->twM, c->fine, c->xmin + mg, c->xmax - mg,
                                            c->ymin + mg, c->ymax - mg, c->flags);
  else
    k_fine_samples<<<cdiv((long)M * 32, 256), 256, 0, s>>>((const double2*)c->icoef, n, M, (const double2*)c->twM,
                                                           c->fine, c->xmin + mg, c->xmax - mg, c->ymin + mg,
                                                           c->ymax - mg, c->flags);
  k_seg_count<<<cdiv(2 * M, 256), 256, 0, s>>>(c->fine, M, c->xmin, c->ymin, h, N, c->seg_count);
  k_scan<<<1, 1024, 0, s>>>(c->seg_count, c->seg_off, 2 * M);
  KFBI_TRY(cudaMemcpyAsync(&c->host_counts[0], c->seg_off + 2 * M, sizeof(int), cudaMemcpyDeviceToHost, s));
  KFBI_TRY(cudaMemcpyAsync(&c->host_counts[1], c->flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  KFBI_TRY(cudaStreamSynchronize(s));
  if (c->host_counts[1] & FLAG_OUTSIDE) return KFBI_ERR_OUTSIDE_BOX;
  int ncr = c->host_counts[0];
  KFBI_CHECK(ensure_cross_capacity(c, ncr));
  c->n_cross = ncr;

  // the nodes' geometry and packed node data depend on the interpolant only: formed now, so
  // that the free-space box table (aux stream, the longest part of an interface) is built
  // while the crossings, sides, irregular nodes and stencils are found on this stream
  c->boxK_ok = false;
  launched(c, 2);
  k_target_geo<<<cdiv((long)n * 32, 256), 256, 0, s>>>((const double2*)c->icoef, n, ncr, ncr, ncr + n, c->cr_alpha,
                                                       (const double2*)c->twn, c->tgeo, c->tgeo_f,
                                                       (double2*)c->tstart, (float2*)c->tstart_f);
  k_npack<<<cdiv(n, 128), 128, 0, s>>>(n, c->xy, c->tgeo + ncr, (double4_32a*)c->npack, (float4*)c->npack_f);
  if (c->boxK != nullptr) KFBI_CHECK(box_matrix_enqueue(c, n));

  launched(c, 4 + (ncr > 0 ? 2 : 0));
  k_emit_pairs<<<cdiv(2 * M, 256), 256, 0, s>>>(c->fine, M, c->xmin, c->ymin, h, N, c->seg_off, c->cr_kind,
                                                c->cr_line, c->cr_seg);
  if (ncr > 0) {
    k_newton<<<cdiv((long)ncr * 32, 256), 256, 0, s>>>((const double2*)c->icoef, n, M, c->fine, c->xmin, c->ymin,
                                                       h, N, ncr, c->cr_kind, c->cr_line, c->cr_seg, c->cr_first,
                                                       c->cr_alpha, c->cr_xi, c->flags);
    k_arm_count<<<cdiv(ncr, 256), 256, 0, s>>>(ncr, N, c->cr_kind, c->cr_line, c->cr_first, c->hcount,
                                              c->vcount, c->hid, c->vid);
  }
  int wblocks = cdiv((long)N * 32, 256);
  k_classify<<<wblocks, 256, 0, s>>>(N, c->hcount, c->side, c->flags);
  k_irr_count<<<wblocks, 256, 0, s>>>(N, c->side, c->vcount, c->rowcnt, c->flags);
  k_scan<<<1, 1024, 0, s>>>(c->rowcnt, c->row_ptr, N);
  KFBI_TRY(cudaMemcpyAsync(&c->host_counts[0], c->row_ptr + N, sizeof(int), cudaMemcpyDeviceToHost, s));
  KFBI_TRY(cudaMemcpyAsync(&c->host_counts[1], c->flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  KFBI_TRY(cudaStreamSynchronize(s));
  if (c->host_counts[1] & FLAG_OUTSIDE) return KFBI_ERR_OUTSIDE_BOX;
  if (c->host_counts[1] & FLAG_UNDERRES) return KFBI_ERR_UNDERRESOLVED;
  int nirr = c->host_counts[0];
  if (nirr > c->cap_irr) return KFBI_ERR_CAPACITY;
  c->n_irr = nirr;

  launched(c, 6 + (ncr > 0 ? 1 : 0));
  k_irr_emit<<<wblocks, 256, 0, s>>>(N, c->xmin, c->ymin, h, c->side, c->hcount, c->vcount, c->hid, c->vid,
                                     c->cr_xi, c->row_ptr, c->irr);
  if (ncr > 0) KFBI_TRY(cudaMemsetAsync(c->arm_rev, 0xFF, sizeof(int) * 2 * (size_t)ncr, s));
  if (nirr > 0) {
    KFBI_TRY(cudaMemsetAsync(c->arm_slot, 0, sizeof(float) * 4 * (size_t)nirr, s));
    k_arm_map<<<cdiv(nirr, 256), 256, 0, s>>>(nirr, c->irr, (float)(1.0 / (h * h)), c->arm_rev,
                                             (float2*)c->arm_coef, c->irr_ci);
    launched(c, 1);
  }
  if (ncr > 0)
    k_target_geo<<<cdiv((long)ncr * 32, 256), 256, 0, s>>>((const double2*)c->icoef, n, ncr, 0, ncr, c->cr_alpha,
                                                           (const double2*)c->twn, c->tgeo, c->tgeo_f,
                                                           (double2*)c->tstart, (float2*)c->tstart_f);
  k_stencil<<<cdiv(n, 128), 128, 0, s>>>(n, c->xy, c->xmin, c->ymin, h, N, c->side, c->tgeo + ncr, c->stencil,
                                         c->probe_mark, c->flags);
  k_probe_count<<<wblocks, 256, 0, s>>>(N, c->probe_mark, c->prow_cnt);
  k_scan<<<1, 1024, 0, s>>>(c->prow_cnt, c->prow_ptr, N);
  k_probe_emit<<<wblocks, 256, 0, s>>>(N, c->probe_mark, c->prow_ptr, c->probe_i, c->probe_j);
  k_stencil_map<<<cdiv(n, 128), 128, 0, s>>>(n, c->probe_mark, c->stencil, c->stencil_f);
  k_prow_list<<<1, 32, 0, s>>>(N, c->prow_cnt, c->prow_list, c->counts);
  launched(c, 1);
  KFBI_TRY(cudaGetLastError());
  KFBI_TRY(cudaMemcpyAsync(&c->host_counts[0], c->prow_ptr + N, sizeof(int), cudaMemcpyDeviceToHost, s));
  KFBI_TRY(cudaMemcpyAsync(&c->host_counts[1], c->flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  KFBI_TRY(cudaMemcpyAsync(&c->host_counts[2], c->counts, sizeof(int), cudaMemcpyDeviceToHost, s));
  KFBI_TRY(cudaStreamSynchronize(s));
  if (c->host_counts[1] & FLAG_OUTSIDE) return KFBI_ERR_OUTSIDE_BOX;
  if (c->host_counts[1] & FLAG_UNDERRES) return KFBI_ERR_UNDERRESOLVED;
  c->n_probe = c->host_counts[0];
  c->n_prow = c->host_counts[2];
  c->boxK_ok = c->boxK != nullptr;  // enqueued above
  if (c->n != n) c->layout_version += 1;
  if (c->n_cross > c->ncr_grid) {
    // the jump launches cover a quarter more crossings than this interface has, so that the
    // next interfaces of a moving curve reuse them
    c->ncr_grid = c->n_cross + c->n_cross / 4 + 64;
    c->layout_version += 1;
  }
  c->n = n;
  c->have_iface = true;
  c->iface_version += 1;
  return KFBI_OK;
}

}  // namespace kfbi
