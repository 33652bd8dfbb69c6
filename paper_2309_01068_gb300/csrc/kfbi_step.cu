// theta-L interface evolution with small-scale decomposition (Sec. 5) on the device.
//
// State: eta = theta - alpha at the nodes, L, Xbar, t and the Adams-Bashforth history
// (M, Q, L, N-hat of the previous level). One step: reconstruct the curve (spectral
// integration of X_a = (L/2pi)(cos theta, sin theta) with its mean removed), set the
// interface, solve the step's BIE, form the normal velocity U, then advance L and Xbar by
// AB2 and theta-hat by the integrating-factor propagator of Sec. 5.3. All interface
// transforms are direct DFTs with exact twiddle indexing (one warp per output).
#include <cmath>

#include "kfbi_internal.cuh"

namespace kfbi {
kfbi_status set_interface_impl(kfbi_ctx* c, int n, const double* xy);
kfbi_status solve_bie_impl(kfbi_ctx* c, int kind, const double* eps_v, const double* rhs, double tol, int max_iter,
                           int restart, double* x, kfbi_solve_info* info,
                           double* dnormal = nullptr);
}  // namespace kfbi

// scalar slots of the device state
enum : int {
  SC_L = 0, SC_XB0, SC_XB1, SC_T, SC_STEPS, SC_MPREV, SC_QPREV0, SC_QPREV1, SC_LPREV, SC_M, SC_Q0, SC_Q1,
  SC_LNEW, SC_LAM, SC_WS_NET, SC_WS_RATIO, SC_A0, SC_COUNT = 20
};

struct kfbi_thetal {
  kfbi_ctx* ctx = nullptr;
  int n = 0;
  int cap = 0;                // node capacity of the arrays (marker doubling grows n up to it)
  kfbi_thetal_params prm{};
  double* eta = nullptr;      // [n]
  double* xy = nullptr;       // [n][2]
  double* density = nullptr;  // [n]
  double* scal = nullptr;     // [SC_COUNT]
  double* tw = nullptr;       // [n] complex e^{2 pi i m / n}
  double* eta_h = nullptr;    // [(n/2+1)] complex
  double* N_h = nullptr;      // [(n/2+1)] complex
  double* Nprev_h = nullptr;  // [(n/2+1)] complex
  double* coef = nullptr;     // [2][(n/2+1)] complex scratch
  double* th_a = nullptr;     // [n]
  double* U = nullptr;        // [n]
  double* V = nullptr;        // [n]
  double* rhs = nullptr;      // [n]
  double* work = nullptr;     // [4n]
  double* epsv = nullptr;     // [n]
  double* dn = nullptr;       // [n]
  double* T = nullptr;        // [N][N] (Stefan)
  double* Tprev = nullptr;
  double* Tw = nullptr;       // [N][N] T1 of the current step
  double* Sg = nullptr;       // [N][N] grid single layer of the current step
  double* host_scal = nullptr;  // pinned [SC_COUNT]
  kfbi_mlp* ws = nullptr;     // learned warm start (not owned), or none
  double* guess = nullptr;    // [n] the network's density
  double* ws_norm = nullptr;  // [3] rms(rhs) of the features, residual norms of the two starts
};

namespace kfbi {

// c_k = (1/n) sum_j f_j e^{-2 pi i k j / n}, k = 0..n/2; nf functions with stride
__global__ void k_st_dft(const double* f, int stride, int nf, int n, const double2* tw, double2* coef) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  int nk = n / 2 + 1;
  if (warp >= nk * nf) return;
  int q = warp / nk, k = warp - q * nk;
  // twiddle index k j mod n advanced by k 32 mod n (no division in the loop); four
  // accumulator pairs shorten the float64 dependency chains
  int idx = (int)(((long)k * lane) % n);
  const int step = (int)(((long)k * 32) % n);
  double re[4] = {0.0, 0.0, 0.0, 0.0}, im[4] = {0.0, 0.0, 0.0, 0.0};
  int j = lane;
  for (; j + 96 < n; j += 128) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double v = f[(long)(j + 32 * c) * stride + q];
      const double2 w = tw[idx];
      idx += step;
      if (idx >= n) idx -= n;
      re[c] += v * w.x;
      im[c] -= v * w.y;
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (j < n) {
      const double v = f[(long)j * stride + q];
      const double2 w = tw[idx];
      idx += step;
      if (idx >= n) idx -= n;
      re[c] += v * w.x;
      im[c] -= v * w.y;
      j += 32;
    }
  }
  const double re_s = warp_sum((re[0] + re[1]) + (re[2] + re[3]));
  const double im_s = warp_sum((im[0] + im[1]) + (im[2] + im[3]));
  if (lane == 0) coef[q * nk + k] = make_double2(re_s / n, im_s / n);
}

// spectral multipliers applied to coefficient sets (k = 0..n/2):
//   MODE_D1: ik (Nyquist -> 0);  MODE_INT: 1/(ik) for 0 < k < n/2, 0 at k = 0 and Nyquist
enum : int { MODE_D1 = 1, MODE_INT = 2 };

// f_j = sum_k w_k Re(mult_k c_k e^{2 pi i k j / n}), w_0 = 1, w_k = 2, w_{n/2} = 1 (even n)
__global__ void k_st_idft(const double2* coef, int nf, int n, const double2* tw, int mode, double* out, int stride) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= n * nf) return;
  int q = warp / n, j = warp - q * n;
  int nk = n / 2 + 1;
  const double2* c = coef + q * nk;
  // twiddle index k j mod n advanced by 32 j mod n; alternate accumulators
  int idx = (int)(((long)lane * j) % n);
  const int step = (int)(((long)32 * j) % n);
  double acc0 = 0.0, acc1 = 0.0;
  int it = 0;
  for (int k = lane; k < nk; k += 32, ++it) {
    const int wi = idx;
    idx += step;
    if (idx >= n) idx -= n;
    double2 ck = c[k];
    bool nyq = (n % 2 == 0) && (k == n / 2);
    if (mode == MODE_D1) {
      if (nyq) continue;
      ck = make_double2(-(double)k * ck.y, (double)k * ck.x);
    } else if (mode == MODE_INT) {
      if (k == 0 || nyq) continue;
      ck = make_double2(ck.y / (double)k, -ck.x / (double)k);
    }
    const double2 w = tw[wi];
    double re = ck.x * w.x - ck.y * w.y;
    double wk = (k == 0 || nyq) ? 1.0 : 2.0;
    if (it & 1) acc1 += wk * re;
    else acc0 += wk * re;
  }
  double acc = warp_sum(acc0 + acc1);
  if (lane == 0) out[(long)j * stride + q] = acc;
}

// X_a = (L / 2 pi)(cos theta, sin theta), theta = alpha + eta
__global__ void k_st_xa(const double* eta, int n, const double* scal, double* xa) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double a = (TWO_PI * (double)j) / (double)n;
  double th = a + eta[j];
  double s, c;
  sincos(th, &s, &c);
  double f = scal[SC_L] / TWO_PI;
  xa[2 * j] = f * c;
  xa[2 * j + 1] = f * s;
}

// X-hat_k = X_a-hat_k / (ik) (k != 0, not Nyquist), X-hat_0 = Xbar
__global__ void k_st_recon_coef(double2* coef, int n, const double* scal) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  int nk = n / 2 + 1;
  if (t >= 2 * nk) return;
  int q = t / nk, k = t - q * nk;
  double2 c = coef[t];
  if (k == 0) c = make_double2(scal[q == 0 ? SC_XB0 : SC_XB1], 0.0);
  else if (n % 2 == 0 && k == n / 2) c = make_double2(0.0, 0.0);
  else c = make_double2(c.y / (double)k, -c.x / (double)k);
  coef[t] = c;
}

__global__ void k_st_theta_a(const double* eta_a, int n, double* th_a) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  th_a[j] = 1.0 + eta_a[j];
}

// Hele-Shaw right-hand side -sigma kappa + J ln|X| (Sec. 3.1), kappa = (2 pi / L) theta_a
// rescaled frame (Sec. 6.1.4): surface tension sigma / R with R = e^{tb}, tb = the scaled time
__global__ void k_st_hs_rhs(const double* xy, const double* th_a, int n, const double* scal, double sigma, double J,
                            int rescale, double* rhs) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double x = xy[2 * j], y = xy[2 * j + 1];
  double curv = (TWO_PI / scal[SC_L]) * th_a[j];
  const double sig = rescale ? sigma * exp(-scal[SC_T]) : sigma;
  rhs[j] = -sig * curv + J * 0.5 * log(x * x + y * y);
}

// U = J x.n / |x|^2 - dn,  n = (sin theta, -cos theta); rescaled frame: (A0 / pi) U - x.n
__global__ void k_st_hs_velocity(const double* xy, const double* eta, const double* dn, int n, double J, int rescale,
                                 const double* scal, double* U) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double a = (TWO_PI * (double)j) / (double)n;
  double th = a + eta[j];
  double s, c;
  sincos(th, &s, &c);
  double x = xy[2 * j], y = xy[2 * j + 1];
  const double xn = x * s - y * c;
  const double u = J * xn / (x * x + y * y) - dn[j];
  U[j] = rescale ? (scal[SC_A0] / PI) * u - xn : u;
}

// area of the curve through the nodes, (1/2) int (x y_a - y x_a) da with X_a = (L / 2 pi)(cos, sin)
// theta (one block); stored as the scaled frame's A0 on the first step
__global__ void k_st_area0(const double* xy, const double* eta, int n, double* scal) {
  __shared__ double sh[32];
  if (scal[SC_STEPS] != 0.0) return;
  double a = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double th = (TWO_PI * (double)j) / (double)n + eta[j];
    double s, c;
    sincos(th, &s, &c);
    a += xy[2 * j] * s - xy[2 * j + 1] * c;
  }
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    scal[SC_A0] = 0.5 * (scal[SC_L] / TWO_PI) * t * (TWO_PI / (double)n);
  }
}

// ---- marker doubling (Sec. 6.1.4): values at alpha = 2 pi j / (2n) of the trigonometric
// interpolant with coefficients c_k (k <= n/2, normalised, the Nyquist term a cosine), one warp
// per output point
__global__ void k_st_upsample(const double2* coef, int n, const double2* tw2, double* out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int m = 2 * n;
  if (warp >= m) return;
  const int j = warp;
  const int K = (n - 1) / 2;
  double acc = 0.0;
  for (int k = 1 + lane; k <= K; k += 32) {
    const double2 e = tw2[(int)(((long)k * j) % m)];  // e^{2 pi i k j / (2n)}
    acc += 2.0 * (coef[k].x * e.x - coef[k].y * e.y);
  }
  acc = warp_sum(acc);
  if (lane == 0) {
    double v = coef[0].x + acc;
    if ((n & 1) == 0) {
      const double2 e = tw2[(int)(((long)(n / 2) * j) % m)];
      v += coef[n / 2].x * e.x;  // c cos(n alpha / 2)
    }
    out[j] = v;
  }
}

// the Adams-Bashforth history N-hat (normalised half spectrum, k <= n/2) of the same function on
// 2n points: k < n/2 kept, the Nyquist cosine split (half at k = n/2), zero above
__global__ void k_st_pad_history(double2* nh, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > n) return;
  if (k == n / 2 && (n & 1) == 0) nh[k] = make_double2(0.5 * nh[k].x, 0.5 * nh[k].y);
  else if (k > n / 2) nh[k] = make_double2(0.0, 0.0);
}

// Stefan: eps_C at the nodes, rhs = -eps_C kappa - T1 (Sec. 3.2), eps_V array
__global__ void k_st_stefan_rhs(const double* eta, const double* th_a, const double* T1n, int n, const double* scal,
                                double eps_c, double aniso, int fold, double eps_v, double* rhs, double* epsv,
                                double* ratio) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double a = (TWO_PI * (double)j) / (double)n;
  double th = a + eta[j];
  double ec = eps_c * (1.0 - aniso * cos((double)fold * (th - 0.5 * PI)));
  double curv = (TWO_PI / scal[SC_L]) * th_a[j];
  rhs[j] = -ec * curv - T1n[j];
  epsv[j] = eps_v;
  // lambda_1 = max |eps_C / eps_V| (case I) or lambda_2 = max |2 eps_C| (case II, eps_V = 0)
  ratio[j] = eps_v > 0.0 ? fabs(ec / eps_v) : fabs(2.0 * ec);
}

// T = 0 in Omega+ (the seed at the melt temperature), St outside
__global__ void k_st_T0(const uint8_t* side, long NN, double St, double* T, double* Tprev) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NN) return;
  double v = side[i] ? 0.0 : St;
  T[i] = v;
  Tprev[i] = v;
}

// rhs of the BDF2 step (T^{n-1} - 4 T^n) / (2 tau), as a product with 1 / (2 tau) (a float64
// division per node made this pass bound by the float64 rate)
__global__ void k_st_bdf_rhs(const double* T, const double* Tprev, long NN, double inv_2dt, double* out) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NN) return;
  out[i] = (Tprev[i] - 4.0 * T[i]) * inv_2dt;
}

// T^{n+1} = T1 - (S psi)_h; history shift
__global__ void k_st_T_update(const double* T1, const double* Sg, long NN, double* T, double* Tprev) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NN) return;
  Tprev[i] = T[i];
  T[i] = T1[i] - Sg[i];
}

__global__ void k_st_copy(const double* a, double* b, int n) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) b[j] = a[j];
}

__global__ void k_st_mul(const double* a, const double* b, int n, double* out) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = a[j] * b[j];
}

// V = (alpha/2pi) M - int_0^alpha theta_a U with the cumulative integral of the
// interpolant: c0 alpha + P(alpha) - P(0), P the periodic antiderivative. With
// M = 2 pi c0 this is V = P(0) - P(alpha). Also forms the one-block reductions M, Q and
// lambda_1 = max |eps_C / eps_V| (Stefan).
__global__ void k_st_tangential(const double* P, const double2* thU_coef, const double* U, const double* eta, int n,
                                double* V, double* scal, const double* ratio) {
  __shared__ double sh[3][32];
  double p0 = P[0];
  double q0 = 0.0, q1 = 0.0, mx = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double v = p0 - P[j];
    V[j] = v;
    double a = (TWO_PI * (double)j) / (double)n;
    double th = a + eta[j];
    double s, c;
    sincos(th, &s, &c);
    q0 += U[j] * s + v * c;
    q1 += -U[j] * c + v * s;
    if (ratio) mx = fmax(mx, ratio[j]);
  }
  q0 = warp_sum(q0);
  q1 = warp_sum(q1);
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][wid] = q0;
    sh[1][wid] = q1;
    sh[2][wid] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0, a1 = 0, m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a0 += sh[0][w];
      a1 += sh[1][w];
      m = fmax(m, sh[2][w]);
    }
    scal[SC_M] = TWO_PI * thU_coef[0].x;
    scal[SC_Q0] = a0 / n;
    scal[SC_Q1] = a1 / n;
    scal[SC_LAM] = m;
  }
}

// rhs of theta_t: (2 pi / L)(theta_a V - U_a)
__global__ void k_st_theta_rhs(const double* th_a, const double* V, const double* U_a, int n, const double* scal,
                               double* out) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  out[j] = (TWO_PI / scal[SC_L]) * (th_a[j] * V[j] - U_a[j]);
}

// AB2 for L and Xbar (first step: history = current level)
__global__ void k_st_scalars(double* scal, double dt) {
  if (threadIdx.x != 0) return;
  bool first = scal[SC_STEPS] == 0.0;
  double M = scal[SC_M], Mp = first ? M : scal[SC_MPREV];
  double Q0 = scal[SC_Q0], Q1 = scal[SC_Q1];
  double Q0p = first ? Q0 : scal[SC_QPREV0], Q1p = first ? Q1 : scal[SC_QPREV1];
  double L = scal[SC_L];
  scal[SC_LNEW] = L + 0.5 * dt * (3.0 * M - Mp);
  scal[SC_XB0] += 0.5 * dt * (3.0 * Q0 - Q0p);
  scal[SC_XB1] += 0.5 * dt * (3.0 * Q1 - Q1p);
  if (first) scal[SC_LPREV] = L;
}

// stiff symbol -lam (2 pi / L)^p |k|^p
__device__ __forceinline__ double stiff(double lam, double L, int p, double k) {
  double a = TWO_PI / L * fabs(k);
  return p == 3 ? -lam * a * a * a : -lam * a * a;
}

// N-hat = FFT(rhs) - s(L^n) eta-hat; eta-hat^{n+1} = e1 eta-hat + dt/2 (3 e1 N-hat - e2 N-hat^{n-1});
// history shift (Sec. 5.3). explicit_ != 0: no stiff part (s = 0, e1 = e2 = 1), the
// Adams-Bashforth comparison scheme of Sec. 6.2.2.
__global__ void k_st_propagate(double2* eta_h, const double2* rhs_h, double2* Nprev, int n, double* scal, double dt,
                               int p, double lam_fixed, int explicit_, int rescale) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  int nk = n / 2 + 1;
  if (k >= nk) return;
  bool first = scal[SC_STEPS] == 0.0;
  double lam = explicit_ ? 0.0 : (lam_fixed > 0.0 ? lam_fixed : scal[SC_LAM]);
  // rescaled Hele-Shaw frame: the stiff part of (A0 / pi) U with surface tension sigma e^{-tb}
  if (rescale && !explicit_) lam = (scal[SC_A0] / PI) * lam_fixed * exp(-scal[SC_T]);
  double L = scal[SC_L], Ln = scal[SC_LNEW], Lp = scal[SC_LPREV];
  double sn = stiff(lam, L, p, k), snew = stiff(lam, Ln, p, k), sp = stiff(lam, Lp, p, k);
  double e1 = exp(0.5 * dt * (sn + snew));
  double e2 = exp(dt * (0.5 * sp + sn + 0.5 * snew));
  double2 eh = eta_h[k];
  double2 Nh = make_double2(rhs_h[k].x - sn * eh.x, rhs_h[k].y - sn * eh.y);
  double2 Np = first ? Nh : Nprev[k];
  eta_h[k] = make_double2(e1 * eh.x + 0.5 * dt * (3.0 * e1 * Nh.x - e2 * Np.x),
                          e1 * eh.y + 0.5 * dt * (3.0 * e1 * Nh.y - e2 * Np.y));
  Nprev[k] = Nh;
}

__global__ void k_st_finish(double* scal, double dt) {
  if (threadIdx.x != 0) return;
  scal[SC_MPREV] = scal[SC_M];
  scal[SC_QPREV0] = scal[SC_Q0];
  scal[SC_QPREV1] = scal[SC_Q1];
  scal[SC_LPREV] = scal[SC_L];
  scal[SC_L] = scal[SC_LNEW];
  scal[SC_T] += dt;
  scal[SC_STEPS] += 1.0;
}

__global__ void k_twiddles_n_step(int n, double2* tw) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  double s, c;
  sincospi(2.0 * (double)m / (double)n, &s, &c);
  tw[m] = make_double2(c, s);
}

static int wb(long warps) { return cdiv(warps * 32, 256); }

// Learned warm start, the choice between two initial densities: residual norms
// ||b - A g|| (network g) and ||b - A x|| (previous step x), one block; the start with the smaller
// residual is kept in x. Counts the network's wins in scal[SC_WS_NET] and stores the ratio of
// the two norms in scal[SC_WS_RATIO].
__global__ void k_ws_choose(int n, const double* b, const double* Ag, const double* Ax, const double* g, double* x,
                            double* scal) {
  __shared__ double sh[2][32];
  __shared__ int take;
  double rg = 0.0, rx = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double a = b[j] - Ag[j], c = b[j] - Ax[j];
    rg += a * a;
    rx += c * c;
  }
  rg = warp_sum(rg);
  rx = warp_sum(rx);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][wid] = rg;
    sh[1][wid] = rx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tg = 0.0, tx = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      tg += sh[0][w];
      tx += sh[1][w];
    }
    take = tg < tx ? 1 : 0;
    scal[SC_WS_NET] += (double)take;
    scal[SC_WS_RATIO] = tx > 0.0 ? sqrt(tg / tx) : 0.0;
  }
  __syncthreads();
  if (take)
    for (int j = threadIdx.x; j < n; j += blockDim.x) x[j] = g[j];
}

// training pair of the last solved system: target = density / rms(rhs)
__global__ void k_ws_target(int n, const double* density, const double* scale, float* target) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) target[j] = (float)(density[j] / *scale);
}

// the two starts of the step's solve, before GMRES (only with a network attached)
static kfbi_status warm_start_choose(kfbi_ctx* c, kfbi_thetal* st, int kind, const double* ev) {
  const int n = st->n;
  cudaStream_t s = c->stream;
  KFBI_CHECK(kfbi_warmstart_predict(c, st->ws, st->rhs, st->guess));
  const int layer = kind == KFBI_BIE_STEFAN_SL ? KFBI_SINGLE : KFBI_DOUBLE;
  KFBI_CHECK(apply_enqueue(c, layer, false, st->guess, st->work, nullptr, nullptr, kind, ev, nullptr));
  KFBI_CHECK(apply_enqueue(c, layer, false, st->density, st->work + n, nullptr, nullptr, kind, ev, nullptr));
  k_ws_choose<<<1, 1024, 0, s>>>(n, st->rhs, st->work, st->work + n, st->guess, st->density, st->scal);
  launched(c, 1);
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

// doubles the markers (eta, density, N-hat history; twiddles of the new count) while
// L / n > refine_ratio h and the capacity allows (Sec. 6.1.4)
static kfbi_status refine_markers(kfbi_ctx* c, kfbi_thetal* st) {
  cudaStream_t s = c->stream;
  while (true) {
    KFBI_TRY(cudaMemcpyAsync(st->host_scal, st->scal, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
    KFBI_TRY(cudaStreamSynchronize(s));
    const int n = st->n;
    if (!(st->host_scal[SC_L] / n > st->prm.refine_ratio * c->h) || 2 * n > st->cap) return KFBI_OK;
    const int nk = n / 2 + 1, m = 2 * n;
    double2* coef = (double2*)st->coef;
    // twiddles of 2n points into the work buffer, then eta and the density through the interpolant
    k_twiddles_n_step<<<cdiv(m, 256), 256, 0, s>>>(m, (double2*)st->work);
    k_st_dft<<<wb(nk), 256, 0, s>>>(st->eta, 1, 1, n, (const double2*)st->tw, coef);
    k_st_upsample<<<wb(m), 256, 0, s>>>(coef, n, (const double2*)st->work, st->V);
    k_st_copy<<<cdiv(m, 256), 256, 0, s>>>(st->V, st->eta, m);
    k_st_dft<<<wb(nk), 256, 0, s>>>(st->density, 1, 1, n, (const double2*)st->tw, coef);
    k_st_upsample<<<wb(m), 256, 0, s>>>(coef, n, (const double2*)st->work, st->V);
    k_st_copy<<<cdiv(m, 256), 256, 0, s>>>(st->V, st->density, m);
    k_st_pad_history<<<cdiv(n + 1, 256), 256, 0, s>>>((double2*)st->Nprev_h, n);
    k_st_copy<<<cdiv(2 * m, 256), 256, 0, s>>>(st->work, st->tw, 2 * m);
    launched(c, 9);
    KFBI_TRY(cudaGetLastError());
    st->n = m;
  }
}

kfbi_status thetal_step_impl(kfbi_ctx* c, kfbi_thetal* st, double dt, kfbi_solve_info* info) {
  cudaStream_t s = c->stream;
  if (st->prm.refine_ratio > 0.0) KFBI_CHECK(refine_markers(c, st));
  const int n = st->n;
  const int nk = n / 2 + 1;
  const double2* tw = (const double2*)st->tw;
  double2* coef = (double2*)st->coef;
  const kfbi_thetal_params& P = st->prm;
  const int tb = cdiv(n, 256);
  launched(c, 22);
  // 1. reconstruct the curve from (eta, L, Xbar)
  k_st_xa<<<tb, 256, 0, s>>>(st->eta, n, st->scal, st->work);
  k_st_dft<<<wb(2L * nk), 256, 0, s>>>(st->work, 2, 2, n, tw, coef);
  k_st_recon_coef<<<cdiv(2 * nk, 256), 256, 0, s>>>(coef, n, st->scal);
  k_st_idft<<<wb(2L * n), 256, 0, s>>>(coef, 2, n, tw, 0, st->xy, 2);
  KFBI_TRY(cudaGetLastError());
  // 2. interface geometry
  KFBI_CHECK(set_interface_impl(c, n, st->xy));
  // 3. theta_a = 1 + eta_a, eta-hat
  k_st_dft<<<wb(nk), 256, 0, s>>>(st->eta, 1, 1, n, tw, (double2*)st->eta_h);
  k_st_idft<<<wb(n), 256, 0, s>>>((const double2*)st->eta_h, 1, n, tw, MODE_D1, st->work, 1);
  k_st_theta_a<<<tb, 256, 0, s>>>(st->work, n, st->th_a);
  kfbi_solve_info si{};
  kfbi_status sst;
  const double* ratio = nullptr;
  if (P.kind == KFBI_STEP_HELE_SHAW) {
    launched(c, 2);
    if (P.rescale) k_st_area0<<<1, 1024, 0, s>>>(st->xy, st->eta, n, st->scal);
    k_st_hs_rhs<<<tb, 256, 0, s>>>(st->xy, st->th_a, n, st->scal, P.sigma, P.J, P.rescale, st->rhs);
    // mixed precision: the refinement's last float64 apply, at the returned density, also
    // gives the normal derivative of its double layer; float64: one more apply
    const bool dn_from_solve = c->precision == KFBI_MIXED;
    if (st->ws != nullptr) KFBI_CHECK(warm_start_choose(c, st, KFBI_BIE_HS_EXTERIOR_MDL, nullptr));
    sst = solve_bie_impl(c, KFBI_BIE_HS_EXTERIOR_MDL, nullptr, st->rhs, P.tol, P.max_iter, P.restart, st->density,
                         &si, dn_from_solve ? st->dn : nullptr);
    if (sst != KFBI_OK && sst != KFBI_ERR_NOT_CONVERGED) return sst;
    if (!dn_from_solve)
      KFBI_CHECK(apply_enqueue(c, KFBI_DOUBLE, false, st->density, st->V, st->dn, nullptr, -1, nullptr, nullptr));
    k_st_hs_velocity<<<tb, 256, 0, s>>>(st->xy, st->eta, st->dn, n, P.J, P.rescale, st->scal, st->U);
  } else {
    const int N = c->N;
    const long NN = (long)N * N;
    const int gb = cdiv(NN, 256);
    double steps = 0.0;
    KFBI_TRY(cudaMemcpyAsync(&steps, st->scal + SC_STEPS, sizeof(double), cudaMemcpyDeviceToHost, s));
    KFBI_TRY(cudaStreamSynchronize(s));
    if (steps == 0.0) k_st_T0<<<gb, 256, 0, s>>>(c->side, NN, P.St, st->T, st->Tprev);
    launched(c, (steps == 0.0) + 3);
    k_st_bdf_rhs<<<gb, 256, 0, s>>>(st->T, st->Tprev, NN, 1.0 / (2.0 * dt), st->Tw);
    // T1: in place by the float64 solve (T1 in Tw, the grid single layer later in Sg), or by
    // the mixed-precision solve, which keeps its right-hand side (T1 in Sg, the single layer
    // later in Tw)
    const bool ir = c->precision == KFBI_MIXED && c->grid_ir > 0;
    double* T1 = ir ? st->Sg : st->Tw;
    double* S2 = ir ? st->Tw : st->Sg;
    if (ir)
      KFBI_CHECK(grid_solve_mixed_enqueue(c, st->Tw, T1, c->grid_ir));
    else
      KFBI_CHECK(grid_solve_enqueue(c, st->Tw, T1));
    KFBI_CHECK(interp_grid_enqueue(c, T1, st->dn));  // T1 at the nodes
    k_st_stefan_rhs<<<tb, 256, 0, s>>>(st->eta, st->th_a, st->dn, n, st->scal, P.eps_c, P.eps_aniso, P.fold, P.eps_v,
                                       st->rhs, st->epsv, st->work + 2 * n);
    ratio = st->work + 2 * n;
    if (st->ws != nullptr) {
      // the network's start is compared on the equation's float64 operator; the ratio buffer
      // (work + 2n) is not touched by the two applies (work, work + n)
      KFBI_CHECK(warm_start_choose(c, st, KFBI_BIE_STEFAN_SL, st->epsv));
    }
    sst = solve_bie_impl(c, KFBI_BIE_STEFAN_SL, st->epsv, st->rhs, P.tol, P.max_iter, P.restart, st->density, &si);
    if (sst != KFBI_OK && sst != KFBI_ERR_NOT_CONVERGED) return sst;
    // T2 = -(S psi)_h from the apply's grid output; T^{n+1} = T1 + T2
    // (mixed: the grid solve of the single layer by the same mixed-precision box solve, with
    // its corrected right-hand side from the float64 jumps)
    if (ir && c->boxbc != KFBI_BOX_FREESPACE_DL)  // (box data: the float64 apply)
      KFBI_CHECK(apply_grid_mixed_enqueue(c, KFBI_SINGLE, st->density, S2, c->grid_ir));
    else
      KFBI_CHECK(apply_enqueue(c, KFBI_SINGLE, false, st->density, st->V, nullptr, S2, -1, nullptr, nullptr));
    k_st_T_update<<<gb, 256, 0, s>>>(T1, S2, NN, st->T, st->Tprev);
    k_st_copy<<<tb, 256, 0, s>>>(st->density, st->U, n);
  }
  KFBI_TRY(cudaGetLastError());
  // 4. tangential velocity, M, Q
  k_st_mul<<<tb, 256, 0, s>>>(st->th_a, st->U, n, st->work);               // theta_a U
  k_st_dft<<<wb(nk), 256, 0, s>>>(st->work, 1, 1, n, tw, coef);
  k_st_idft<<<wb(n), 256, 0, s>>>(coef, 1, n, tw, MODE_INT, st->work + n, 1);  // periodic antiderivative
  k_st_tangential<<<1, 1024, 0, s>>>(st->work + n, coef, st->U, st->eta, n, st->V, st->scal, ratio);
  // 5. U_a and the rhs of theta_t
  k_st_dft<<<wb(nk), 256, 0, s>>>(st->U, 1, 1, n, tw, coef + nk);
  k_st_idft<<<wb(n), 256, 0, s>>>(coef + nk, 1, n, tw, MODE_D1, st->work, 1);  // U_a
  k_st_theta_rhs<<<tb, 256, 0, s>>>(st->th_a, st->V, st->work, n, st->scal, st->work + n);
  k_st_dft<<<wb(nk), 256, 0, s>>>(st->work + n, 1, 1, n, tw, coef);            // rhs-hat
  // 6. AB2 scalars, propagator, history
  k_st_scalars<<<1, 32, 0, s>>>(st->scal, dt);
  const int expl = P.scheme == KFBI_SCHEME_EXPLICIT ? 1 : 0;
  if (P.kind == KFBI_STEP_HELE_SHAW)
    k_st_propagate<<<cdiv(nk, 256), 256, 0, s>>>((double2*)st->eta_h, coef, (double2*)st->Nprev_h, n, st->scal, dt, 3,
                                                 P.sigma, expl, P.rescale);
  else  // Stefan case I (second order) or II (eps_V = 0, third order); lambda from k_st_tangential
    k_st_propagate<<<cdiv(nk, 256), 256, 0, s>>>((double2*)st->eta_h, coef, (double2*)st->Nprev_h, n, st->scal, dt,
                                                 P.eps_v > 0.0 ? 2 : 3, -1.0, expl, 0);
  k_st_idft<<<wb(n), 256, 0, s>>>((const double2*)st->eta_h, 1, n, tw, 0, st->eta, 1);
  k_st_finish<<<1, 32, 0, s>>>(st->scal, dt);
  KFBI_TRY(cudaGetLastError());
  KFBI_TRY(cudaStreamSynchronize(s));
  if (info) *info = si;
  return sst;
}

}  // namespace kfbi

// --------------------------------------------------------------------------- C ABI
using namespace kfbi;

static void thetal_free(kfbi_thetal* st) {
  void* ptrs[] = {st->eta, st->xy, st->density, st->scal, st->tw, st->eta_h, st->N_h, st->Nprev_h, st->coef,
                  st->th_a, st->U, st->V, st->rhs, st->work, st->epsv, st->dn, st->T, st->Tprev, st->Tw, st->Sg,
                  st->guess, st->ws_norm};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (st->host_scal) cudaFreeHost(st->host_scal);
}

template <typename P>
static kfbi_status talloc(P** p, size_t count) {
  KFBI_TRY(cudaMalloc((void**)p, sizeof(P) * (count > 0 ? count : 1)));
  KFBI_TRY(cudaMemset(*p, 0, sizeof(P) * (count > 0 ? count : 1)));
  return KFBI_OK;
}

static kfbi_status thetal_create_impl(kfbi_ctx* c, int n, const double* eta, double L, const double* xbar,
                                      const kfbi_thetal_params* prm, kfbi_thetal* st) {
  st->ctx = c;
  st->n = n;
  st->prm = *prm;
  // arrays sized for the context's node capacity when markers may be doubled
  st->cap = prm->refine_ratio > 0.0 ? c->max_nodes : n;
  const int cap = st->cap;
  const int nk = cap / 2 + 1;
  KFBI_CHECK(talloc(&st->eta, cap));
  KFBI_CHECK(talloc(&st->xy, 2 * (size_t)cap));
  KFBI_CHECK(talloc(&st->density, cap));
  KFBI_CHECK(talloc(&st->scal, SC_COUNT));
  KFBI_CHECK(talloc(&st->tw, 2 * (size_t)cap));
  KFBI_CHECK(talloc(&st->eta_h, 2 * (size_t)nk));
  KFBI_CHECK(talloc(&st->N_h, 2 * (size_t)nk));
  KFBI_CHECK(talloc(&st->Nprev_h, 2 * (size_t)nk));
  KFBI_CHECK(talloc(&st->coef, 4 * (size_t)nk));
  KFBI_CHECK(talloc(&st->th_a, cap));
  KFBI_CHECK(talloc(&st->U, cap));
  KFBI_CHECK(talloc(&st->V, cap));
  KFBI_CHECK(talloc(&st->rhs, cap));
  KFBI_CHECK(talloc(&st->work, 4 * (size_t)cap));
  KFBI_CHECK(talloc(&st->epsv, cap));
  KFBI_CHECK(talloc(&st->dn, cap));
  KFBI_CHECK(talloc(&st->guess, cap));
  KFBI_CHECK(talloc(&st->ws_norm, 3));
  if (prm->kind == KFBI_STEP_STEFAN) {
    size_t NN = (size_t)c->N * c->N;
    KFBI_CHECK(talloc(&st->T, NN));
    KFBI_CHECK(talloc(&st->Tprev, NN));
    KFBI_CHECK(talloc(&st->Tw, NN));
    KFBI_CHECK(talloc(&st->Sg, NN));
  }
  KFBI_TRY(cudaMallocHost((void**)&st->host_scal, SC_COUNT * sizeof(double)));
  for (int i = 0; i < SC_COUNT; ++i) st->host_scal[i] = 0.0;
  st->host_scal[SC_L] = L;
  st->host_scal[SC_XB0] = xbar[0];
  st->host_scal[SC_XB1] = xbar[1];
  KFBI_TRY(stream_enter(c));
  KFBI_TRY(cudaMemcpyAsync(st->scal, st->host_scal, SC_COUNT * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  KFBI_TRY(cudaMemcpyAsync(st->eta, eta, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  k_twiddles_n_step<<<cdiv(n, 256), 256, 0, c->stream>>>(n, (double2*)st->tw);
  KFBI_TRY(cudaGetLastError());
  KFBI_TRY(cudaStreamSynchronize(c->stream));
  KFBI_TRY(stream_exit(c));
  return KFBI_OK;
}

extern "C" {

kfbi_status kfbi_thetal_create(kfbi_ctx* c, int n, const double* eta, double L, const double* xbar,
                               const kfbi_thetal_params* prm, kfbi_thetal** out) {
  if (c == nullptr || eta == nullptr || xbar == nullptr || prm == nullptr || out == nullptr) return KFBI_ERR_ARG;
  *out = nullptr;
  if (n < 8 || n > c->max_nodes || !(L > 0.0)) return KFBI_ERR_ARG;
  if (prm->kind != KFBI_STEP_HELE_SHAW && prm->kind != KFBI_STEP_STEFAN) return KFBI_ERR_ARG;
  if (prm->kind == KFBI_STEP_HELE_SHAW && c->boxbc != KFBI_BOX_FREESPACE_DL) return KFBI_ERR_ARG;
  if (prm->kind == KFBI_STEP_STEFAN && (c->boxbc != KFBI_BOX_NEUMANN0 || !(prm->eps_v >= 0.0))) return KFBI_ERR_ARG;
  if (prm->scheme != KFBI_SCHEME_SEMI_IMPLICIT && prm->scheme != KFBI_SCHEME_EXPLICIT) return KFBI_ERR_ARG;
  if (!(prm->refine_ratio >= 0.0) || (prm->rescale != 0 && prm->kind != KFBI_STEP_HELE_SHAW)) return KFBI_ERR_ARG;
  if (!(prm->tol > 0.0) || prm->max_iter < 1 || prm->restart < 1 || prm->restart > MAX_RESTART) return KFBI_ERR_ARG;
  kfbi_thetal* st = new kfbi_thetal();
  kfbi_status s = thetal_create_impl(c, n, eta, L, xbar, prm, st);
  if (s != KFBI_OK) {
    thetal_free(st);
    delete st;
    return s;
  }
  *out = st;
  return KFBI_OK;
}

void kfbi_thetal_destroy(kfbi_thetal* st) {
  if (st == nullptr) return;
  if (st->ctx) cudaStreamSynchronize(st->ctx->stream);
  thetal_free(st);
  delete st;
}

kfbi_status kfbi_step(kfbi_ctx* c, kfbi_thetal* st, double dt, kfbi_solve_info* info) {
  if (c == nullptr || st == nullptr || st->ctx != c || !(dt > 0.0)) return KFBI_ERR_ARG;
  if (st->prm.kind == KFBI_STEP_STEFAN) {
    // the operator Delta - 3/(2 dt) of the BDF2 step is the context's Delta - kappa
    double want = 3.0 / (2.0 * dt);
    if (fabs(want - c->kappa) > 1e-12 * want) return KFBI_ERR_ARG;
  }
  KFBI_TRY(stream_enter(c));
  kfbi_status s = thetal_step_impl(c, st, dt, info);
  KFBI_TRY(stream_exit(c));
  return s;
}

kfbi_status kfbi_thetal_read(kfbi_thetal* st, double* eta, double* xy, double* density, double* nhat, double* T,
                             double* T_prev, double* scalars) {
  if (st == nullptr) return KFBI_ERR_ARG;
  cudaStream_t s = st->ctx->stream;
  const int n = st->n;
  const size_t NN = (size_t)st->ctx->N * st->ctx->N;
  const size_t nk = (size_t)(n / 2 + 1);
  KFBI_TRY(stream_enter(st->ctx));
  if (eta) KFBI_TRY(cudaMemcpyAsync(eta, st->eta, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (xy) KFBI_TRY(cudaMemcpyAsync(xy, st->xy, 2 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (density) KFBI_TRY(cudaMemcpyAsync(density, st->density, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (nhat) KFBI_TRY(cudaMemcpyAsync(nhat, st->Nprev_h, 2 * nk * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (T && st->T) KFBI_TRY(cudaMemcpyAsync(T, st->T, NN * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (T_prev && st->Tprev) KFBI_TRY(cudaMemcpyAsync(T_prev, st->Tprev, NN * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (scalars) {
    KFBI_TRY(cudaMemcpyAsync(st->host_scal, st->scal, SC_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
    KFBI_TRY(cudaStreamSynchronize(s));
    for (int i = 0; i < SC_COUNT; ++i) scalars[i] = st->host_scal[i];
  }
  KFBI_TRY(stream_exit(st->ctx));
  return KFBI_OK;
}

kfbi_status kfbi_thetal_count(kfbi_thetal* st, int* n) {
  if (st == nullptr || n == nullptr) return KFBI_ERR_ARG;
  *n = st->n;
  return KFBI_OK;
}

kfbi_status kfbi_thetal_set_warmstart(kfbi_thetal* st, kfbi_mlp* mlp) {
  if (st == nullptr) return KFBI_ERR_ARG;
  st->ws = mlp;
  return KFBI_OK;
}

kfbi_status kfbi_thetal_training_pair(kfbi_thetal* st, float* feat, float* target) {
  if (st == nullptr || feat == nullptr || target == nullptr) return KFBI_ERR_ARG;
  kfbi_ctx* c = st->ctx;
  if (!c->have_iface || c->n != st->n) return KFBI_ERR_STATE;
  KFBI_CHECK(kfbi_warmstart_features(c, st->rhs, feat, st->ws_norm));
  KFBI_TRY(stream_enter(c));
  k_ws_target<<<cdiv(st->n, 256), 256, 0, c->stream>>>(st->n, st->density, st->ws_norm, target);
  launched(c, 1);
  KFBI_TRY(cudaGetLastError());
  KFBI_TRY(stream_exit(c));
  return KFBI_OK;
}

kfbi_status kfbi_thetal_write(kfbi_thetal* st, const double* eta, const double* density, const double* nhat,
                              const double* T, const double* T_prev, const double* scalars) {
  if (st == nullptr) return KFBI_ERR_ARG;
  cudaStream_t s = st->ctx->stream;
  const int n = st->n;
  const size_t NN = (size_t)st->ctx->N * st->ctx->N;
  const size_t nk = (size_t)(n / 2 + 1);
  KFBI_TRY(stream_enter(st->ctx));
  if (eta) KFBI_TRY(cudaMemcpyAsync(st->eta, eta, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (density) KFBI_TRY(cudaMemcpyAsync(st->density, density, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (nhat) KFBI_TRY(cudaMemcpyAsync(st->Nprev_h, nhat, 2 * nk * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (T && st->T) KFBI_TRY(cudaMemcpyAsync(st->T, T, NN * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (T_prev && st->Tprev) KFBI_TRY(cudaMemcpyAsync(st->Tprev, T_prev, NN * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (scalars) {
    KFBI_TRY(cudaStreamSynchronize(s));
    for (int i = 0; i < SC_COUNT; ++i) st->host_scal[i] = scalars[i];
    KFBI_TRY(cudaMemcpyAsync(st->scal, st->host_scal, SC_COUNT * sizeof(double), cudaMemcpyHostToDevice, s));
    KFBI_TRY(cudaStreamSynchronize(s));
  }
  KFBI_TRY(stream_exit(st->ctx));
  return KFBI_OK;
}

}  // extern "C"
