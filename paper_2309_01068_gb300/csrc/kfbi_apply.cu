// The KFBI apply (Sec. 4): jumps at crossings and nodes (App. A.1), corrected five-point
// right-hand side (Sec. 4.2), free-space box data (Sec. 4.1), the fast DST/DCT solve and
// the jump-corrected 6-point interpolation (Sec. 4.3). Every kernel is templated on the
// grid arithmetic type T (double for KFBI_FP64, float for the inner applies of
// KFBI_MIXED); interface inputs and outputs stay float64.
//
// Data flow of one apply (N x N grid, spectral grid `spec` row-major [j][k]):
//   k_dens_coef      density Fourier coefficients (DFT, exact twiddle indexing)
//   k_target_jumps   jumps at every crossing and node from the coefficients
//   k_jumps_fft      (float32, power-of-two n) both of the above in one kernel, the
//                    coefficients by a shared-memory FFT in every block
//   k_box_data       free-space box data on the four faces (Hele-Shaw box only)
//   k_face_dst       DST-II along x of the two dense face rows (Hele-Shaw box only; with the
//                    box table its face rows are pre-transformed and this kernel is skipped)
//   k_row_forward    per row: corrections at its irregular nodes + box terms -> DST along x
//   k_col_solve      per column: DST along y, divide by the eigenvalue, inverse along y
//   k_probe_values   inverse along x only at the interpolation points
//   k_interp         6-point jump-corrected interpolation -> boundary operator values
#include <cmath>
#include <mutex>
#include <type_traits>
#include <utility>

#include "kfbi_dct.cuh"
#include "kfbi_fft.cuh"
#include "kfbi_internal.cuh"

namespace kfbi {

template <typename T>
__device__ __forceinline__ T wsum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T qnan();
template <>
__device__ __forceinline__ float qnan<float>() { return __int_as_float(0x7fc00000); }
template <>
__device__ __forceinline__ double qnan<double>() { return __longlong_as_double(0x7ff8000000000000LL); }

// largest dynamic shared memory a kernel stages its inputs in (bytes); larger inputs are read
// from global memory
constexpr size_t SMEM_STAGE_MAX = 96 * 1024;

template <typename T>
struct Tabs;  // typed views of the context's tables and geometry
template <>
struct Tabs<double> {
  static const double* sin(const kfbi_ctx* c) { return c->sintab; }
  static const double* lam(const kfbi_ctx* c) { return c->lam; }
  static const V2<double>* twN(const kfbi_ctx* c) { return (const V2<double>*)c->twN; }
  static const V2<double>* stw(const kfbi_ctx* c) { return (const V2<double>*)c->stw_d; }
  static const TargetGeo* geo(const kfbi_ctx* c) { return c->tgeo; }
  static const Stencil* stencil(const kfbi_ctx* c) { return c->stencil; }
  static const V2<double>* twn(const kfbi_ctx* c) { return (const V2<double>*)c->twn; }
  static const V2<double>* tstart(const kfbi_ctx* c) { return (const V2<double>*)c->tstart; }
  static const double4_32a* npack(const kfbi_ctx* c) { return (const double4_32a*)c->npack; }
};
template <>
struct Tabs<float> {
  static const float* sin(const kfbi_ctx* c) { return c->sintab_f; }
  static const float* lam(const kfbi_ctx* c) { return c->lam_f; }
  static const V2<float>* twN(const kfbi_ctx* c) { return (const V2<float>*)c->twN_f; }
  static const V2<float>* stw(const kfbi_ctx* c) { return (const V2<float>*)c->stw; }
  static const TargetGeoF* geo(const kfbi_ctx* c) { return c->tgeo_f; }
  static const StencilF* stencil(const kfbi_ctx* c) { return c->stencil_f; }
  static const V2<float>* twn(const kfbi_ctx* c) { return (const V2<float>*)c->twn_f; }
  static const V2<float>* tstart(const kfbi_ctx* c) { return (const V2<float>*)c->tstart_f; }
  static const float4* npack(const kfbi_ctx* c) { return (const float4*)c->npack_f; }
};

// per-type fields of an irregular node
__device__ __forceinline__ double irr_d(const IrrNode& q, int a, double) { return q.d[a]; }
__device__ __forceinline__ float irr_d(const IrrNode& q, int a, float) { return q.df[a]; }
__device__ __forceinline__ double irr_sign(const IrrNode& q, double) { return q.sign; }
__device__ __forceinline__ float irr_sign(const IrrNode& q, float) { return q.signf; }

__global__ void k_to_float(const double* a, float* b, int n, const int* skip) {
  pdl_wait();
  if (*skip) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// --------------------------------------------------------------------------- density
// c_k = (1/n) sum_j phi_j e^{-2 pi i k j / n} (k = 0..n/2): one warp per k, twiddle index
// k j mod n advanced incrementally; the block stages the density and the twiddles in shared
// memory (SMEM = true) or reads them from global memory (large n). Block 0 also forms
// int phi ds = sum_j phi_j s_a,j 2 pi / n (trapezoidal rule) for the Hele-Shaw operator, as a
// block-wide tree so that its dependency depth stays logarithmic in n.
template <typename T, bool SMEM, typename S_t>
__global__ void k_dens_coef(const T* phi, int n, const V2<T>* tw, const S_t* st, V2<T>* coef, T* dint,
                            const int* skip) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ T red[32];
  V2<T>* stw = (V2<T>*)smem_raw;
  T* sphi = (T*)(stw + n);
  // the twiddles are fixed with the interface: staged before the wait for the previous kernel
  if (SMEM)
    for (int j = threadIdx.x; j < n; j += blockDim.x) stw[j] = tw[j];
  pdl_wait();
  if (*skip) return;
  if (SMEM) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) sphi[j] = phi[j];
    __syncthreads();
  }
  int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (blockIdx.x == 0 && dint != nullptr) {
    T s0 = 0, s1 = 0;
    int j = threadIdx.x;
    for (; j + (int)blockDim.x < n; j += 2 * blockDim.x) {
      s0 += (SMEM ? sphi[j] : phi[j]) * (T)st[j].w;
      s1 += (SMEM ? sphi[j + blockDim.x] : phi[j + blockDim.x]) * (T)st[j + blockDim.x].w;
    }
    if (j < n) s0 += (SMEM ? sphi[j] : phi[j]) * (T)st[j].w;
    T s = wsum(s0 + s1);
    if (lane == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
      T t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : (T)0;
      t = wsum(t);
      if (threadIdx.x == 0) *dint = t;
    }
  }
  if (k > n / 2) return;
  int idx = (int)(((long)k * lane) % n);
  const int step = (int)(((long)k * 32) % n);
  T re = 0, im = 0;
  for (int j = lane; j < n; j += 32) {
    T v = SMEM ? sphi[j] : phi[j];
    V2<T> w = SMEM ? stw[idx] : tw[idx];
    re += v * w.x;
    im -= v * w.y;
    idx += step;
    if (idx >= n) idx -= n;
  }
  re = wsum(re);
  im = wsum(im);
  if (lane == 0) coef[k] = V2<T>{re / (T)n, im / (T)n};
}

// Warp-level jumps at one target (App. A.1, Table 2): the warp sums the density interpolant
// and its first two derivatives from the precomputed twiddle starts (lane l sums the modes
// [k0_l, k0_l + chunk) from e0 = e^{i k0_l alpha}, rotating by s1 = e^{i alpha}; the Nyquist
// term uses q = e^{i n alpha / 2}), then every lane solves the 2x2 and 3x3 systems and holds
// J = ([u], [u_x], [u_y], [u_xx], [u_yy], [u_xy]).
// Shared-memory layout of the coefficients for it (jump_layout): c_0, then lane l's modes
// [1 + l chunk, 1 + (l+1) chunk) from position 1 + l S, S = chunk rounded up to an odd
// number so that the 32 lanes' simultaneous reads fall in distinct banks, then the Nyquist
// coefficient at 1 + 32 S.
__host__ __device__ inline int jump_chunk(int n) { return ((n - 1) / 2 + 31) / 32; }
__host__ __device__ inline int jump_stride(int n) { const int c = jump_chunk(n); return (c & 1) ? c : c + 1; }
__host__ __device__ inline int jump_layout_size(int n) { return 2 + 32 * jump_stride(n); }

// lane_coef: this lane's modes k0, k0 + 1, ... (contiguous); c0 = c_0, nyq = c_{n/2} (even n)
template <typename T, typename G>
__device__ __forceinline__ void jump_eval(const V2<T>* lane_coef, V2<T> c0, V2<T> cnyq, int n, V2<T> e0, V2<T> s1,
                                          V2<T> q, const G& g, int layer, T kappa, int lane, T J[6]) {
  const int K = (n - 1) / 2;
  const int chunk = jump_chunk(n);
  int k0 = 1 + lane * chunk;
  int k1 = min(K + 1, k0 + chunk);
  T a = 0, b = 0, d = 0;
  if (k0 < k1) {
    if constexpr (sizeof(T) == 8) {
      // float64: four interleaved rotations (modes k0 + 4 i + r) and accumulators, so that
      // each dependency chain is a quarter as long (float64 latency is long on this part)
      const V2<T> s2 = cmul(s1, s1), s4 = cmul(s2, s2);
      V2<T> e[4] = {e0, cmul(e0, s1), cmul(e0, s2), cmul(cmul(e0, s2), s1)};
      T aa[4] = {0, 0, 0, 0}, bb[4] = {0, 0, 0, 0}, dd[4] = {0, 0, 0, 0};
      for (int k = k0; k < k1; k += 4) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          if (k + r < k1) {
            const V2<T> ck = lane_coef[k + r - k0];
            const T re = ck.x * e[r].x - ck.y * e[r].y;
            const T im = ck.x * e[r].y + ck.y * e[r].x;
            const T kk = (T)(k + r);
            aa[r] += re;
            bb[r] -= kk * im;
            dd[r] -= kk * kk * re;
            e[r] = cmul(e[r], s4);
          }
        }
      }
      a = (aa[0] + aa[1]) + (aa[2] + aa[3]);
      b = (bb[0] + bb[1]) + (bb[2] + bb[3]);
      d = (dd[0] + dd[1]) + (dd[2] + dd[3]);
    } else {
      V2<T> e = e0;
      const V2<T> s = s1;
      for (int k = k0; k < k1; ++k) {
        V2<T> ck = lane_coef[k - k0];
        T re = ck.x * e.x - ck.y * e.y;
        T im = ck.x * e.y + ck.y * e.x;
        T kk = (T)k;
        a += re;
        b -= kk * im;
        d -= kk * kk * re;
        e = cmul(e, s);
      }
    }
  }
  a = (T)2 * wsum(a) + c0.x;
  b = (T)2 * wsum(b);
  d = (T)2 * wsum(d);
  if ((n & 1) == 0) {
    T m = (T)(n / 2);
    T nyq = cnyq.x;
    a += nyq * q.x;
    b -= m * nyq * q.y;
    d -= m * m * nyq * q.x;
  }
  T Phi, Phia, Phiaa, Psi, Psia;
  if (layer == KFBI_DOUBLE) {
    Phi = a; Phia = b; Phiaa = d; Psi = 0; Psia = 0;
  } else {
    Phi = 0; Phia = 0; Phiaa = 0; Psi = -a; Psia = -b;
  }
  T xa = (T)g.xa, ya = (T)g.ya, xaa = (T)g.xaa, yaa = (T)g.yaa, sa = (T)g.sa, saa = (T)g.saa;
  T is2 = (T)1 / (sa * sa);
  T ux = (xa * Phia + ya * sa * Psi) * is2;
  T uy = (ya * Phia - xa * sa * Psi) * is2;
  T b0 = Phiaa - xaa * ux - yaa * uy;
  T b1 = saa * Psi + sa * Psia - yaa * ux + xaa * uy;
  T b2 = kappa * Phi;
  J[0] = Phi;
  J[1] = ux;
  J[2] = uy;
  J[3] = (T)g.A3i[0] * b0 + (T)g.A3i[1] * b1 + (T)g.A3i[2] * b2;
  J[4] = (T)g.A3i[3] * b0 + (T)g.A3i[4] * b1 + (T)g.A3i[5] * b2;
  J[5] = (T)g.A3i[6] * b0 + (T)g.A3i[7] * b1 + (T)g.A3i[8] * b2;
}

// Jumps at every target (crossings, then nodes), one warp per target; the block stages the
// density coefficients in shared memory first (SMEM = true; large n reads them from global memory). J[t] = ([u], [u_x], [u_y], [u_xx], [u_yy], [u_xy]).
template <typename T, typename G, bool SMEM>
__global__ void k_target_jumps(const V2<T>* coef, int n, const int* ncr, const G* tg, const V2<T>* tstart, int layer,
                               T kappa, T* Jout, const int* skip) {
  // targets: the interface's crossings (count on the device, so that a captured launch stays
  // valid for the next interface) and its n nodes; the grid covers the crossing capacity
  const int ntg = *ncr + n;
  int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  // geometry and twiddle starts of this target (set with the interface) before the wait
  G geo{};
  V2<T> e0{}, s1{}, q{};
  if (t < ntg) {
    geo = tg[t];
    const V2<T>* ts = tstart + (long)t * TSTART_STRIDE;
    e0 = ts[lane];
    s1 = ts[32];
    q = ts[33];
  }
  pdl_wait();
  if (*skip) return;
  extern __shared__ unsigned char smem_raw[];
  const int chunk = jump_chunk(n);
  const V2<T>* lane_coef = coef + 1 + lane * chunk;
  V2<T> c0, cnyq{0, 0};
  if (SMEM) {
    V2<T>* w = (V2<T>*)smem_raw;
    const int S = jump_stride(n), K = (n - 1) / 2;
    for (int k = 1 + (int)threadIdx.x; k <= K; k += blockDim.x) {
      const int l = (k - 1) / chunk;
      w[1 + l * S + (k - 1 - l * chunk)] = coef[k];
    }
    if (threadIdx.x == 0) {
      w[0] = coef[0];
      if ((n & 1) == 0) w[1 + 32 * S] = coef[n / 2];
    }
    __syncthreads();
    lane_coef = w + 1 + lane * S;
    c0 = w[0];
    if ((n & 1) == 0) cnyq = w[1 + 32 * S];
  } else {
    c0 = coef[0];
    if ((n & 1) == 0) cnyq = coef[n / 2];
  }
  if (t >= ntg) return;
  T J[6];
  jump_eval<T, G>(lane_coef, c0, cnyq, n, e0, s1, q, geo, layer, kappa, lane, J);
  // lane < 6 stores J[lane] (selected without indexing the array, which stays in registers)
  T v = J[5];
#pragma unroll
  for (int r = 4; r >= 0; --r) v = lane == r ? J[r] : v;
  if (lane < 6) Jout[(long)t * 6 + lane] = v;
}

// The jumps of k_target_jumps (App. A.1, Table 2) with the density's Fourier coefficients (the
// trigonometric interpolant of the nodal density) formed inside every block, for
// the float32 inner applies with a power-of-two node count n <= 4096 (in place of k_dens_coef
// + k_target_jumps: one launch and one global round trip fewer per apply). Each block takes
// the length-n FFT of the density in shared memory (c_k = X_k / n, the same coefficients as
// the DFT of k_dens_coef up to rounding order), lays them out as k_target_jumps does and
// evaluates its eight targets; block 0 also forms int phi ds. Shared memory: two buffers of
// max(n, jump layout) complex values and the staged FFT twiddles (at most 96 KB at n = 4096).
__host__ __device__ inline int jfft_buf(int n) {
  const int l = jump_layout_size(n);
  return n > l ? n : l;
}
__host__ __device__ inline size_t jfft_smem(int n, int logn) {
  return sizeof(V2<float>) * (2 * (size_t)jfft_buf(n) + (size_t)staged_count(n, logn));
}
constexpr int JFFT_THREADS = 512;
constexpr int JFFT_PER = 4096 / JFFT_THREADS;  // density values per thread at most

template <typename G, typename S_t>
__global__ void __launch_bounds__(JFFT_THREADS, 1)
    k_jumps_fft(const float* phi, int n, int logn, const V2<float>* twn, const S_t* st, float* dint, const int* ncr,
                const G* tg, const V2<float>* tstart, int layer, float kappa, float* Jout, const int* arm_rev,
                const float2* arm_coef, float* arm_slot, const int* skip) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ float red[JFFT_THREADS / 32];
  const int L = jfft_buf(n);
  V2<float>* A = (V2<float>*)smem_raw;
  V2<float>* B = A + L;
  V2<float>* stw = B + L;
  const int ntg = *ncr + n;
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if ((int)blockIdx.x * (JFFT_THREADS / 32) >= ntg) {
    pdl_wait();  // no target in this block (the grid covers the crossing capacity)
    return;
  }
  // fixed with the interface, read before the wait: the target's geometry and twiddle starts,
  // the FFT's staged twiddles w^{r jm n / (4 Ns)} = conj(e^{2 pi i r jm / (4 Ns)}) from the
  // node roots, and (block 0) the arclength weights of the density integral
  G geo{};
  V2<float> e0{}, s1{}, q{};
  // the arm this lane corrects (lanes 0, 1 of a crossing's warp; arm_slot set: the column
  // kernel forms the row transform from these corrections)
  int arm = -1;
  float2 acoef{0.f, 0.f};
  if (t < ntg) {
    geo = tg[t];
    const V2<float>* ts = tstart + (long)t * TSTART_STRIDE;
    e0 = ts[lane];
    s1 = ts[32];
    q = ts[33];
    if (arm_slot != nullptr && lane < 2 && t < *ncr) {
      arm = arm_rev[2 * t + lane];
      if (arm >= 0) acoef = arm_coef[2 * t + lane];
    }
  }
  const int cnt = staged_count(n, logn);
  for (int i = threadIdx.x; i < cnt; i += JFFT_THREADS) {
    int off = 0, Ns = (logn & 1) ? 2 : 1;
    while (i >= off + 3 * Ns) {
      off += 3 * Ns;
      Ns <<= 2;
    }
    const int r = (i - off) / Ns + 1, jm = (i - off) - (r - 1) * Ns;
    const V2<float> w = twn[r * jm * (n / (4 * Ns))];
    stw[i] = V2<float>{w.x, -w.y};
  }
  const bool want_int = blockIdx.x == 0 && dint != nullptr;
  float wt[JFFT_PER];
#pragma unroll
  for (int u = 0; u < JFFT_PER; ++u) {
    const int j = threadIdx.x + u * JFFT_THREADS;
    wt[u] = (want_int && j < n) ? st[j].w : 0.0f;
  }
  pdl_wait();
  // the density and the skip flag in one round trip
  float v[JFFT_PER];
#pragma unroll
  for (int u = 0; u < JFFT_PER; ++u) {
    const int j = threadIdx.x + u * JFFT_THREADS;
    v[u] = j < n ? phi[j] : 0.0f;
  }
  if (*skip) return;
  if (want_int) {
    float s = 0.0f;
#pragma unroll
    for (int u = 0; u < JFFT_PER; ++u) s += v[u] * wt[u];
    s = wsum(s);
    if (lane == 0) red[threadIdx.x >> 5] = s;
  }
#pragma unroll
  for (int u = 0; u < JFFT_PER; ++u) {
    const int j = threadIdx.x + u * JFFT_THREADS;
    if (j < n) A[j] = V2<float>{v[u], 0.0f};
  }
  __syncthreads();
  if (want_int && threadIdx.x < 32) {
    float s = threadIdx.x < JFFT_THREADS / 32 ? red[threadIdx.x] : 0.0f;
    s = wsum(s);
    if (threadIdx.x == 0) *dint = s;
  }
  const V2<float>* X = fft_stockham<float>(A, B, 1, n, logn, stw, false);
  V2<float>* w = X == A ? B : A;
  const float inv_n = 1.0f / (float)n;
  const int S = jump_stride(n), K = (n - 1) / 2, chunk = jump_chunk(n);
  for (int k = 1 + (int)threadIdx.x; k <= K; k += JFFT_THREADS) {
    const int l = (k - 1) / chunk;
    w[1 + l * S + (k - 1 - l * chunk)] = V2<float>{X[k].x * inv_n, X[k].y * inv_n};
  }
  if (threadIdx.x == 0) {
    w[0] = V2<float>{X[0].x * inv_n, X[0].y * inv_n};
    w[1 + 32 * S] = V2<float>{X[n / 2].x * inv_n, X[n / 2].y * inv_n};  // n is even
  }
  __syncthreads();
  if (t >= ntg) return;
  float J[6];
  jump_eval<float, G>(w + 1 + lane * S, w[0], w[1 + 32 * S], n, e0, s1, q, geo, layer, kappa, lane, J);
  float o = J[5];
#pragma unroll
  for (int r = 4; r >= 0; --r) o = lane == r ? J[r] : o;
  if (lane < 6) Jout[(long)t * 6 + lane] = o;
  // the arm's correction sign / h^2 (J0 + d J1 + d^2 J2 / 2), J1, J2 the derivatives along it
  if (arm >= 0) {
    const bool xarm = (arm & 3) < 2;
    const float d = acoef.x;
    arm_slot[arm] = acoef.y * (J[0] + d * (xarm ? J[1] : J[2]) + 0.5f * d * d * (xarm ? J[3] : J[4]));
  }
}

// Free-space box data (Sec. 4.1): g(p) = (1/n) sum_l phi_l (X_l - p).(y_a, -x_a)_l / |X_l - p|^2
// at the 4N face midpoints (west, east, south, north), stored pre-scaled as the
// right-hand side term -2 g / h^2. npack[l] = (x, y, y_a, -x_a) of node l.
template <typename T, typename T4, bool SMEM>
__global__ void k_box_data(const T* phi, int n, const T4* npack, int N, double xmin, double xmax, double ymin,
                           double ymax, double h, T scale, T* boxg, const int* skip) {
  pdl_wait();
  if (*skip) return;
  extern __shared__ unsigned char smem_raw[];
  T4* sp = (T4*)smem_raw;  // (x, y, phi y_a, -phi x_a)
  if (SMEM) {
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
      T4 q = npack[l];
      T f = phi[l];
      q.z *= f;
      q.w *= f;
      sp[l] = q;
    }
    __syncthreads();
  }
  int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= 4 * N) return;
  int face = w / N, idx = w - face * N;
  // face midpoint: float64 rounding as the oracle's grid; float32 arithmetic in the float32
  // apply (the float64 pipe is slow and its precision is not needed there)
  T tpx, tpy;
  if constexpr (sizeof(T) == 8) {
    if (face == 0) { tpx = xmin; tpy = grid_coord(ymin, h, idx); }
    else if (face == 1) { tpx = xmax; tpy = grid_coord(ymin, h, idx); }
    else if (face == 2) { tpx = grid_coord(xmin, h, idx); tpy = ymin; }
    else { tpx = grid_coord(xmin, h, idx); tpy = ymax; }
  } else {
    const T c = ((T)idx + (T)0.5) * (T)h;
    if (face == 0) { tpx = (T)xmin; tpy = (T)ymin + c; }
    else if (face == 1) { tpx = (T)xmax; tpy = (T)ymin + c; }
    else if (face == 2) { tpx = (T)xmin + c; tpy = (T)ymin; }
    else { tpx = (T)xmin + c; tpy = (T)ymax; }
  }
  T acc = 0;
  for (int l = lane; l < n; l += 32) {
    T4 q;
    if (SMEM) {
      q = sp[l];
    } else {
      q = npack[l];
      T f = phi[l];
      q.z *= f;
      q.w *= f;
    }
    T dx = q.x - tpx, dy = q.y - tpy;
    acc += fdiv_t(dx * q.z + dy * q.w, dx * dx + dy * dy);
  }
  acc = wsum(acc);
  if (lane == 0) boxg[w] = scale * acc;
}

// Free-space box data as a product with a kernel fixed by the interface: for face point w
// (west, east, south, north faces, N each) and node l,
//   K[w][l] = -2 / (h^2 n) ((X_l - p_w).(y_a, -x_a)_l) / |X_l - p_w|^2
// (the trapezoidal double layer of Sec. 4.1 at p_w, pre-scaled as the right-hand side term
// -2 g / h^2), so that boxg = K phi. Computed once per interface in float64 with a float32
// copy, rows of box_ld(n) entries (zeros past n); every apply then reads it (4N n values)
// instead of re-evaluating it.
// Thread per (node column l, face, chunk of BOXK_CHUNK face points): the node's offset along
// the face normal and its products are formed once, each entry then costs a few float64
// operations and one correctly rounded reciprocal (__drcp_rn).
constexpr int BOXK_CHUNK = 64;
__global__ void k_box_matrix(int N, int n, int ld, const double4_32a* npack, double xmin, double xmax, double ymin,
                             double ymax, double h, double scale, double* K, float* Kf) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  const int face = blockIdx.y;
  const int i0 = blockIdx.z * BOXK_CHUNK, i1 = min(N, i0 + BOXK_CHUNK);
  if (l >= ld) return;
  double* Kr = K + (long)face * N * ld + l;
  float* Kfr = Kf + (long)face * N * ld + l;
  if (l >= n) {
    for (int idx = i0; idx < i1; ++idx) {
      Kr[(long)idx * ld] = 0.0;
      Kfr[(long)idx * ld] = 0.0f;
    }
    return;
  }
  const double4_32a q = npack[l];
  // west/east faces: x fixed (offset a along x), y = grid_coord(ymin, h, idx) varies;
  // south/north faces: y fixed, x varies. (q.z, q.w) = (y_a, -x_a) of the node.
  const bool vert = face < 2;
  const double a = vert ? q.x - (face == 0 ? xmin : xmax) : q.y - (face == 2 ? ymin : ymax);
  const double na = a * (vert ? q.z : q.w);  // normal-offset part of the numerator
  const double a2 = a * a;
  const double bq = vert ? q.y : q.x, bz = vert ? q.w : q.z, lo = vert ? ymin : xmin;
  for (int idx = i0; idx < i1; ++idx) {
    const double t = bq - grid_coord(lo, h, idx);  // offset along the face
    const double num = fma(t, bz, na);
    const double den = fma(t, t, a2);
    const double k = scale * num * __drcp_rn(den);
    Kr[(long)idx * ld] = k;
    Kfr[(long)idx * ld] = (float)k;
  }
}

// four consecutive table or density values (16-byte aligned for float, 32 for double)
__device__ __forceinline__ void load4(const float* p, float v[4]) {
  const float4 f = *(const float4*)p;
  v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
}
__device__ __forceinline__ void load4(const double* p, double v[4]) {
  const double2 a = ((const double2*)p)[0], b = ((const double2*)p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// boxg[w] = sum_l K[w][l] phi_l: one warp per face point; lane l takes nodes 4 l + 128 t + c
// with one 16-byte table load per four nodes (VEC: phi read the same way, else per value),
// then the nodes past the last full group of four one by one
template <typename T, bool VEC>
__global__ void k_box_gemv(const T* K, int ld, const T* phi, int n, int rows, T* boxg, const int* skip) {
  pdl_wait();
  if (*skip) return;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= rows) return;
  const T* row = K + (long)w * ld;
  const int n4 = n & ~3;
  T a[4] = {0, 0, 0, 0};
#pragma unroll 2
  for (int l = 4 * lane; l < n4; l += 128) {
    T kv[4], pv[4];
    load4(row + l, kv);
    if (VEC) {
      load4(phi + l, pv);
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) pv[c] = phi[l + c];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) a[c] += kv[c] * pv[c];
  }
  if (n4 + lane < n) a[0] += row[n4 + lane] * phi[n4 + lane];
  const T s = wsum((a[0] + a[1]) + (a[2] + a[3]));
  if (lane == 0) boxg[w] = s;
}

// copies the staged twiddles to shared memory (before the block's first __syncthreads)
template <typename T>
__device__ __forceinline__ void stage_twiddles(const V2<T>* tw, V2<T>* sTw, int cnt) {
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) sTw[t] = tw[t];
}

// --------------------------------------------------------------------------- face rows
// DST-II / DCT-II along x of the south and north face data (two dense rows of the free-space
// right-hand side), one block; out[0..N) = south, out[N..2N) = north, in mode order.
template <typename T>
__global__ void k_face_dst(int N, int logN, int dct, const V2<T>* tw, const T* tab, const T* boxg, T* out,
                           const int* skip) {
  extern __shared__ unsigned char smem_raw[];
  V2<T>* A = (V2<T>*)smem_raw;
  V2<T>* B = A + N;
  V2<T>* sTw = B + N;  // staged twiddles (one global round trip instead of one per stage)
  stage_twiddles(tw, sTw, staged_count(N, logN));  // fixed with the context: before the wait
  pdl_wait();
  if (*skip) return;
  const T* gs = boxg + 2 * N;
  const T* gn = boxg + 3 * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    T a = gs[i], b = gn[i];
    if (!dct && (i & 1)) { a = -a; b = -b; }
    A[mk_pos(i, N)] = V2<T>{a, b};
  }
  __syncthreads();
  V2<T>* X = fft_stockham<T>(A, B, 1, N, logN, sTw, false);
  for (int m = threadIdx.x; m <= N / 2; m += blockDim.x) {
    V2<T> Xm, XNm;
    T cm, sm;
    dct_cs<T>(tab, N, m, cm, sm);
    dct_post<T>(X, N, m, cm, sm, Xm, XNm);
    int km = dct ? m : N - 1 - m;
    out[km] = Xm.x;
    out[N + km] = Xm.y;
    if (m > 0 && m < N / 2) {
      int kNm = dct ? N - m : m - 1;
      out[kNm] = XNm.x;
      out[N + kNm] = XNm.y;
    }
  }
}

// The free-space box table's (Sec. 4.1) south and north rows replaced by their DST-II along the
// face (the transform of the fast solve, Sec. 4.2),
// node column by node column: row 2N + k becomes sum_i S_k(i) K[2N + i][l] (S_k as in the row
// transform below) and row 3N + k the same for the north face. The box product K phi then
// yields the two dense face rows' x-transforms directly, so no apply needs k_face_dst.
// One block per node column: the column's south and north values as one complex FFT
// (Makhoul reordering, as k_face_dst), in float64, written to both tables.
__global__ void k_box_face_table(int N, int logN, int ld, const V2<double>* tw, const double* tab, double* K,
                                 float* Kf) {
  extern __shared__ unsigned char smem_raw[];
  V2<double>* A = (V2<double>*)smem_raw;
  V2<double>* B = A + N;
  V2<double>* sTw = B + N;
  stage_twiddles(tw, sTw, staged_count(N, logN));
  const long l = blockIdx.x;
  double* ks = K + (long)2 * N * ld + l;
  double* kn = K + (long)3 * N * ld + l;
  float* fs = Kf + (long)2 * N * ld + l;
  float* fn = Kf + (long)3 * N * ld + l;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double a = ks[(long)i * ld], b = kn[(long)i * ld];
    if (i & 1) {
      a = -a;
      b = -b;
    }
    A[mk_pos(i, N)] = V2<double>{a, b};
  }
  __syncthreads();
  const V2<double>* X = fft_stockham<double>(A, B, 1, N, logN, sTw, false);
  for (int m = threadIdx.x; m <= N / 2; m += blockDim.x) {
    V2<double> Xm, XNm;
    double cm, sm;
    dct_cs<double>(tab, N, m, cm, sm);
    dct_post<double>(X, N, m, cm, sm, Xm, XNm);
    const long km = (long)(N - 1 - m) * ld;
    ks[km] = Xm.x;
    kn[km] = Xm.y;
    fs[km] = (float)Xm.x;
    fn[km] = (float)Xm.y;
    if (m > 0 && m < N / 2) {
      const long kNm = (long)(m - 1) * ld;
      ks[kNm] = XNm.x;
      kn[kNm] = XNm.y;
      fs[kNm] = (float)XNm.x;
      fn[kNm] = (float)XNm.y;
    }
  }
}

// --------------------------------------------------------------------------- row transform
// Sparse forward transform along x of row j (Sec. 4.2: the corrected right-hand side is zero
// away from irregular nodes and, for free-space box data, the boundary cells):
//   spec[j][k] = sum_i C[j][i] S_k(i),  S_k(i) = sin(pi (k+1)(2i+1)/(2N)) (DST-II) or
//   cos(pi k (2i+1)/(2N)) (DCT-II), from the table sin(pi m / (2N)), m mod 4N.
// The corrections of the row's irregular nodes are formed here from the crossing jumps:
//   C = sign/h^2 sum_arms (J0 + d J1 + d^2/2 J2), J1, J2 = ([u_x], [u_xx]) on horizontal
//   arms and ([u_y], [u_yy]) on vertical arms, sign = -1 at an Omega+ node, +1 at Omega-.
constexpr int ROW_CAP = 512;

// the fields of an irregular node that its correction needs, in registers
template <typename T>
struct IrrRegs {
  int tg[4];
  T d[4];
  T sign;
  int i;
};
template <typename T>
__device__ __forceinline__ IrrRegs<T> irr_regs(const IrrNode& q) {
  IrrRegs<T> r;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    r.tg[a] = q.target[a];
    r.d[a] = irr_d(q, a, T(0));
  }
  r.sign = irr_sign(q, T(0));
  r.i = q.i;
  return r;
}
constexpr int ROW_THREADS = 256;  // N <= 4096 gives at most 16 outputs per thread

template <typename T>
__global__ void __launch_bounds__(ROW_THREADS) k_row_forward(int N, int dct, const int* row_ptr, const IrrNode* irr,
                                                            const T* J, T inv_h2, const T* boxg,
                                                            const T* facespec, const T* tab, float scale, T* spec,
                                                            V2<T>* rowinfo, const int* skip) {
  __shared__ int si[ROW_CAP];
  __shared__ T sv[ROW_CAP];
  const int j = blockIdx.x;
  // the row's irregular nodes are fixed with the interface: this thread's first one is read
  // before the wait for the previous kernel (the jumps it needs come after)
  const int b = row_ptr[j], e = row_ptr[j + 1];
  IrrRegs<T> first{};
  if ((int)threadIdx.x < e - b) first = irr_regs<T>(irr[b + threadIdx.x]);
  // free-space box data of the row (west and east cells): complete before this kernel
  // starts (the stream waited for the side stream that forms it)
  T w = 0, ea = 0;
  if (boxg != nullptr) {
    w = boxg[j];
    ea = boxg[N + j];
  }
  pdl_wait();
  if (*skip) return;
  // rowinfo: a row without irregular nodes (other than a dense face row) holds only the box
  // terms w S_k(0) + e S_k(N-1) (zero without box data); its pair (w, e) is stored for the
  // column kernel, which forms the row itself, instead of its N values. Written rows are
  // marked by a NaN in the first entry.
  if (rowinfo != nullptr) {
    const bool face_row = boxg != nullptr && (j == 0 || j == N - 1);
    if (e == b && !face_row) {
      if (threadIdx.x == 0) rowinfo[j] = V2<T>{w, ea};
      return;
    }
    if (threadIdx.x == 0) rowinfo[j] = V2<T>{qnan<T>(), (T)0};
  }
  const int per = (N + ROW_THREADS - 1) / ROW_THREADS;
  T acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0;
  for (int c0 = b; c0 < e; c0 += ROW_CAP) {
    int cnt = min(ROW_CAP, e - c0);
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += ROW_THREADS) {
      const IrrRegs<T> node = (c0 == b && t == (int)threadIdx.x) ? first : irr_regs<T>(irr[c0 + t]);
      T sum = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int tg = node.tg[a];
        if (tg < 0) continue;
        const T* jj = J + (long)tg * 6;
        const T d = node.d[a];
        const T j1 = a < 2 ? jj[1] : jj[2];
        const T j2 = a < 2 ? jj[3] : jj[4];
        sum += jj[0] + d * j1 + (T)0.5 * d * d * j2;
      }
      si[t] = 2 * node.i + 1;
      sv[t] = node.sign * inv_h2 * sum;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      if (q >= per) break;
      int k = threadIdx.x + q * ROW_THREADS;
      T a = acc[q];
      if (k < N) {
        if (dct)
          for (int t = 0; t < cnt; ++t) a += sv[t] * tsin(tab, k * si[t] + N, N, scale);
        else
          for (int t = 0; t < cnt; ++t) a += sv[t] * tsin(tab, (k + 1) * si[t], N, scale);
      }
      acc[q] = a;
    }
  }
  const T* face = nullptr;
  if (boxg != nullptr) {
    if (j == 0) face = facespec;
    else if (j == N - 1) face = facespec + N;
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    if (q >= per) break;
    int k = threadIdx.x + q * ROW_THREADS;
    if (k >= N) break;
    T a = acc[q];
    if (boxg != nullptr) {
      if (dct) a += w * tsin(tab, k + N, N, scale) + ea * tsin(tab, k * (2 * N - 1) + N, N, scale);
      else a += w * tsin(tab, k + 1, N, scale) + ea * tsin(tab, (k + 1) * (2 * N - 1), N, scale);
      if (face != nullptr) a += face[k];
    }
    spec[(long)j * N + k] = a;
  }
}

// --------------------------------------------------------------------------- column solve
// For each column k of spec (x-mode k): forward transform along y, divide by
// lam_y(l) + lam_x(k) - kappa, inverse transform along y, in place. A block owns P column
// pairs; pair p holds columns (k0 + 2p, k0 + 2p + 1) as the real and imaginary parts of
// one complex FFT. Two shared buffers alternate between the FFT stages. One instantiation per
// grid size (N = 2^LOGN), so that the index arithmetic is constant.
template <typename T, int LOGN>
__global__ void __launch_bounds__(1024) k_col_solve(int, int, int P, int dct, const V2<T>* tw, const T* tab, const T* lam, T kappa, T* spec,
                            const T* rinv, const V2<T>* rowinfo, const int* skip) {
  constexpr int N = 1 << LOGN, logN = LOGN;
  extern __shared__ unsigned char smem_raw[];
  V2<T>* A = (V2<T>*)smem_raw;
  V2<T>* B = A + (long)P * N;
  V2<T>* sTw = B + (long)P * N;       // staged FFT twiddles
  const int nst = staged_count(N, logN);
  constexpr bool STAGE = sizeof(T) == 4;
  V2<T>* sCs = sTw + nst;             // float32: (cos, sin)(pi m / 2N), m = 0..N/2
  const T* sLam = STAGE ? (const T*)(sCs + N / 2 + 1) : lam;  // eigenvalues
  const int k0 = blockIdx.x * (2 * P);
  const int W = 2 * P, lw = __ffs(W) - 1;
  // every global read of the block is issued before the first barrier: the grid's tables
  // (twiddles, eigenvalues, DCT rotations, fixed with the context) straight into shared
  // memory before the wait for the previous kernel, then the column data through a register
  // buffer (eight loads in flight per thread)
  stage_twiddles(tw, sTw, nst);
  if (STAGE) {
    T* w = (T*)(sCs + N / 2 + 1);
    for (int t = threadIdx.x; t < N; t += blockDim.x) w[t] = lam[t];
    for (int m = threadIdx.x; m <= N / 2; m += blockDim.x) dct_cs<T>(tab, N, m, sCs[m].x, sCs[m].y);
  }
  // rows the row transform did not write (rowinfo, see k_row_forward) are w S_k(0) + e S_k(N-1)
  // for this thread's column k (blockDim is a multiple of W, so every element it loads is in
  // the same column)
  // (float32 only: the float64 kernel must keep its registers within the 1024-thread launch)
  constexpr bool ROWS = sizeof(T) == 4;
  T s0 = 0, sN = 0;
  if (ROWS && rowinfo != nullptr) {
    const int k = k0 + ((int)threadIdx.x & (W - 1));
    if (dct) {
      s0 = tsin(tab, k + N, N, qscale(N));
      sN = tsin(tab, k * (2 * N - 1) + N, N, qscale(N));
    } else {
      s0 = tsin(tab, k + 1, N, qscale(N));
      sN = tsin(tab, (k + 1) * (2 * N - 1), N, qscale(N));
    }
  }
  pdl_wait();
  if (*skip) return;
  const int tot = N * W;
  for (int t0 = 0; t0 < tot; t0 += 8 * (int)blockDim.x) {
    T buf[8];
    V2<T> rbuf[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = t0 + u * (int)blockDim.x + (int)threadIdx.x;
      if (t < tot) {
        buf[u] = spec[(long)(t >> lw) * N + k0 + (t & (W - 1))];
        if (ROWS && rowinfo != nullptr) rbuf[u] = rowinfo[t >> lw];
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = t0 + u * (int)blockDim.x + (int)threadIdx.x;
      if (t < tot) {
        const int j = t >> lw, c = t & (W - 1);
        T v = buf[u];
        if (ROWS && rowinfo != nullptr && rbuf[u].x == rbuf[u].x) v = rbuf[u].x * s0 + rbuf[u].y * sN;
        if (!dct && (j & 1)) v = -v;
        ((T*)&A[(long)(c >> 1) * N + mk_pos(j, N)])[c & 1] = v;
      }
    }
  }
  __syncthreads();
  V2<T>* X = fft_ct<T, LOGN, false>(A, B, P, sTw);
  V2<T>* Y = X == A ? B : A;
  const int half = N >> 1;
  const T kap = kappa;
  for (int p = 0; p < P; ++p) {
    const V2<T>* x = X + (long)p * N;
    V2<T>* y = Y + (long)p * N;
    const T lx0 = sLam[k0 + 2 * p] - kap, lx1 = sLam[k0 + 2 * p + 1] - kap;
    for (int m = threadIdx.x; m <= half; m += blockDim.x) {
      V2<T> cs;
      if (STAGE) cs = sCs[m];
      else dct_cs<T>(tab, N, m, cs.x, cs.y);
      V2<T> Xm, XNm;
      dct_post<T>(x, N, m, cs.x, cs.y, Xm, XNm);
      const int l1 = dct ? m : N - 1 - m, l2 = dct ? N - m : m - 1;
      V2<T> Gm, GNm{0, 0};
      if (sizeof(T) == 8 && rinv != nullptr) {
        // float64: products with the context's reciprocal table instead of divisions
        const T* r0 = rinv + (long)(k0 + 2 * p) * N;
        const T* r1 = r0 + N;
        Gm = V2<T>{Xm.x * r0[l1], Xm.y * r1[l1]};
        if (m == half) GNm = Gm;
        else if (m > 0) GNm = V2<T>{XNm.x * r0[l2], XNm.y * r1[l2]};
      } else {
        const T ly = sLam[l1];
        Gm = V2<T>{fdiv_t(Xm.x, ly + lx0), fdiv_t(Xm.y, ly + lx1)};
        if (m == half) {
          GNm = Gm;
        } else if (m > 0) {
          const T ly2 = sLam[l2];
          GNm = V2<T>{fdiv_t(XNm.x, ly2 + lx0), fdiv_t(XNm.y, ly2 + lx1)};
        }
      }
      V2<T> Zm, ZNm;
      dct_pre<T>(N, m, cs.x, cs.y, Gm, GNm, Zm, ZNm);
      y[m] = Zm;
      if (m > 0 && m < half) y[N - m] = ZNm;
    }
  }
  __syncthreads();
  V2<T>* Z = fft_ct<T, LOGN, true>(Y, X, P, sTw);
  const T invN = (T)1 / (T)N;
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    const int j = t >> lw, c = t & (W - 1);
    T v = ((const T*)&Z[(long)(c >> 1) * N + mk_pos(j, N)])[c & 1] * invN;
    if (!dct && (j & 1)) v = -v;
    spec[(long)j * N + k0 + c] = v;
  }
}

template <typename T>
using ColKernel = void (*)(int, int, int, int, const V2<T>*, const T*, const T*, T, T*, const T*, const V2<T>*,
                           const int*);
// the column kernel for N = 2^logN, 16 <= N <= 4096
template <typename T>
static ColKernel<T> col_kernel(int logN) {
  switch (logN) {
    case 4: return k_col_solve<T, 4>;
    case 5: return k_col_solve<T, 5>;
    case 6: return k_col_solve<T, 6>;
    case 7: return k_col_solve<T, 7>;
    case 8: return k_col_solve<T, 8>;
    case 9: return k_col_solve<T, 9>;
    case 10: return k_col_solve<T, 10>;
    case 11: return k_col_solve<T, 11>;
    default: return k_col_solve<T, 12>;
  }
}

// --------------------------------------------------------------------------- column solve, FFTs in registers
// The float32 column solve for N = A B <= 1024 with every FFT held in registers: B lanes own a
// column pair (two real columns as one complex sequence, Makhoul reordering as above) and each
// lane keeps A of its N points. Four-step decomposition of the length-N transform,
//   X[k1 + A k2] = sum_t W_B^{t k2} W_N^{t k1} sum_a v[t + B a] W_A^{a k1},
// so an FFT is an A-point DFT in registers, a twiddle, one transpose through shared memory
// (within the lanes' own warp: __syncwarp only) and B-point DFTs in registers. The inverse runs
// the same steps in mirror order and leaves the points in the layout they were loaded in. The
// DCT/DST post- and pre-processing pairs bin m with bin N - m, which another lane of the group
// holds: one shuffle per register brings it over.

// grid split of the register column kernel: N = A B, A = 2^ceil(logN / 2) points per lane,
// B = 2^floor(logN / 2) lanes per column pair, F column pairs (F B threads) per block
template <int LOGN>
struct ColRegPlan {
  static constexpr int N = 1 << LOGN;
  static constexpr int A = 1 << ((LOGN + 1) / 2);
  static constexpr int B = 1 << (LOGN / 2);
  static constexpr int F0 = 128 / B;
  static constexpr int F = F0 < N / 2 ? F0 : N / 2;
  static constexpr int THREADS = F * B;
  static constexpr int TPAD = (A * (B + 1) > B * (A + 1) ? A * (B + 1) : B * (A + 1));  // transpose buffer
  static constexpr size_t SMEM = sizeof(V2f) * ((size_t)N + (N / 2 + 1) + (size_t)N + (size_t)F * TPAD) +
                                 sizeof(float) * (size_t)N;
};

template <int LOGN>
__global__ void __launch_bounds__(ColRegPlan<LOGN>::THREADS) k_col_solve_reg(int dct, const V2f* twN, const float* tab,
                                                                             const float* lam, float kappa, float* spec,
                                                                             const V2f* rowinfo, const int* skip) {
  using P = ColRegPlan<LOGN>;
  constexpr int N = P::N, A = P::A, B = P::B, Q = A / B;
  extern __shared__ unsigned char smem_raw[];
  V2f* sTw = (V2f*)smem_raw;            // e^{-2 pi i m / N}, m < N
  V2f* sRow = sTw + N;                  // rows' box-data pairs (w, e), NaN in w for written rows
  V2f* sCs = sRow + N;                  // (cos, sin)(pi m / (2N)), m <= N/2
  V2f* sX = sCs + (N / 2 + 1);          // transpose buffers, TPAD per column pair
  float* sLam = (float*)(sX + P::F * P::TPAD);
  const int f = (int)threadIdx.x / B;   // column pair of this lane group
  const int t = (int)threadIdx.x % B;   // lane within the group
  const int k0 = (blockIdx.x * P::F + f) * 2;
  V2f* S = sX + f * P::TPAD;
  // tables fixed with the context, before the wait for the previous kernel
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    sTw[i] = twN[i];
    sLam[i] = lam[i];
  }
  for (int m = threadIdx.x; m <= N / 2; m += blockDim.x) dct_cs<float>(tab, N, m, sCs[m].x, sCs[m].y);
  // rows the row transform left out: w S_k(0) + e S_k(N-1) for this lane's two columns
  V2f s0 = {0.f, 0.f}, sN = {0.f, 0.f};
  if (rowinfo != nullptr) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int k = k0 + c;
      float a, b;
      if (dct) {
        a = tsin(tab, k + N, N, qscale(N));
        b = tsin(tab, k * (2 * N - 1) + N, N, qscale(N));
      } else {
        a = tsin(tab, k + 1, N, qscale(N));
        b = tsin(tab, (k + 1) * (2 * N - 1), N, qscale(N));
      }
      if (c == 0) { s0.x = a; sN.x = b; } else { s0.y = a; sN.y = b; }
    }
  }
  pdl_wait();
  if (*skip) return;
  // the lane's points v[t + B a], a < A: all loads in flight, then the row pairs staged
  V2f x[A];
#pragma unroll
  for (int a = 0; a < A; ++a) {
    const int j = mk_row(t + B * a, N);
    x[a] = *(const V2f*)(spec + (long)j * N + k0);
  }
  if (rowinfo != nullptr)
    for (int i = threadIdx.x; i < N; i += blockDim.x) sRow[i] = rowinfo[i];
  __syncthreads();
#pragma unroll
  for (int a = 0; a < A; ++a) {
    const int j = mk_row(t + B * a, N);
    V2f v = x[a];
    if (rowinfo != nullptr) {
      const V2f r = sRow[j];
      if (r.x == r.x) v = V2f{r.x * s0.x + r.y * sN.x, r.x * s0.y + r.y * sN.y};
    }
    if (!dct && (j & 1)) v = V2f{-v.x, -v.y};
    x[a] = v;
  }
  // ---- forward FFT: A-point DFTs, twiddle, transpose, B-point DFTs
  rg_dft<A, false>(x);
#pragma unroll
  for (int k1 = 1; k1 < A; ++k1) x[k1] = cmul(x[k1], sTw[(t * k1) & (N - 1)]);
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) S[k1 * (B + 1) + t] = x[k1];
  __syncwarp();
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int b = 0; b < B; ++b) x[q * B + b] = S[(t + B * q) * (B + 1) + b];
  rg_dft_each<B, false, A>(x, std::make_integer_sequence<int, Q>{});
  // lane t now holds X[m], m = (t + B q) + A k2, at register q B + k2
  // ---- bins N - m from the partner lane (B - t) mod B: register A - 1 - r there (lane 0 pairs
  // within itself)
  V2f z[A];
  const int src = (B - t) & (B - 1);
#pragma unroll
  for (int r = 0; r < A; ++r) {
    V2f v;
    v.x = __shfl_sync(0xffffffffu, x[A - 1 - r].x, src, B);
    v.y = __shfl_sync(0xffffffffu, x[A - 1 - r].y, src, B);
    const int r0 = r < B ? ((B - r) & (B - 1)) : (A - 1 - r + B);
    z[r] = t == 0 ? x[r0] : v;
  }
  // ---- DCT post-processing, eigenvalue division, pre-processing of the inverse, per bin
  const float lx0 = sLam[k0] - kappa, lx1 = sLam[k0 + 1] - kappa;
  constexpr int half = N / 2;
#pragma unroll
  for (int r = 0; r < A; ++r) {
    const int m = (t + B * (r / B)) + A * (r % B);
    const bool lo = m <= half;
    const int mm = lo ? m : N - m;          // the bin the post-processing is written for
    const V2f Zm = lo ? x[r] : z[r];        // Z[mm]
    const V2f ZNm = lo ? z[r] : x[r];       // Z[N - mm]
    const V2f cs = sCs[mm];
    V2f Xm, XNm;
    {
      const V2f Va{0.5f * (Zm.x + ZNm.x), 0.5f * (Zm.y - ZNm.y)};
      const V2f Vb{0.5f * (Zm.y + ZNm.y), -0.5f * (Zm.x - ZNm.x)};
      Xm = V2f{cs.x * Va.x + cs.y * Va.y, cs.x * Vb.x + cs.y * Vb.y};
      XNm = V2f{cs.y * Va.x - cs.x * Va.y, cs.y * Vb.x - cs.x * Vb.y};
    }
    const int l1 = dct ? mm : N - 1 - mm;
    const float ly = sLam[l1];
    V2f Gm{__fdividef(Xm.x, ly + lx0), __fdividef(Xm.y, ly + lx1)};
    V2f GNm{0.f, 0.f};
    if (mm == half) {
      GNm = Gm;
    } else if (mm > 0) {
      const float ly2 = sLam[dct ? N - mm : mm - 1];
      GNm = V2f{__fdividef(XNm.x, ly2 + lx0), __fdividef(XNm.y, ly2 + lx1)};
    }
    V2f Zo, ZNo;
    dct_pre<float>(N, mm, cs.x, cs.y, Gm, GNm, Zo, ZNo);
    z[r] = lo ? Zo : ZNo;
  }
  // ---- inverse FFT: B-point DFTs, twiddle, transpose, A-point DFTs
  rg_dft_each<B, true, A>(z, std::make_integer_sequence<int, Q>{});
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int n1 = 1; n1 < B; ++n1) {
      const V2f w = sTw[((t + B * q) * n1) & (N - 1)];
      z[q * B + n1] = cmul(z[q * B + n1], V2f{w.x, -w.y});
    }
  __syncwarp();  // the forward transpose's reads are complete
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int n1 = 0; n1 < B; ++n1) S[n1 * (A + 1) + t + B * q] = z[q * B + n1];
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) z[k1] = S[t * (A + 1) + k1];
  rg_dft<A, true>(z);
  // lane t holds v'[t + B n2] at register n2: back to the rows, scaled by 1/N
  constexpr float invN = 1.0f / (float)N;
#pragma unroll
  for (int a = 0; a < A; ++a) {
    const int j = mk_row(t + B * a, N);
    float s = invN;
    if (!dct && (j & 1)) s = -s;
    *(float2*)(spec + (long)j * N + k0) = make_float2(z[a].x * s, z[a].y * s);
  }
}

using ColRegKernel = void (*)(int, const V2f*, const float*, const float*, float, float*, const V2f*, const int*);
// the register column kernel and its launch shape for N = 2^logN, 16 <= N <= 1024
static ColRegKernel col_reg_kernel(int logN, int* threads, int* pairs, size_t* smem) {
  switch (logN) {
#define KFBI_COLREG(L)                     \
  case L:                                  \
    *threads = ColRegPlan<L>::THREADS;     \
    *pairs = ColRegPlan<L>::F;             \
    *smem = ColRegPlan<L>::SMEM;           \
    return k_col_solve_reg<L>;
    KFBI_COLREG(4)
    KFBI_COLREG(5)
    KFBI_COLREG(6)
    KFBI_COLREG(7)
    KFBI_COLREG(8)
    KFBI_COLREG(9)
    KFBI_COLREG(10)
#undef KFBI_COLREG
    default:
      return nullptr;
  }
}

// Probe values: inverse transform along x evaluated only at the interpolation points,
//   u[j][i] = (2/N) sum_k w_k spec[j][k] sin(pi (k+1)(2i+1)/(2N)), w_{N-1} = 1/2  (DST-III)
//   u[j][i] = (2/N) sum_k w_k spec[j][k] cos(pi k (2i+1)/(2N)), w_0 = 1/2        (DCT-III)
// one warp per probe q (row probe_j[q], column probe_i[q]): lane l sums the modes
// 4 l + 128 t + c (c < 4) read straight from the spectral grid (L2-resident after the column
// solve), so that every warp has the same work however the probes fall in the rows.
template <typename T>
__global__ void __launch_bounds__(256, 4) k_probe_values(int N, int dct, const int* nprobe, const int* probe_j,
                                                         const int* probe_i,
                               const T* spec, const T* tab, float scale, T* pval, const int* skip) {
  // the probe count is on the device (the grid covers 6 n, the most an interface can have)
  const int n_probe = *nprobe;
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  // the probe's position (set with the interface) before the wait
  int j = 0, i = 0;
  if (q < n_probe) {
    j = probe_j[q];
    i = probe_i[q];
  }
  pdl_wait();
  if (*skip || q >= n_probe) return;
  const int mask = 4 * N - 1, m = 2 * i + 1;
  const T* row = spec + (long)j * N;
  const int step = (128 * m) & mask;
  int idx = dct ? ((4 * lane * m + N) & mask) : (((4 * lane + 1) * m) & mask);
  T acc[4] = {0, 0, 0, 0};
#pragma unroll 8  // all eight 16-byte row loads of a lane in flight at N = 1024
  for (int k0 = 4 * lane; k0 < N; k0 += 128) {
    T v[4];
    if constexpr (sizeof(T) == 4) {
      const float4 f = *(const float4*)(row + k0);
      v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) v[c] = row[k0 + c];
    }
    if (dct && k0 == 0) v[0] *= (T)0.5;
    if (!dct && k0 + 4 == N) v[3] *= (T)0.5;
    int id = idx;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      acc[c] += v[c] * tsin(tab, id, N, scale);
      id = (id + m) & mask;
    }
    idx = (idx + step) & mask;
  }
  const T s = wsum((acc[0] + acc[1]) + (acc[2] + acc[3]));
  if (lane == 0) pval[q] = s * ((T)2 / (T)N);
}

// Dense transforms along x of row pairs (grid output and the plain box solve).
// inverse = 0, forward: spec[j][.] = DST-II/DCT-II of rhs[j][.] (rhs float64 or float32, mode
// order); inverse = 1: out[j][.] = exact inverse of spec[j][.] (out float64); inverse = 2: the
// inverse added to out[j][.] (a correction of the mixed-precision grid solve).
template <typename X>
struct NoDeduce {
  using type = X;
};
// the body of k_row_dense; CT > 0: N = 2^CT at compile time (constant index arithmetic and the
// compile-time Stockham stages of fft_ct), CT = 0: N at run time
template <typename T, typename In, int CT>
__device__ __forceinline__ void row_dense_body(int N, int logN, int dct, int inverse, const V2<T>* tw, const T* tab,
                                               const In* rhs, T* spec, double* out) {
  extern __shared__ unsigned char smem_raw[];
  V2<T>* A = (V2<T>*)smem_raw;
  V2<T>* B = A + N;
  const int j0 = 2 * blockIdx.x;  // rows j0 (real part), j0 + 1 (imaginary part)
  const int half = N >> 1;
  if (!inverse) {
    for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
      int r = t / N, i = t - r * N;
      T v = (T)rhs[(long)(j0 + r) * N + i];
      if (!dct && (i & 1)) v = -v;
      ((T*)&A[mk_pos(i, N)])[r] = v;
    }
    __syncthreads();
    V2<T>* X;
    if constexpr (CT > 0)
      X = fft_ct<T, CT, false>(A, B, 1, tw);
    else
      X = fft_stockham<T>(A, B, 1, N, logN, tw, false);
    for (int m = threadIdx.x; m <= half; m += blockDim.x) {
      V2<T> Xm, XNm;
      T cm, sm;
    dct_cs<T>(tab, N, m, cm, sm);
    dct_post<T>(X, N, m, cm, sm, Xm, XNm);
      int km = dct ? m : N - 1 - m;
      spec[(long)j0 * N + km] = Xm.x;
      spec[(long)(j0 + 1) * N + km] = Xm.y;
      if (m > 0 && m < half) {
        int kNm = dct ? N - m : m - 1;
        spec[(long)j0 * N + kNm] = XNm.x;
        spec[(long)(j0 + 1) * N + kNm] = XNm.y;
      }
    }
  } else {
    for (int m = threadIdx.x; m <= half; m += blockDim.x) {
      int km = dct ? m : N - 1 - m;
      V2<T> Gm{spec[(long)j0 * N + km], spec[(long)(j0 + 1) * N + km]};
      V2<T> GNm{0, 0};
      if (m == half) {
        GNm = Gm;
      } else if (m > 0) {
        int kNm = dct ? N - m : m - 1;
        GNm = V2<T>{spec[(long)j0 * N + kNm], spec[(long)(j0 + 1) * N + kNm]};
      }
      V2<T> Zm, ZNm;
      T cm, sm;
      dct_cs<T>(tab, N, m, cm, sm);
      dct_pre<T>(N, m, cm, sm, Gm, GNm, Zm, ZNm);
      A[m] = Zm;
      if (m > 0 && m < half) A[N - m] = ZNm;
    }
    __syncthreads();
    V2<T>* Z;
    if constexpr (CT > 0)
      Z = fft_ct<T, CT, true>(A, B, 1, tw);
    else
      Z = fft_stockham<T>(A, B, 1, N, logN, tw, true);
    const T invN = (T)1 / (T)N;
    for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
      int r = t / N, i = t - r * N;
      T v = ((const T*)&Z[mk_pos(i, N)])[r] * invN;
      if (!dct && (i & 1)) v = -v;
      const long o = (long)(j0 + r) * N + i;
      if (inverse == 2)
        out[o] += (double)v;
      else
        out[o] = (double)v;
    }
  }
}
template <typename T, typename In = double>
__global__ void k_row_dense(int N, int logN, int dct, int inverse, const V2<T>* tw, const T* tab,
                            const typename NoDeduce<In>::type* rhs, T* spec, double* out) {
  row_dense_body<T, In, 0>(N, logN, dct, inverse, tw, tab, rhs, spec, out);
}
// the same for N = 2^LOGN fixed at compile time (the float32 dense transforms of the mixed grid
// solves and grid outputs)
template <typename T, typename In, int LOGN>
__global__ void __launch_bounds__(512) k_row_dense_ct(int dct, int inverse, const V2<T>* tw, const T* tab,
                                                      const typename NoDeduce<In>::type* rhs, T* spec, double* out) {
  row_dense_body<T, In, LOGN>(1 << LOGN, LOGN, dct, inverse, tw, tab, rhs, spec, out);
}
template <typename T, typename In>
using RowDenseCt = void (*)(int, int, const V2<T>*, const T*, const In*, T*, double*);
template <typename T, typename In>
static RowDenseCt<T, In> row_dense_ct(int logN) {
  switch (logN) {
    case 4: return k_row_dense_ct<T, In, 4>;
    case 5: return k_row_dense_ct<T, In, 5>;
    case 6: return k_row_dense_ct<T, In, 6>;
    case 7: return k_row_dense_ct<T, In, 7>;
    case 8: return k_row_dense_ct<T, In, 8>;
    case 9: return k_row_dense_ct<T, In, 9>;
    case 10: return k_row_dense_ct<T, In, 10>;
    case 11: return k_row_dense_ct<T, In, 11>;
    case 12: return k_row_dense_ct<T, In, 12>;
    default: return nullptr;
  }
}

// --------------------------------------------------------------------------- interpolation
// Per node (Sec. 4.3): b_m = u(q_m) + [q_m in Omega-] C(q_m), v+ = r0.b, grad v+ = (r1.b, r2.b);
// value (v+ + v-)/2 = v+ - [v]/2; dnormal = n.(grad v+ - [grad v]/2). One warp per node,
// lane m < 6 handles stencil point m. The result is written as
//   out = a x + b value + c int(x) ds   (a, b, c select the boundary integral operator)
// in the arithmetic type T (a = eps_v[p] when eps_v is given) and stored as float64.
template <typename T, typename S_t>
__global__ void k_interp(int n, const S_t* st, const T* pval, const T* Jall, const int* ncr, const T* x_in,
                         const double* eps_v, T ca, T cb, T cc, const T* dint, double* out, double* dnormal,
                         const int* skip) {
  int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  // this lane's stencil point (set with the interface) before the wait
  const int m = lane;
  int probe = 0, minus = 0;
  T dx = 0, dy = 0, r0 = 0, r1 = 0, r2 = 0, nx = 0, ny = 0;
  if (p < n) {
    const S_t& S = st[p];
    if (m < 6) {
      probe = S.probe[m];
      minus = S.minus[m];
      dx = (T)S.dx[m];
      dy = (T)S.dy[m];
      r0 = (T)S.r0[m];
      r1 = (T)S.r1[m];
      r2 = (T)S.r2[m];
    }
    if (m == 0) {
      nx = (T)S.nx;
      ny = (T)S.ny;
    }
  }
  pdl_wait();
  if (*skip) return;
  if (p >= n) return;
  // the nodes' jumps follow the crossings' (their count is on the device)
  const T* J = Jall ? Jall + ((long)*ncr + p) * 6 : nullptr;
  T v = 0, gx = 0, gy = 0;
  if (m < 6) {
    T u = pval[probe];
    if (J != nullptr && minus) {
      u += J[0] + dx * J[1] + dy * J[2] + (T)0.5 * dx * dx * J[3] + dx * dy * J[5] + (T)0.5 * dy * dy * J[4];
    }
    v = r0 * u;
    gx = r1 * u;
    gy = r2 * u;
  }
  for (int o = 4; o > 0; o >>= 1) {
    v += __shfl_down_sync(0xffffffffu, v, o);
    gx += __shfl_down_sync(0xffffffffu, gx, o);
    gy += __shfl_down_sync(0xffffffffu, gy, o);
  }
  if (lane != 0) return;
  if (J != nullptr) {
    v -= (T)0.5 * J[0];
    gx -= (T)0.5 * J[1];
    gy -= (T)0.5 * J[2];
  }
  // explicit fused multiply-adds: the Gram-Schmidt kernel that forms these values itself
  // (interp_finish) rounds them in the same order, independent of compiler contraction
  T o = cb * v;
  if (x_in != nullptr) o = fma(eps_v != nullptr ? (T)eps_v[p] : ca, x_in[p], o);
  if (dint != nullptr) o = fma(cc, *dint, o);
  out[p] = (double)o;
  if (dnormal != nullptr) dnormal[p] = (double)(nx * gx + ny * gy);
}

// --------------------------------------------------------------------------- host side
// shared memory of k_col_solve: two P x N complex buffers, the staged twiddles (<= N) and, in
// float32, the N/2 + 1 rotations of the DCT pre/post-processing and the N eigenvalues (float64
// reads those two from global memory: it is bound by its float64 arithmetic, and N = 4096
// would not fit)
template <typename T>
static size_t col_smem(int N, int P) {
  size_t b = 2 * sizeof(V2<T>) * (size_t)P * N + sizeof(V2<T>) * (size_t)N;
  if (sizeof(T) == 4) b += sizeof(V2<T>) * (size_t)(N / 2 + 1) + sizeof(T) * (size_t)N;
  return b;
}

// largest column-pair count whose buffers fit the shared-memory budget
constexpr size_t COL_SMEM_MAX = 200 * 1024;
template <typename T>
static int col_pairs_max(int N) {
  int P = 4;
  while (P > 1 && (2 * P > N || col_smem<T>(N, P) > COL_SMEM_MAX)) P /= 2;
  return P;
}

// column pairs per block: float64 1, float32 2 unless overridden (kfbi_set_option)
template <typename T>
static int col_pairs(int N, int override_P = 0) {
  int P = sizeof(T) == 8 ? 1 : (override_P > 0 ? override_P : 2);
  const int pm = col_pairs_max<T>(N);
  if (P > pm) P = pm;
  while (2 * P > N) P /= 2;
  return P < 1 ? 1 : P;
}

// one radix-4 item per thread and stage: P N / 4 threads (at least a warp, at most 1024)
static int col_threads(int N, int P) {
  int t = P * N / 4;
  return t < 32 ? 32 : (t > 1024 ? 1024 : t);
}

// Matrices of the tensor-core column solve: forward F[l][j] = sin(pi (l+1)(2j+1) / (2N)) (DST-II)
// or cos(pi l (2j+1) / (2N)) (DCT-II), and its exact inverse G[j][l] = (2/N) w_l F[l][j] with
// w = 1/2 at l = N-1 (DST-III) or l = 0 (DCT-III), else 1; formed in float64, stored in float32.
__global__ void k_col_tc_mats(int N, int dct, float* F, float* G) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * N) return;
  const int l = t / N, j = t - l * N;
  const double arg = (double)(dct ? l : l + 1) * (double)(2 * j + 1) / (2.0 * N);
  const double v = dct ? cospi(arg) : sinpi(arg);
  const double w = (dct ? l == 0 : l == N - 1) ? 0.5 : 1.0;
  F[(long)l * N + j] = (float)v;
  G[(long)j * N + l] = (float)(2.0 / N * w * v);
}

kfbi_status col_tc_setup(kfbi_ctx* c) {
  if (c->col_fwd != nullptr) return KFBI_OK;
  const int N = c->N;
  const size_t NN = (size_t)N * N;
  KFBI_TRY(cudaMalloc((void**)&c->col_fwd, sizeof(float) * NN));
  KFBI_TRY(cudaMalloc((void**)&c->col_inv, sizeof(float) * NN));
  KFBI_TRY(cudaMalloc((void**)&c->col_tmp, sizeof(float) * NN));
  KFBI_TRY(cudaMalloc((void**)&c->col_tc_err, sizeof(int)));
  KFBI_TRY(cudaMemsetAsync(c->col_tc_err, 0, sizeof(int), c->stream));
  k_col_tc_mats<<<cdiv((long)NN, 256), 256, 0, c->stream>>>(N, c->boxbc == KFBI_BOX_NEUMANN0, c->col_fwd,
                                                            c->col_inv);
  KFBI_TRY(cudaGetLastError());
  KFBI_TRY(cudaStreamSynchronize(c->stream));
  return KFBI_OK;
}

// the column solve as two tensor-core contractions: tmp = (F spec) / (lam_y(l) + lam_x(k) - kappa),
// spec = G tmp (spec[j][k]: row j, column k; B(n = k, k = j) = spec[j][k]), both operands in three
// bfloat16 terms (six products each)
static kfbi_status launch_col_tc(kfbi_ctx* c, float* spec) {
  const int N = c->N;
  TcGemmArgs g;
  g.terms = 6;  // float32-level products: the column solve feeds the float32 inner applies
  g.error = c->col_tc_err;
  g.bn = 32;    // 32-column tiles: N / 32 CTAs per 128-row tile instead of one
  g.A = c->col_fwd;
  g.lda = N;
  g.B = spec;
  g.ldb = N;
  g.transB = 1;
  g.C = c->col_tmp;
  g.ldc = N;
  g.M = N;
  g.N = N;
  g.K = N;
  g.mode = TC_EIGEN;
  g.dm = c->lam_f;
  g.dn = c->lam_f;
  g.shift = (float)(-c->kappa);
  KFBI_CHECK(tc_gemm(g, c->stream));
  g.A = c->col_inv;
  g.B = c->col_tmp;
  g.C = spec;
  g.mode = TC_STORE;
  KFBI_CHECK(tc_gemm(g, c->stream));
  return KFBI_OK;
}

// the column solve runs the register-resident radix-16 kernel (kfbi_colfft.cu) unless a
// tensor-core, four-step register or radix-4 form is selected, or N < 32
template <typename T>
static bool col_uses_fft16(const kfbi_ctx* c) {
  if (!col_fft_supported(c->logN, sizeof(T) == 4)) return false;
  if (sizeof(T) == 4) return !c->col_tc && !c->col_reg && (c->col_radix4 & 1) == 0;
  return (c->col_radix4 & 2) == 0;
}

template <typename T>
static kfbi_status launch_col_solve(kfbi_ctx* c, T* spec, const V2<T>* rowinfo, const int* skip,
                                    const RowSrc* rows = nullptr) {
  const int N = c->N;
  const bool rec = c->timing && !c->capturing && c->timing_used < TIMING_CAP;
  if (rec) KFBI_TRY(cudaEventRecord(c->tev[2 * c->timing_used], c->stream));
  int rthreads = 0, rpairs = 0;
  size_t rsmem = 0;
  ColRegKernel rk = nullptr;
  bool tcp = false;
  if constexpr (sizeof(T) == 4) {
    tcp = c->col_tc && c->col_fwd != nullptr;
    if (!tcp && c->col_reg) rk = col_reg_kernel(c->logN, &rthreads, &rpairs, &rsmem);
  }
  if (tcp) {
    KFBI_CHECK(launch_col_tc(c, (float*)spec));
    launched(c, 1);  // two launches: one more than the single column kernel counted below
  } else if (col_uses_fft16<T>(c)) {
    KFBI_CHECK(col_fft_launch(c, sizeof(T) == 4, spec, rowinfo, skip, c->use_pdl && !rec, rows));
  } else if (rk != nullptr) {
    KFBI_TRY(launch_k(c->use_pdl && !rec, rk, dim3(N / (2 * rpairs)), dim3(rthreads), rsmem, c->stream,
                      (int)(c->boxbc == KFBI_BOX_NEUMANN0), (const V2f*)Tabs<float>::twN(c), Tabs<float>::sin(c),
                      Tabs<float>::lam(c), (float)c->kappa, (float*)spec, (const V2f*)rowinfo, skip));
  } else {
    const int P = col_pairs<T>(N, c->col_P);
    size_t smem = col_smem<T>(N, P);
    KFBI_TRY(launch_k(c->use_pdl && !rec, col_kernel<T>(c->logN), dim3(N / (2 * P)), dim3(col_threads(N, P)), smem,
                      c->stream, N, c->logN, P, (int)(c->boxbc == KFBI_BOX_NEUMANN0), Tabs<T>::stw(c), Tabs<T>::sin(c),
                      Tabs<T>::lam(c), (T)c->kappa, spec, sizeof(T) == 8 ? (const T*)c->rinv : nullptr, rowinfo, skip));
  }
  launched(c, 1);
  if (rec) {
    KFBI_TRY(cudaEventRecord(c->tev[2 * c->timing_used + 1], c->stream));
    c->tprec[c->timing_used] = sizeof(T) == 4 ? 1 : 0;
    c->timing_used += 1;
  }
  return KFBI_OK;
}

// back-to-back column solves on the context's spectral grid (see kfbi_time_column)
static kfbi_status time_column(kfbi_ctx* c, bool fp32, int reps, double* us) {
  const auto one = [&]() -> kfbi_status {
    if (fp32) {
      const V2<float>* ri = !c->col_tc ? (const V2<float>*)c->rowinfo : nullptr;
      return launch_col_solve<float>(c, (float*)c->spec, ri, c->zero_flag);
    }
    const V2<double>* ri = col_uses_fft16<double>(c) ? (const V2<double>*)c->rowinfo : nullptr;
    return launch_col_solve<double>(c, c->spec, ri, c->zero_flag);
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  KFBI_TRY(cudaEventCreate(&e0));
  kfbi_status st = cudaEventCreate(&e1) == cudaSuccess ? KFBI_OK : KFBI_ERR_CUDA;
  if (st == KFBI_OK) st = one();  // warm-up: tables and grid in L2
  if (st == KFBI_OK && cudaEventRecord(e0, c->stream) != cudaSuccess) st = KFBI_ERR_CUDA;
  for (int i = 0; i < reps && st == KFBI_OK; ++i) st = one();
  if (st == KFBI_OK && cudaEventRecord(e1, c->stream) != cudaSuccess) st = KFBI_ERR_CUDA;
  float ms = 0.f;
  if (st == KFBI_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
    st = KFBI_ERR_CUDA;
  if (st == KFBI_OK) *us = 1e3 * (double)ms / reps;
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return st;
}

template <typename T, typename In = double>
static kfbi_status launch_row_dense(kfbi_ctx* c, int inverse, const typename NoDeduce<In>::type* rhs, T* spec,
                                    double* out) {
  const int N = c->N;
  size_t smem = 2 * sizeof(V2<T>) * (size_t)N;
  // float32: 512 threads per row pair (16 warps of latency hiding per block; 256 measured 3 %
  // slower on the Stefan 4096^2 step)
  if constexpr (sizeof(T) == 4) {
    const RowDenseCt<T, In> k = row_dense_ct<T, In>(c->logN);
    if (k != nullptr) {
      k<<<N / 2, 512, smem, c->stream>>>(c->boxbc == KFBI_BOX_NEUMANN0, inverse, Tabs<T>::stw(c), Tabs<T>::sin(c), rhs,
                                         spec, out);
      launched(c, 1);
      return KFBI_OK;
    }
  }
  k_row_dense<T, In><<<N / 2, sizeof(T) == 4 ? 512 : 256, smem, c->stream>>>(N, c->logN, c->boxbc == KFBI_BOX_NEUMANN0, inverse,
                                                     Tabs<T>::stw(c), Tabs<T>::sin(c), rhs, spec, out);
  launched(c, 1);
  return KFBI_OK;
}

kfbi_status ir_solve_corrections(kfbi_ctx* c, const double* J, double* grid, int sweeps, const int* skip);
__global__ void k_gather_probes(int N, const int* prow_ptr, const int* probe_i, const double* grid, double* pval);

template <typename T>
static kfbi_status apply_t(kfbi_ctx* c, int layer, const double* density, double* values, double* dnormal,
                           double* grid, int bie_kind, const double* eps_v, const int* skip, const float* density_f,
                           bool skip_interp) {
  const long long l0 = c->launches;
  using T4 = typename std::conditional<sizeof(T) == 8, double4_32a, float4>::type;
  cudaStream_t s = c->stream;
  const int N = c->N, n = c->n;
  const int dct = c->boxbc == KFBI_BOX_NEUMANN0;
  const bool fs = c->boxbc == KFBI_BOX_FREESPACE_DL;
  const T* tab = Tabs<T>::sin(c);
  V2<T>* coef = (V2<T>*)c->dcoef;
  T* boxg = (T*)c->boxg;
  T* face = (T*)c->facespec;
  T* spec = (T*)c->spec;
  // rows without irregular nodes left to the column kernel: float32 applies, and float64
  // applies whose column solve is the radix-16 kernel (the tensor-core column solve reads
  // whole rows, so the row transform writes them all)
  V2<T>* rowinfo = ((sizeof(T) == 4 && !c->col_tc) || col_uses_fft16<T>(c)) ? (V2<T>*)c->rowinfo : nullptr;
  T* J = (T*)c->jumps;
  // the density integral of the Hele-Shaw operator, in the apply's type (float64 slot 0 or a
  // float32 slot in the same buffer)
  T* dint_t = sizeof(T) == 8 ? (T*)c->dint : (T*)(c->dint + 4);
  T* pval = (T*)c->probe_val;
  const int nk = n / 2 + 1;
  const bool want_int = bie_kind == KFBI_BIE_HS_EXTERIOR_MDL;
  const float scale = (float)(PI / (2.0 * N));
  // the density in the grid precision (float32 inner applies use the caller's float copy or
  // convert it here once)
  const T* dens_t;
  if (sizeof(T) == 4) {
    if (density_f == nullptr) {
      k_to_float<<<cdiv(n, 256), 256, 0, s>>>(density, c->dens_f, n, skip);
      launched(c, 1);
      density_f = c->dens_f;
    }
    dens_t = (const T*)density_f;
  } else {
    dens_t = (const T*)density;
  }
  // with the box table, its south and north rows hold the face rows' transforms (the box
  // product writes them to boxg[2N, 4N), which the row transform adds to rows 0 and N - 1)
  const bool face_from_table = fs && c->boxK_ok && c->use_boxK;
  if (face_from_table) face = boxg + 2 * N;
  if (fs) {
    // the box quadrature and its face transform depend only on the density: they run on the
    // side stream while the coefficients and jumps are formed, and join before the row transform
    cudaStream_t s2 = c->aux;
    KFBI_TRY(cudaEventRecord(c->ev_fork, s));
    KFBI_TRY(cudaStreamWaitEvent(s2, c->ev_fork, 0));
    const size_t smb = (size_t)n * sizeof(T4);
    const T bscale = (T)(-2.0 / (c->h * c->h * (double)n));
    if (face_from_table) {
      const T* Kt = sizeof(T) == 8 ? (const T*)c->boxK : (const T*)c->boxK_f;
      if (((uintptr_t)dens_t & (4 * sizeof(T) - 1)) == 0)
        k_box_gemv<T, true><<<cdiv((long)4 * N * 32, 256), 256, 0, s2>>>(Kt, box_ld(n), dens_t, n, 4 * N, boxg, skip);
      else
        k_box_gemv<T, false><<<cdiv((long)4 * N * 32, 256), 256, 0, s2>>>(Kt, box_ld(n), dens_t, n, 4 * N, boxg, skip);
    } else if (smb <= SMEM_STAGE_MAX)
      k_box_data<T, T4, true><<<cdiv((long)4 * N * 32, 256), 256, smb, s2>>>(
          dens_t, n, Tabs<T>::npack(c), N, c->xmin, c->xmax, c->ymin, c->ymax, c->h, bscale, boxg, skip);
    else
      k_box_data<T, T4, false><<<cdiv((long)4 * N * 32, 256), 256, 0, s2>>>(
          dens_t, n, Tabs<T>::npack(c), N, c->xmin, c->xmax, c->ymin, c->ymax, c->h, bscale, boxg, skip);
    if (!face_from_table) {
      size_t smf = 3 * sizeof(V2<T>) * (size_t)N;
      KFBI_TRY(launch_k(c->use_pdl, k_face_dst<T>, dim3(1), dim3(256), smf, s2, N, c->logN, dct, Tabs<T>::stw(c),
                        tab, (const T*)boxg, face, skip));
    }
    KFBI_TRY(cudaEventRecord(c->ev_join, s2));
    launched(c, face_from_table ? 1 : 2);
  }
  // launch shapes from capacities and device counts: the same launches serve every interface
  // of this layout (a captured graph is kept across interfaces)
  const int* d_ncr = c->seg_off + 2 * SUBSAMPLES * n;
  const int ntg_cap = c->ncr_grid + n;
  using G = typename std::remove_cv<typename std::remove_pointer<decltype(Tabs<T>::geo(c))>::type>::type;
  using SD = typename std::remove_cv<typename std::remove_pointer<decltype(Tabs<T>::stencil(c))>::type>::type;
  bool fused = false;
  // float32 with the jump kernel and the radix-16 column kernel: the jump kernel also writes
  // each crossed arm's correction and the column kernel forms the row transform itself (no
  // row-transform launch, no write and re-read of the spectral grid between them)
  bool rows_in_col = false;
  if constexpr (sizeof(T) == 4) {
    // float32, power-of-two n: coefficients and jumps in one kernel
    if (c->fuse_dft && n >= 16 && n <= 4096 && (n & (n - 1)) == 0) {
      rows_in_col = c->fuse_rows && col_uses_fft16<T>(c) && col_fft_rows_fit(c);
      const int logn = ilog2(n);
      KFBI_TRY(launch_k(c->use_pdl, k_jumps_fft<G, SD>, dim3(cdiv((long)ntg_cap * 32, JFFT_THREADS)),
                        dim3(JFFT_THREADS), jfft_smem(n, logn), s, (const float*)dens_t, n, logn, Tabs<T>::twn(c),
                        Tabs<T>::stencil(c), (float*)(want_int ? dint_t : nullptr), d_ncr, Tabs<T>::geo(c),
                        Tabs<T>::tstart(c), layer, (float)c->kappa, (float*)J, (const int*)c->arm_rev,
                        (const float2*)c->arm_coef, rows_in_col ? c->arm_slot : nullptr, skip));
      launched(c, 1);
      fused = true;
    }
  }
  if (!fused) {
    const size_t smd = (size_t)n * (sizeof(V2<T>) + sizeof(T));
    if (smd <= SMEM_STAGE_MAX) {
      KFBI_TRY(launch_k(c->use_pdl, k_dens_coef<T, true, SD>, dim3(cdiv((long)nk * 32, 256)), dim3(256), smd, s,
                        (const T*)dens_t, n, Tabs<T>::twn(c), Tabs<T>::stencil(c), (V2<T>*)coef,
                        (T*)(want_int ? dint_t : nullptr), skip));
    } else {
      k_dens_coef<T, false><<<cdiv((long)nk * 32, 256), 256, 0, s>>>(dens_t, n, Tabs<T>::twn(c), Tabs<T>::stencil(c),
                                                                     coef, want_int ? dint_t : nullptr, skip);
    }
    const size_t smj = (size_t)jump_layout_size(n) * sizeof(V2<T>);
    if (smj <= SMEM_STAGE_MAX)
      KFBI_TRY(launch_k(c->use_pdl, k_target_jumps<T, G, true>, dim3(cdiv((long)ntg_cap * 32, 256)), dim3(256), smj, s,
                        (const V2<T>*)coef, n, d_ncr, Tabs<T>::geo(c), Tabs<T>::tstart(c), layer, (T)c->kappa, J, skip));
    else
      KFBI_TRY(launch_k(c->use_pdl, k_target_jumps<T, G, false>, dim3(cdiv((long)ntg_cap * 32, 256)), dim3(256), 0, s,
                        (const V2<T>*)coef, n, d_ncr, Tabs<T>::geo(c), Tabs<T>::tstart(c), layer, (T)c->kappa, J, skip));
    launched(c, 2);
  }
  if (fs) KFBI_TRY(cudaStreamWaitEvent(s, c->ev_join, 0));
  // float64 applies of a mixed context on the largest grids (no box data): the grid solve by
  // float32 solves with float64 residual sweeps from the corrections at the irregular nodes,
  // and the probe values gathered from the solved grid
  bool ir_apply = false;
  if constexpr (sizeof(T) == 8) ir_apply = grid == nullptr && c->ir_grid != nullptr && c->grid_ir > 0;
  if (ir_apply) {
    const int sweeps = c->apply_sweeps > 0 ? c->apply_sweeps : c->grid_ir;
    KFBI_CHECK(ir_solve_corrections(c, (const double*)J, c->ir_grid, sweeps, skip));
    k_gather_probes<<<N, 128, 0, s>>>(N, c->prow_ptr, c->probe_i, c->ir_grid, (double*)pval);
    launched(c, 1);
  } else if (rows_in_col) {
    RowSrc rs;
    rs.row_ptr = c->row_ptr;
    rs.ci = c->irr_ci;
    rs.slot = (const float4*)c->arm_slot;
    rs.boxg = fs ? (const float*)boxg : nullptr;
    rs.face = fs ? (const float*)face : nullptr;
    KFBI_CHECK(launch_col_solve<T>(c, spec, nullptr, skip, &rs));
  } else {
    KFBI_TRY(launch_k(c->use_pdl, k_row_forward<T>, dim3(N), dim3(ROW_THREADS), 0, s, N, dct, (const int*)c->row_ptr,
                      (const IrrNode*)c->irr, (const T*)J, (T)(1.0 / (c->h * c->h)), (const T*)(fs ? boxg : nullptr),
                      (const T*)face, tab, scale, spec, rowinfo, skip));
    launched(c, 1);
    KFBI_CHECK(launch_col_solve<T>(c, spec, rowinfo, skip));
  }
  if (!ir_apply) {
    KFBI_TRY(launch_k(c->use_pdl, k_probe_values<T>, dim3(cdiv((long)6 * n * 32, 256)), dim3(256), 0, s, N, dct,
                      (const int*)(c->prow_ptr + N), (const int*)c->probe_j, (const int*)c->probe_i, (const T*)spec,
                      tab, scale, pval, skip));
    launched(c, 1);
  }
  if (grid != nullptr) KFBI_CHECK(launch_row_dense<T>(c, 1, nullptr, spec, grid));
  using S_t = typename std::remove_cv<typename std::remove_pointer<decltype(Tabs<T>::stencil(c))>::type>::type;
  T ca = 0, cb = 1, cc = 0;
  const double* ev = nullptr;
  const T* xin = nullptr;
  if (bie_kind == KFBI_BIE_INTERIOR_DL) { ca = (T)0.5; xin = dens_t; }
  else if (bie_kind == KFBI_BIE_HS_EXTERIOR_MDL) { ca = (T)-0.5; cc = 1; xin = dens_t; }
  else if (bie_kind == KFBI_BIE_STEFAN_SL) { cb = -1; ev = eps_v; xin = dens_t; }
  if (!skip_interp) {
    KFBI_TRY(launch_k(c->use_pdl, k_interp<T, S_t>, dim3(cdiv((long)n * 32, 256)), dim3(256), 0, s, n,
                      Tabs<T>::stencil(c), (const T*)pval, (const T*)J, d_ncr, xin, ev, ca, cb, cc,
                      (const T*)(want_int ? dint_t : nullptr), values, dnormal, skip));
    launched(c, 1);
  }
  c->per_apply_launches[sizeof(T) == 4 ? 1 : 0] = (int)(c->launches - l0);
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

// Shared-memory limits of the kernels whose dynamic shared memory may exceed 48 KB. The limit
// is a property of the kernel for the whole process, not of a context, so it is set to the
// largest size any context can launch with (grids up to 4096 cells, staged inputs up to
// SMEM_STAGE_MAX); a launch still reserves only the shared memory it asks for.
constexpr int MAX_GRID_N = 4096;
template <typename T>
static kfbi_status setup_t(kfbi_ctx*) {
  int col = 0;
  for (int N = 16; N <= MAX_GRID_N; N *= 2) {
    const int P = sizeof(T) == 8 ? 1 : col_pairs_max<T>(N);
    const int b = (int)col_smem<T>(N, P);
    col = b > col ? b : col;
  }
  const int row = (int)(3 * sizeof(V2<T>) * (size_t)MAX_GRID_N);  // k_face_dst: A, B, twiddles
  using T4 = typename std::conditional<sizeof(T) == 8, double4_32a, float4>::type;
  using G = typename std::remove_cv<typename std::remove_pointer<decltype(Tabs<T>::geo(nullptr))>::type>::type;
  using S_t = typename std::remove_cv<typename std::remove_pointer<decltype(Tabs<T>::stencil(nullptr))>::type>::type;
  const int stage = (int)SMEM_STAGE_MAX;
  for (int lg = 4; lg <= 12; ++lg)
    KFBI_TRY(cudaFuncSetAttribute(col_kernel<T>(lg), cudaFuncAttributeMaxDynamicSharedMemorySize, col));
  KFBI_TRY(cudaFuncSetAttribute(k_row_dense<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, row));
  if constexpr (sizeof(T) == 4) {  // the float32 residual input of the mixed grid solve
    KFBI_TRY((cudaFuncSetAttribute(k_row_dense<T, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, row)));
    for (int lg = 4; lg <= 12; ++lg) {
      KFBI_TRY((cudaFuncSetAttribute(row_dense_ct<T, double>(lg), cudaFuncAttributeMaxDynamicSharedMemorySize, row)));
      KFBI_TRY((cudaFuncSetAttribute(row_dense_ct<T, float>(lg), cudaFuncAttributeMaxDynamicSharedMemorySize, row)));
    }
  }
  KFBI_TRY(cudaFuncSetAttribute(k_face_dst<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, row));
  KFBI_TRY(cudaFuncSetAttribute(k_dens_coef<T, true, S_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, stage));
  KFBI_TRY(cudaFuncSetAttribute(k_box_data<T, T4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, stage));
  KFBI_TRY(cudaFuncSetAttribute(k_target_jumps<T, G, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, stage));
  if constexpr (sizeof(T) == 4) {
    KFBI_TRY(cudaFuncSetAttribute(k_jumps_fft<G, S_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, stage));
    for (int lg = 4; lg <= 10; ++lg) {
      int th = 0, pr = 0;
      size_t sm = 0;
      ColRegKernel rk = col_reg_kernel(lg, &th, &pr, &sm);
      KFBI_TRY(cudaFuncSetAttribute(rk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    }
  }
  return KFBI_OK;
}

kfbi_status apply_setup_attributes(kfbi_ctx* c) {
  KFBI_TRY(cudaFuncSetAttribute(k_box_face_table, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(3 * sizeof(V2<double>) * (size_t)MAX_GRID_N)));
  KFBI_CHECK(setup_t<double>(c));
  KFBI_CHECK(col_fft_setup_attributes());
  return setup_t<float>(c);
}

// bie_kind < 0: plain layer potential
kfbi_status apply_enqueue(kfbi_ctx* c, int layer, bool fp32, const double* density, double* values, double* dnormal,
                          double* grid, int bie_kind, const double* eps_v, const int* skip, const float* density_f,
                          bool skip_interp) {
  if (skip == nullptr) skip = c->zero_flag;
  if (fp32)
    return apply_t<float>(c, layer, density, values, dnormal, grid, bie_kind, eps_v, skip, density_f, skip_interp);
  return apply_t<double>(c, layer, density, values, dnormal, grid, bie_kind, eps_v, skip, nullptr, false);
}

InterpArgs<float> interp_args_f32(kfbi_ctx* c, int bie_kind, const double* eps_v, const float* density_f) {
  // the same choices as apply_t<float> makes for its k_interp launch
  InterpArgs<float> a;
  a.st = c->stencil_f;
  a.pval = (const float*)c->probe_val;
  a.Jall = (const float*)c->jumps;
  a.ncr = c->seg_off + 2 * SUBSAMPLES * c->n;
  a.dint = bie_kind == KFBI_BIE_HS_EXTERIOR_MDL ? (const float*)(c->dint + 4) : nullptr;
  if (bie_kind == KFBI_BIE_INTERIOR_DL) { a.ca = 0.5f; a.x_in = density_f; }
  else if (bie_kind == KFBI_BIE_HS_EXTERIOR_MDL) { a.ca = -0.5f; a.cc = 1.0f; a.x_in = density_f; }
  else if (bie_kind == KFBI_BIE_STEFAN_SL) { a.cb = -1.0f; a.eps_v = eps_v; a.x_in = density_f; }
  return a;
}

kfbi_status box_matrix_enqueue(kfbi_ctx* c, int n) {
  const int ld = box_ld(n);
  launched(c, 2);
  // on the aux stream after the node data: the applies' box products also run there (stream
  // order), graph launches and the next interface wait on ev_boxK (box_table_join)
  KFBI_TRY(cudaEventRecord(c->ev_boxK0, c->stream));
  KFBI_TRY(cudaStreamWaitEvent(c->aux, c->ev_boxK0, 0));
  const dim3 grid(cdiv(ld, 128), 4, cdiv(c->N, BOXK_CHUNK));
  k_box_matrix<<<grid, 128, 0, c->aux>>>(c->N, n, ld, (const double4_32a*)c->npack, c->xmin, c->xmax, c->ymin,
                                         c->ymax, c->h, -2.0 / (c->h * c->h * (double)n), c->boxK, c->boxK_f);
  k_box_face_table<<<n, 256, 3 * sizeof(V2<double>) * (size_t)c->N, c->aux>>>(
      c->N, c->logN, ld, Tabs<double>::stw(c), Tabs<double>::sin(c), c->boxK, c->boxK_f);
  KFBI_TRY(cudaGetLastError());
  KFBI_TRY(cudaEventRecord(c->ev_boxK, c->aux));
  c->boxK_pending = true;
  return KFBI_OK;
}

kfbi_status box_table_join(kfbi_ctx* c, cudaStream_t s) {
  if (!c->boxK_pending) return KFBI_OK;
  KFBI_TRY(cudaStreamWaitEvent(s, c->ev_boxK, 0));
  if (s == c->stream) c->boxK_pending = false;
  return KFBI_OK;
}

kfbi_status grid_solve_enqueue(kfbi_ctx* c, const double* rhs, double* u) {
  double* spec = c->spec;
  KFBI_CHECK(launch_row_dense<double>(c, 0, rhs, spec, nullptr));
  KFBI_CHECK(launch_col_solve<double>(c, spec, nullptr, c->zero_flag));
  KFBI_CHECK(launch_row_dense<double>(c, 1, nullptr, spec, u));
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

// r = rhs - (Delta_h - kappa) u, rounded to float32 (the right-hand side of a float32
// correction solve). Delta_h is the five-point Laplacian whose eigenvectors the solve's
// transforms are: cell-centred, with the ghost values of the box condition, u_{-1} = -u_0,
// u_N = -u_{N-1} (DST-II, Dirichlet) or u_{-1} = u_0, u_N = u_{N-1} (DCT-II, Neumann); the
// residual is formed in float64 (Sec. 4.2's operator; the refinement is not in the paper).
// f - (Delta_h - kappa) u at grid node (i, j) = f + (4 / h^2 + kappa) u_ij - (sum of the four
// neighbours) / h^2, d4 = 4 / h^2 + kappa (five float64 operations: on this part the float64
// rate, not memory, bounds a pass over the grid)
__device__ __forceinline__ double grid_resid_at(int N, int dct, double inv_h2, double d4, double f, const double* u,
                                                int i, int j) {
  const long idx = (long)j * N + i;
  const double c = u[idx];
  const double g = dct ? c : -c;  // ghost value across the box face
  const double w = i > 0 ? u[idx - 1] : g;
  const double e = i < N - 1 ? u[idx + 1] : g;
  const double so = j > 0 ? u[idx - N] : g;
  const double no = j < N - 1 ? u[idx + N] : g;
  return fma(-inv_h2, (w + e) + (so + no), fma(d4, c, f));
}
// one row per blockIdx.y; rhs = nullptr: a right-hand side that is zero here (the sparse
// corrections are put in by k_resid_fix)
__global__ void k_grid_resid(int N, int dct, double inv_h2, double d4, const double* rhs, const double* u, float* r) {
  const int j = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const long idx = (long)j * N + i;
  const double f = rhs != nullptr ? rhs[idx] : 0.0;
  r[idx] = (float)grid_resid_at(N, dct, inv_h2, d4, f, u, i, j);
}

// The corrected right-hand side of the apply's grid solve at each irregular node (the value
// k_row_forward transforms: sign / h^2 times the arms' J0 + d J1 + d^2 J2 / 2), with its grid
// index; one block per row.
__global__ void k_corr_nodes(int N, const int* row_ptr, const IrrNode* irr, const double* J, double inv_h2,
                             double* cval, int* cpos) {
  const int j = blockIdx.x;
  const int b = row_ptr[j], e = row_ptr[j + 1];
  for (int t = b + (int)threadIdx.x; t < e; t += blockDim.x) {
    const IrrRegs<double> node = irr_regs<double>(irr[t]);
    double sum = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int tg = node.tg[a];
      if (tg < 0) continue;
      const double* jj = J + (long)tg * 6;
      const double d = node.d[a];
      const double j1 = a < 2 ? jj[1] : jj[2];
      const double j2 = a < 2 ? jj[3] : jj[4];
      sum += jj[0] + d * j1 + 0.5 * d * d * j2;
    }
    cval[t] = node.sign * inv_h2 * sum;
    cpos[t] = j * N + node.i;
  }
}
// r[pos] = the correction (float32) at every irregular node (r zero elsewhere)
__global__ void k_corr_scatter(const int* nirr, const double* cval, const int* cpos, float* r) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < *nirr) r[cpos[q]] = (float)cval[q];
}
// the residual at the irregular nodes, where the right-hand side is the correction
__global__ void k_resid_fix(int N, int dct, double inv_h2, double d4, const int* nirr, const double* cval,
                            const int* cpos, const double* u, float* r) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= *nirr) return;
  const int pos = cpos[q], j = pos / N, i = pos - j * N;
  r[pos] = (float)grid_resid_at(N, dct, inv_h2, d4, cval[q], u, i, j);
}

// Mixed-precision box solve: u = (Delta_h - kappa)^{-1} rhs by a float32 solve (rows, columns,
// rows as in grid_solve_enqueue, float32 spectral grid and tables), then `sweeps` corrections:
// r = rhs - (Delta_h - kappa) u in float64, u += the float32 solve of r. The float32 grid and
// the residual share the float64 spectral buffer (N^2 floats each). rhs and u must not alias.
kfbi_status grid_solve_mixed_enqueue(kfbi_ctx* c, const double* rhs, double* u, int sweeps) {
  if (c->precision != KFBI_MIXED) return KFBI_ERR_ARG;
  const int N = c->N;
  const long NN = (long)N * N;
  float* specf = (float*)c->spec;
  float* r = specf + NN;
  KFBI_CHECK(launch_row_dense<float>(c, 0, rhs, specf, nullptr));
  KFBI_CHECK(launch_col_solve<float>(c, specf, nullptr, c->zero_flag));
  KFBI_CHECK(launch_row_dense<float>(c, 1, nullptr, specf, u));
  for (int sw = 0; sw < sweeps; ++sw) {
    const double inv_h2 = 1.0 / (c->h * c->h);
    k_grid_resid<<<dim3(cdiv(N, 256), N), 256, 0, c->stream>>>(N, c->boxbc == KFBI_BOX_NEUMANN0, inv_h2,
                                                               4.0 * inv_h2 + c->kappa, rhs, u, r);
    launched(c, 1);
    KFBI_CHECK((launch_row_dense<float, float>(c, 0, r, specf, nullptr)));
    KFBI_CHECK(launch_col_solve<float>(c, specf, nullptr, c->zero_flag));
    KFBI_CHECK(launch_row_dense<float>(c, 2, nullptr, specf, u));
  }
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

// Grid output of a layer potential (the apply's grid solve (Delta_h - kappa) u = C with the
// corrected right-hand side C of its float64 jumps, Sec. 4.2) for KFBI_MIXED contexts without
// box data: the float64 density coefficients and jumps, C at the irregular nodes (float64),
// then the mixed-precision box solve with C as a sparse right-hand side
// (ir_solve_corrections). The interface values of the apply are not formed.
kfbi_status apply_grid_mixed_enqueue(kfbi_ctx* c, int layer, const double* density, double* grid, int sweeps) {
  if (c->precision != KFBI_MIXED || c->boxbc == KFBI_BOX_FREESPACE_DL) return KFBI_ERR_ARG;
  using T = double;
  cudaStream_t s = c->stream;
  const int n = c->n, nk = n / 2 + 1;
  const int* skip = c->zero_flag;
  V2<T>* coef = (V2<T>*)c->dcoef;
  T* J = (T*)c->jumps;
  const int* d_ncr = c->seg_off + 2 * SUBSAMPLES * n;
  const int ntg_cap = c->ncr_grid + n;
  using G = typename std::remove_cv<typename std::remove_pointer<decltype(Tabs<T>::geo(c))>::type>::type;
  using SD = typename std::remove_cv<typename std::remove_pointer<decltype(Tabs<T>::stencil(c))>::type>::type;
  // the density's coefficients and the jumps at every target, as apply_t<double> forms them
  const size_t smd = (size_t)n * (sizeof(V2<T>) + sizeof(T));
  if (smd <= SMEM_STAGE_MAX)
    KFBI_TRY(launch_k(c->use_pdl, k_dens_coef<T, true, SD>, dim3(cdiv((long)nk * 32, 256)), dim3(256), smd, s,
                      density, n, Tabs<T>::twn(c), Tabs<T>::stencil(c), coef, (T*)nullptr, skip));
  else
    k_dens_coef<T, false><<<cdiv((long)nk * 32, 256), 256, 0, s>>>(density, n, Tabs<T>::twn(c), Tabs<T>::stencil(c),
                                                                   coef, nullptr, skip);
  const size_t smj = (size_t)jump_layout_size(n) * sizeof(V2<T>);
  if (smj <= SMEM_STAGE_MAX)
    KFBI_TRY(launch_k(c->use_pdl, k_target_jumps<T, G, true>, dim3(cdiv((long)ntg_cap * 32, 256)), dim3(256), smj, s,
                      (const V2<T>*)coef, n, d_ncr, Tabs<T>::geo(c), Tabs<T>::tstart(c), layer, (T)c->kappa, J, skip));
  else
    KFBI_TRY(launch_k(c->use_pdl, k_target_jumps<T, G, false>, dim3(cdiv((long)ntg_cap * 32, 256)), dim3(256), 0, s,
                      (const V2<T>*)coef, n, d_ncr, Tabs<T>::geo(c), Tabs<T>::tstart(c), layer, (T)c->kappa, J, skip));
  launched(c, 2);
  KFBI_CHECK(ir_solve_corrections(c, J, grid, sweeps, skip));
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

// The grid solve (Delta_h - kappa) u = C of an apply whose corrected right-hand side C is
// nonzero only at the irregular nodes (float64 jumps J, no box data), by mixed-precision
// refinement: C scattered (float32) into the residual buffer, u = its float32 solve, then
// `sweeps` times r = C - (Delta_h - kappa) u (float64; C put in at the irregular nodes by
// k_resid_fix), u += the float32 solve of r.
kfbi_status ir_solve_corrections(kfbi_ctx* c, const double* J, double* grid, int sweeps, const int* skip) {
  cudaStream_t s = c->stream;
  const int N = c->N;
  const long NN = (long)N * N;
  const int dct = c->boxbc == KFBI_BOX_NEUMANN0;
  const double inv_h2 = 1.0 / (c->h * c->h);
  float* specf = (float*)c->spec;
  float* r = specf + NN;
  const int* nirr = c->row_ptr + N;  // irregular-node count (device)
  const int qb = cdiv(c->cap_irr, 256);
  k_corr_nodes<<<N, ROW_THREADS, 0, s>>>(N, c->row_ptr, (const IrrNode*)c->irr, J, inv_h2, c->corr_val, c->corr_pos);
  KFBI_TRY(cudaMemsetAsync(r, 0, sizeof(float) * (size_t)NN, s));
  k_corr_scatter<<<qb, 256, 0, s>>>(nirr, c->corr_val, c->corr_pos, r);
  launched(c, 2);
  KFBI_CHECK((launch_row_dense<float, float>(c, 0, r, specf, nullptr)));
  KFBI_CHECK(launch_col_solve<float>(c, specf, nullptr, skip));
  KFBI_CHECK(launch_row_dense<float>(c, 1, nullptr, specf, grid));
  for (int sw = 0; sw < sweeps; ++sw) {
    const double d4 = 4.0 * inv_h2 + c->kappa;
    k_grid_resid<<<dim3(cdiv(N, 256), N), 256, 0, s>>>(N, dct, inv_h2, d4, nullptr, grid, r);
    k_resid_fix<<<qb, 256, 0, s>>>(N, dct, inv_h2, d4, nirr, c->corr_val, c->corr_pos, grid, r);
    launched(c, 2);
    KFBI_CHECK((launch_row_dense<float, float>(c, 0, r, specf, nullptr)));
    KFBI_CHECK(launch_col_solve<float>(c, specf, nullptr, skip));
    KFBI_CHECK(launch_row_dense<float>(c, 2, nullptr, specf, grid));
  }
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

// gather a dense grid at the probes, then interpolate with zero jumps
__global__ void k_gather_probes(int N, const int* prow_ptr, const int* probe_i, const double* grid, double* pval) {
  int j = blockIdx.x;
  int b = prow_ptr[j], e = prow_ptr[j + 1];
  for (int q = b + threadIdx.x; q < e; q += blockDim.x) pval[q] = grid[(long)j * N + probe_i[q]];
}

kfbi_status interp_grid_enqueue(kfbi_ctx* c, const double* grid, double* values) {
  cudaStream_t s = c->stream;
  double* pval = c->probe_val;
  launched(c, 2);
  k_gather_probes<<<c->N, 128, 0, s>>>(c->N, c->prow_ptr, c->probe_i, grid, pval);
  k_interp<double><<<cdiv((long)c->n * 32, 256), 256, 0, s>>>(c->n, c->stencil, pval, nullptr, nullptr, nullptr,
                                                               nullptr, 0.0, 1.0, 0.0, nullptr, values, nullptr,
                                                               c->zero_flag);
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

// --------------------------------------------------------------------------- allocation-free solve
// kfbi_grid_solve_noalloc: the plain box solve of kfbi_grid_solve for callers that cannot
// allocate device memory (see include/kfbi.h). Its scratch lives in one file-scope device
// array: one slot holding the column kernel's skip flag (cleared by every call before the
// kernel reads it), then the spectral grid (N^2), the sine table (4N), the eigenvalues (N) and
// the staged FFT twiddles (2N). Every call rewrites all of it before reading it. The array is shared
// by every call in the process.
constexpr int NOALLOC_MAX_N = 512;
constexpr size_t NOALLOC_HEAD = 32;  // doubles reserved for flags, keeps the grid 256-byte aligned
constexpr size_t NOALLOC_DOUBLES = NOALLOC_HEAD + (size_t)NOALLOC_MAX_N * NOALLOC_MAX_N + 8 * (size_t)NOALLOC_MAX_N;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

// staged Stockham twiddle t (layout of fft_stockham): w^{r jm N / (4 Ns)} = e^{-i pi r jm / (2 Ns)}
__device__ bool staged_twiddle(int N, int logN, int t, double* re, double* im) {
  int off = 0;
  for (int Ns = (logN & 1) ? 2 : 1; Ns < N; Ns <<= 2) {
    if (t < off + 3 * Ns) {
      int r = (t - off) / Ns + 1, jm = (t - off) % Ns;
      double sn, cs;
      sincospi((double)(r * jm) / (2.0 * Ns), &sn, &cs);
      *re = cs;
      *im = -sn;
      return true;
    }
    off += 3 * Ns;
  }
  return false;
}

__global__ void k_noalloc_tables(int N, int logN, double h, int neumann, double* tab, double* lam, double* tw,
                                 int* flag) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m == 0) *flag = 0;
  if (m < 4 * N) tab[m] = sinpi((double)m / (2.0 * N));
  if (m < N) {
    double sk = sinpi(((double)m + (neumann ? 0.0 : 1.0)) / (2.0 * N));
    lam[m] = -4.0 * sk * sk / (h * h);
    double re = 0.0, im = 0.0;
    staged_twiddle(N, logN, m, &re, &im);
    tw[2 * m] = re;
    tw[2 * m + 1] = im;
  }
}

// device address of the scratch array, looked up once per device (host code may not use the
// array's name as a device pointer)
static double* noalloc_scratch(kfbi_status* st) {
  static std::mutex mu;
  static double* addr[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    *st = KFBI_ERR_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      note_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
      *st = KFBI_ERR_CUDA;
      return nullptr;
    }
    addr[dev] = (double*)p;
  }
  *st = KFBI_OK;
  return addr[dev];
}

static kfbi_status grid_solve_noalloc_impl(int N, double h, double kappa, int boxbc, const double* rhs, double* u,
                                           cudaStream_t s) {
  kfbi_status st = KFBI_OK;
  double* base = noalloc_scratch(&st);
  if (st != KFBI_OK) return st;
  int* flag = (int*)base;
  double* spec = base + NOALLOC_HEAD;
  double* tab = spec + (size_t)N * N;
  double* lam = tab + 4 * (size_t)N;
  double* tw = lam + N;
  const int logN = ilog2(N);
  const int dct = boxbc == KFBI_BOX_NEUMANN0;
  k_noalloc_tables<<<cdiv(4L * N, 256), 256, 0, s>>>(N, logN, h, dct, tab, lam, tw, flag);
  size_t sm_row = 2 * sizeof(V2<double>) * N;  // <= 16 KB for N <= 512
  k_row_dense<double><<<N / 2, 256, sm_row, s>>>(N, logN, dct, 0, (const V2<double>*)tw, tab, rhs, spec, nullptr);
  const int P = col_pairs<double>(N);
  size_t sm_col = col_smem<double>(N, P);  // <= 28 KB for N <= 512
  col_kernel<double>(logN)<<<N / (2 * P), col_threads(N, P), sm_col, s>>>(N, logN, P, dct, (const V2<double>*)tw, tab, lam,
                                                                  kappa, spec, nullptr, nullptr, flag);
  k_row_dense<double><<<N / 2, 256, sm_row, s>>>(N, logN, dct, 1, (const V2<double>*)tw, tab, nullptr, spec, u);
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

}  // namespace kfbi

extern "C" kfbi_status kfbi_time_column(kfbi_ctx* c, int fp32, int reps, double* us_per_launch) {
  if (c == nullptr || us_per_launch == nullptr || reps < 1 || reps > 100000 || (fp32 != 0 && fp32 != 1))
    return KFBI_ERR_ARG;
  if (c->capturing) return KFBI_ERR_STATE;
  const bool tm = c->timing;
  c->timing = false;  // no per-launch events between the solves
  KFBI_TRY(kfbi::stream_enter(c));
  kfbi_status st = kfbi::time_column(c, fp32 != 0, reps, us_per_launch);
  c->timing = tm;
  KFBI_TRY(kfbi::stream_exit(c));
  return st;
}

extern "C" kfbi_status kfbi_grid_solve_noalloc(int N, double h, double kappa, int boxbc, const double* rhs, double* u,
                                               void* stream) {
  if (N < 16 || (N & (N - 1)) != 0 || rhs == nullptr || u == nullptr) return KFBI_ERR_ARG;
  if (N > kfbi::NOALLOC_MAX_N) return KFBI_ERR_CAPACITY;
  if (!(h > 0.0) || !(kappa >= 0.0) || boxbc < KFBI_BOX_DIRICHLET0 || boxbc > KFBI_BOX_FREESPACE_DL)
    return KFBI_ERR_ARG;
  if (boxbc == KFBI_BOX_NEUMANN0 && kappa == 0.0) return KFBI_ERR_SINGULAR;
  return kfbi::grid_solve_noalloc_impl(N, h, kappa, boxbc, rhs, u, (cudaStream_t)stream);
}
