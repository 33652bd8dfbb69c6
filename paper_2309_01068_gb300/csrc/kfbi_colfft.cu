// Column solve of the fast grid solver (Sec. 4.2: the 5-point operator is diagonal in the
// DST/DCT basis) with register-resident FFTs. For every column k of the spectral grid
// (x-mode k after the row transform): the DST-II (Dirichlet box) or DCT-II (Neumann box) along
// y, division by lam_y(l) + lam_x(k) - kappa, and the inverse transform, in place.
//
// Two real columns k, k + 1 form one complex sequence (Makhoul reordering: a DCT-II of length
// N is a complex FFT of length N plus a rotation of each bin pair m, N - m). Each column pair
// is owned by N/PT threads that hold PT points each (PT = 16, or 8 for twice the warps on
// grids up to 1024) through the whole solve:
//   stage 0      radix-PT DFT of points u + r N/PT, read straight from the grid rows
//   stages 1..   Stockham stages of radix PT (the last one of radix 2, 4 or 8) through one
//                padded shared-memory buffer per pair
//   last stage   its outputs, the bins j + r N/R, stay in registers; the thread's butterflies
//                are chosen so that it also holds every partner bin N - m, so the DCT post-
//                processing, the eigenvalue division and the pre-processing of the inverse
//                need no exchange
//   inverse      the adjoint of each stage in reverse order (inverse DFT, then the conjugate
//                twiddle, reading where the forward stage wrote and writing where it read),
//                ending in the rows of the grid.
// With 16 points, N = 1024 takes three stages (16, 16, 4): four shared-memory round trips and
// six barriers per solve, against ten radix-4 stages of the shared-memory Stockham kernel; with
// 8 points four stages (8, 8, 8, 2).
// FR (float32, 16 points): the kernel also forms its input rows from the irregular-node
// corrections instead of reading the row transform's output (KFBI_OPT_FUSE_ROWS).
#include <type_traits>
#include <utility>

#include "kfbi_dct.cuh"
#include "kfbi_internal.cuh"

namespace kfbi {
namespace {

// Stage plan for N = 2^LOGN, 5 <= LOGN <= 12, PT points per thread (16 or 8, B = log2 PT bits
// per full stage): stage 0 of radix PT, then stages of radix PT, and a last stage of radix 2^b
// with 1 <= b < B, so that every thread holds at least two last-stage butterflies; when the
// remaining bits are a multiple of B, one stage of radix PT/2 comes before a last stage of radix
// 2. PT = 16: N = 1024 is 16, 16, 4; PT = 8: 8, 8, 8, 2.
template <int LOGN, int PT = 16>
struct FPlan {
  static_assert(PT == 8 || PT == 16, "8 or 16 points per thread");
  static constexpr int N = 1 << LOGN;
  static constexpr int B = PT == 16 ? 4 : 3;
  static constexpr int TH = N / PT;  // threads per column pair
  static constexpr int RB = LOGN - B;
  static constexpr bool EVEN = RB % B == 0;
  static constexpr int NFULL = EVEN ? RB / B - 1 : RB / B;
  static constexpr int NST = NFULL + (EVEN ? 3 : 2);
  static constexpr int RL = 1 << (EVEN ? 1 : RB % B);
  static constexpr int radix(int s) { return s == 0 ? PT : s == NST - 1 ? RL : (EVEN && s == NST - 2) ? PT / 2 : PT; }
  static constexpr int span(int s) {
    int p = 1;
    for (int i = 0; i < s; ++i) p *= radix(i);
    return p;
  }
  // twiddles of stage s >= 1 at [tw_off(s) + (r - 1) span(s) + jm] (r < radix(s), jm < span(s)):
  // neighbouring threads read neighbouring entries
  static constexpr int tw_off(int s) {
    int o = 0;
    for (int i = 1; i < s; ++i) o += (radix(i) - 1) * span(i);
    return o;
  }
  static constexpr int TW = tw_off(NST);
};

// column pairs per block: at least one warp per block (PMIN), or twice that
template <int LOGN, int PT>
constexpr int pairs_min() {
  return FPlan<LOGN, PT>::TH >= 32 ? 1 : 32 / FPlan<LOGN, PT>::TH;
}

// padded shared-memory index: one spare slot per 16, so that the stage-0 writes (stride 16)
// fall in distinct banks
__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }

// complex elements of one pair's buffer, chosen so that the P pairs of a block sit in distinct
// banks for the accesses of one phase (16 float2 or 8 double2 per 128 bytes)
template <typename T, int N, int P>
constexpr int pair_stride() {
  const int base = N + N / 16;
  if (P == 1) return base;
  const int M = sizeof(T) == 4 ? 16 : 8;
  const int want = (M / P) > 0 ? (M / P) % M : 1;
  return base + ((want - base) % M + M) % M;
}

// shared memory of a block: P pair buffers, the stage twiddles, the rows' box-data pairs, the
// eigenvalues
template <typename T, int LOGN, int P, int PT>
constexpr size_t fft_smem() {
  return sizeof(V2<T>) * ((size_t)P * pair_stride<T, (1 << LOGN), P>() + FPlan<LOGN, PT>::TW + (1 << LOGN)) +
         sizeof(T) * (1 << LOGN);
}

// compile-time loop: f(std::integral_constant<int, i>) for i < n
template <typename F, int... I>
__device__ __forceinline__ void sfor_(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int n, typename F>
__device__ __forceinline__ void sfor(F&& f) {
  sfor_(f, std::make_integer_sequence<int, n>{});
}

// vector loads and stores of one complex value (8 or 16 bytes, aligned)
template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using t = float2;
};
template <>
struct Vec<double> {
  using t = double2;
};
template <typename T>
__device__ __forceinline__ V2<T> ld2(const V2<T>* p) {
  const typename Vec<T>::t v = *reinterpret_cast<const typename Vec<T>::t*>(p);
  return V2<T>{v.x, v.y};
}
template <typename T>
__device__ __forceinline__ V2<T> ldg2(const V2<T>* p) {
  const typename Vec<T>::t v = __ldg(reinterpret_cast<const typename Vec<T>::t*>(p));
  return V2<T>{v.x, v.y};
}
template <typename T>
__device__ __forceinline__ void st2(V2<T>* p, V2<T> a) {
  typename Vec<T>::t v;
  v.x = a.x;
  v.y = a.y;
  *reinterpret_cast<typename Vec<T>::t*>(p) = v;
}

// twiddle r of stage S for butterfly offset jm from the block's table: w^(r jm N / (Ns R)),
// w = e^{-2 pi i / N}, or its conjugate (inverse)
template <typename T, int LOGN, int PT, int S, bool INV>
__device__ __forceinline__ V2<T> twid(const V2<T>* sT, int r, int jm) {
  using PL = FPlan<LOGN, PT>;
  V2<T> w = ld2(sT + PL::tw_off(S) + (r - 1) * PL::span(S) + jm);
  if (INV) w.y = -w.y;
  return w;
}

// stage S's part of the twiddle table, gathered from the table of w^m (m < N) by the block's
// NT threads with all loads in flight before the stores
template <typename T, int LOGN, int PT, int S, int NT>
__device__ __forceinline__ void stage_table(const V2<T>* twN, V2<T>* sT) {
  using PL = FPlan<LOGN, PT>;
  constexpr int N = PL::N, R = PL::radix(S), NS = PL::span(S), WS = N / (NS * R);
  constexpr int CNT = (R - 1) * NS, PER = (CNT + NT - 1) / NT;
  V2<T> v[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int t = (int)threadIdx.x + i * NT;
    if (t < CNT) {
      const int r = t / NS + 1, jm = t & (NS - 1);
      v[i] = ldg2(twN + ((r * jm * WS) & (N - 1)));
    }
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int t = (int)threadIdx.x + i * NT;
    if (t < CNT) st2(sT + PL::tw_off(S) + t, v[i]);
  }
}

// one bin pair of the solve: A = Z[m], B = Z[N - m] of the forward FFT (0 <= m <= N/2) in,
// the inverse FFT's input at m and N - m out (B is not meaningful for m = 0 and m = N/2).
// DCT-II post-processing of both sequences, division by lam(l) + lam_x - kappa (float64 with
// the context's reciprocal table when it has one), pre-processing of the inverse.
// lam is the block's copy of the eigenvalues in shared memory.
template <typename T>
__device__ __forceinline__ void bin_pair(int m, int N, int dct, const T* tab, const T* lam, T lx0, T lx1,
                                         const T* r0, const T* r1, V2<T>& A, V2<T>& B) {
  T c, s;
  dct_cs<T>(tab, N, m, c, s);
  V2<T> Xm, XNm;
  dct_post_v<T>(A, B, c, s, Xm, XNm);
  const int l1 = dct ? m : N - 1 - m;
  const int l2 = dct ? N - m : m - 1;
  V2<T> Gm, GNm{(T)0, (T)0};
  if (r0 != nullptr) {
    Gm = V2<T>{Xm.x * __ldg(r0 + l1), Xm.y * __ldg(r1 + l1)};
    if (m > 0 && 2 * m < N) GNm = V2<T>{XNm.x * __ldg(r0 + l2), XNm.y * __ldg(r1 + l2)};
  } else {
    const T ly = lam[l1];
    Gm = V2<T>{fdiv_t(Xm.x, ly + lx0), fdiv_t(Xm.y, ly + lx1)};
    if (m > 0 && 2 * m < N) {
      const T ly2 = lam[l2];
      GNm = V2<T>{fdiv_t(XNm.x, ly2 + lx0), fdiv_t(XNm.y, ly2 + lx1)};
    }
  }
  if (2 * m == N) GNm = Gm;
  dct_pre<T>(N, m, c, s, Gm, GNm, A, B);
}

// forward middle stage s: butterflies j = u + TH g (g < PT / R), span Ns, radix R
template <typename T, int LOGN, int PT, int S>
__device__ __forceinline__ void stage_fwd(V2<T>* buf, V2<T> (&x)[PT], int u, const V2<T>* sT) {
  using PL = FPlan<LOGN, PT>;
  constexpr int N = PL::N, R = PL::radix(S), NS = PL::span(S), G = PT / R, TH = PL::TH;
  V2<T> w[G][R];
  sfor<G>([&](auto gi) {
    constexpr int g = decltype(gi)::value;
    const int j = u + TH * g, jm = j & (NS - 1);
#pragma unroll
    for (int r = 0; r < R; ++r) x[g * R + r] = ld2(buf + pidx(j + r * (N / R)));
#pragma unroll
    for (int r = 1; r < R; ++r) w[g][r] = twid<T, LOGN, PT, S, false>(sT, r, jm);
  });
  __syncthreads();  // every read of the buffer is done before it is overwritten
  sfor<G>([&](auto gi) {
    constexpr int g = decltype(gi)::value;
    const int j = u + TH * g, jm = j & (NS - 1);
#pragma unroll
    for (int r = 1; r < R; ++r) x[g * R + r] = cmul(x[g * R + r], w[g][r]);
    rg_dft_at<R, false, g * R>(x);
    const int base = (j / NS) * NS * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) st2(buf + pidx(base + r * NS), x[g * R + r]);
  });
  __syncthreads();
}

// adjoint of stage_fwd<S> (inverse DFT, conjugate twiddle, scatter back)
template <typename T, int LOGN, int PT, int S>
__device__ __forceinline__ void stage_inv(V2<T>* buf, V2<T> (&x)[PT], int u, const V2<T>* sT) {
  using PL = FPlan<LOGN, PT>;
  constexpr int N = PL::N, R = PL::radix(S), NS = PL::span(S), G = PT / R, TH = PL::TH;
  V2<T> w[G][R];
  sfor<G>([&](auto gi) {
    constexpr int g = decltype(gi)::value;
    const int j = u + TH * g, jm = j & (NS - 1);
    const int base = (j / NS) * NS * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) x[g * R + r] = ld2(buf + pidx(base + r * NS));
#pragma unroll
    for (int r = 1; r < R; ++r) w[g][r] = twid<T, LOGN, PT, S, true>(sT, r, jm);
  });
  __syncthreads();
  sfor<G>([&](auto gi) {
    constexpr int g = decltype(gi)::value;
    const int j = u + TH * g;
    rg_dft_at<R, true, g * R>(x);
#pragma unroll
    for (int r = 1; r < R; ++r) x[g * R + r] = cmul(x[g * R + r], w[g][r]);
#pragma unroll
    for (int r = 0; r < R; ++r) st2(buf + pidx(j + r * (N / R)), x[g * R + r]);
  });
  __syncthreads();
}

// butterfly b of the last stage for thread u: j = u + TH b for b < G/2, and the mirror
// images Ns - u - TH (b - G/2) for b >= G/2 (thread 0: Ns/2 in place of Ns), so that bin m and
// bin N - m are in the same thread
template <int LOGN, int PT, int B>
__device__ __forceinline__ int last_j(int u) {
  using PL = FPlan<LOGN, PT>;
  constexpr int RL = PL::RL, G = PT / RL, NSL = PL::N / RL, TH = PL::TH;
  if constexpr (B < G / 2) {
    return u + TH * B;
  } else if constexpr (B == G / 2) {
    return u == 0 ? NSL / 2 : NSL - u;
  } else {
    return NSL - u - TH * (B - G / 2);
  }
}

template <int S, int E, typename F>
__device__ __forceinline__ void srange(F&& f) {
  if constexpr (S < E) {
    f(std::integral_constant<int, S>{});
    srange<S + 1, E>(f);
  }
}

// FR (float32): the kernel forms its input rows itself instead of reading the row transform's
// output: row j of column k is
//   sum over the row's irregular nodes t of sv_t S_k(2 i_t + 1) + w_j S_k(0) + e_j S_k(N-1)
//   (+ the face row's transform for j = 0, N - 1),
// S_k the DST-II (DCT-II) basis function, sv_t the sum of node t's four arm corrections, (w_j,
// e_j) the free-space box data of the row. The row pointers and column factors (fixed with the
// interface) are staged before the wait for the jump kernel, the corrections and box data after.
template <typename T, int LOGN, int P, bool FR, int PT>
__global__ void __launch_bounds__(P * FPlan<LOGN, PT>::TH) k_col_fft(int dct, const V2<T>* __restrict__ twN,
                                                                const T* __restrict__ tab, const T* __restrict__ lam,
                                                                T kappa, T* spec, const T* __restrict__ rinv,
                                                                const V2<T>* __restrict__ rowinfo, RowSrc rs,
                                                                const int* skip) {
  using PL = FPlan<LOGN, PT>;
  constexpr int N = PL::N, TH = PL::TH, RL = PL::RL, G = PT / RL, NST = PL::NST, NSL = N / RL;
  constexpr int PS = pair_stride<T, N, P>();
  extern __shared__ float4 col_fft_smem[];
  const int p = (int)threadIdx.x % P, u = (int)threadIdx.x / P;
  const int k0 = (int)blockIdx.x * (2 * P) + 2 * p;  // this thread's columns k0, k0 + 1
  V2<T>* buf = reinterpret_cast<V2<T>*>(col_fft_smem) + p * PS;
  V2<T>* sT = reinterpret_cast<V2<T>*>(col_fft_smem) + P * PS;  // stage twiddles
  V2<T>* sRow = sT + PL::TW;                                     // rowinfo[j], j < N
  T* sLam = reinterpret_cast<T*>(sRow + N);                      // lam[l], l < N
  int* sRp = reinterpret_cast<int*>(sLam + N);                   // FR: row pointers [N + 1] (N + 2 slots)
  float* sSv = reinterpret_cast<float*>(sRp + N + 2);            // FR: sv_t [cap], cap even
  float* sTab = sSv + rs.cap;                                    // FR: the block's sines [tab][2P], 8-byte aligned
  int nirr = 0;
  if constexpr (FR) {
    // row pointers, and for the first rs.tab nodes the sines of the block's 2P columns
    // S_k(2 i_t + 1) (the rest are evaluated as the rows are formed)
    for (int t = threadIdx.x; t <= N; t += P * TH) sRp[t] = __ldg(rs.row_ptr + t);
    nirr = __ldg(rs.row_ptr + N);
    // node t's sines S_{kb + c}(ci), c < 2P: sin((kb + 1 + c) theta) (DST-II) or
    // cos((kb + c) theta) (DCT-II), theta = pi ci / (2N), each from its exactly reduced integer
    // argument (a rotation recurrence would cost float32 accuracy)
    const int ntab = min(nirr, rs.tab);
    const int kb = (int)blockIdx.x * (2 * P) + (dct ? 0 : 1);
    const float qs = qscale(N);
    constexpr int BATCH = 8;
    for (int t0 = 0; t0 < ntab; t0 += BATCH * P * TH) {
      int ci[BATCH];
#pragma unroll
      for (int i = 0; i < BATCH; ++i) {
        const int t = t0 + (int)threadIdx.x + i * P * TH;
        ci[i] = t < ntab ? __ldg(rs.ci + t) : 0;
      }
#pragma unroll
      for (int i = 0; i < BATCH; ++i) {
        const int t = t0 + (int)threadIdx.x + i * P * TH;
        if (t < ntab) {
          float v[2 * P];
#pragma unroll
          for (int c = 0; c < 2 * P; ++c) v[c] = tsin(tab, (kb + c) * ci[i] + (dct ? N : 0), N, qs);
          float* dst = sTab + t * (2 * P);
#pragma unroll
          for (int c = 0; c < 2 * P; c += 2) *reinterpret_cast<float2*>(dst + c) = make_float2(v[c], v[c + 1]);
        }
      }
    }
  }
  // the tables (fixed with the context) go to shared memory before the wait for the row
  // transform; the first barrier below orders these writes before every read
  srange<1, NST>([&](auto si) { stage_table<T, LOGN, PT, decltype(si)::value, P * TH>(twN, sT); });
  {
    constexpr int PER = (N + P * TH - 1) / (P * TH);
    T v[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int t = (int)threadIdx.x + i * P * TH;
      if (t < N) v[i] = __ldg(lam + t);
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int t = (int)threadIdx.x + i * P * TH;
      if (t < N) sLam[t] = v[i];
    }
  }
  const T lx0 = __ldg(lam + k0) - kappa, lx1 = __ldg(lam + k0 + 1) - kappa;
  const T* r0 = rinv != nullptr ? rinv + (long)k0 * N : nullptr;
  const T* r1 = rinv != nullptr ? r0 + N : nullptr;
  // rows the row transform did not write (rowinfo): w S_k(0) + e S_k(N-1) for both columns
  V2<T> s0{(T)0, (T)0}, sN{(T)0, (T)0};
  if (rowinfo != nullptr || FR) {
    const float qs = qscale(N);
    if (dct) {
      s0 = V2<T>{tsin(tab, k0 + N, N, qs), tsin(tab, k0 + 1 + N, N, qs)};
      sN = V2<T>{tsin(tab, k0 * (2 * N - 1) + N, N, qs), tsin(tab, (k0 + 1) * (2 * N - 1) + N, N, qs)};
    } else {
      s0 = V2<T>{tsin(tab, k0 + 1, N, qs), tsin(tab, k0 + 2, N, qs)};
      sN = V2<T>{tsin(tab, (k0 + 1) * (2 * N - 1), N, qs), tsin(tab, (k0 + 2) * (2 * N - 1), N, qs)};
    }
  }
  pdl_wait();
  if (*skip) return;

  // ---- stage 0: points u + r N/PT of the reordered pair (rows 2i for r < PT/2, 2N-1-2i above;
  // the DST takes (-1)^row of the odd rows)
  V2<T> x[PT];
  if constexpr (FR) {
    // corrections and box data, once per block, then each of the thread's rows
    for (int t0 = 0; t0 < nirr; t0 += 4 * P * TH) {
      float4 v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int t = t0 + (int)threadIdx.x + i * P * TH;
        if (t < nirr) v[i] = rs.slot[t];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int t = t0 + (int)threadIdx.x + i * P * TH;
        if (t < nirr) sSv[t] = (v[i].x + v[i].y) + (v[i].z + v[i].w);
      }
    }
    if (rs.boxg != nullptr)
      for (int t = threadIdx.x; t < N; t += P * TH) sRow[t] = V2<T>{rs.boxg[t], rs.boxg[N + t]};
    __syncthreads();
    const float qs = qscale(N);
#pragma unroll
    for (int r = 0; r < PT; ++r) {
      const int i = u + r * TH;
      const int row = r < PT / 2 ? 2 * i : 2 * N - 1 - 2 * i;
      T a0 = 0, a1 = 0;
      const int e = sRp[row + 1];
      const int et = min(e, rs.tab);
      int t = sRp[row];
      for (; t < et; ++t) {
        const T sv = sSv[t];
        const V2<T> sn = ld2(reinterpret_cast<const V2<T>*>(sTab + t * (2 * P) + 2 * p));
        a0 += sv * sn.x;
        a1 += sv * sn.y;
      }
      for (; t < e; ++t) {
        const int ci = __ldg(rs.ci + t);
        const T sv = sSv[t];
        if (dct) {
          a0 += sv * tsin(tab, k0 * ci + N, N, qs);
          a1 += sv * tsin(tab, (k0 + 1) * ci + N, N, qs);
        } else {
          a0 += sv * tsin(tab, (k0 + 1) * ci, N, qs);
          a1 += sv * tsin(tab, (k0 + 2) * ci, N, qs);
        }
      }
      if (rs.boxg != nullptr) {
        const V2<T> we = ld2(sRow + row);
        a0 += we.x * s0.x + we.y * sN.x;
        a1 += we.x * s0.y + we.y * sN.y;
      }
      if (rs.face != nullptr && (row == 0 || row == N - 1)) {
        const T* f = rs.face + (row == 0 ? 0 : N);
        a0 += f[k0];
        a1 += f[k0 + 1];
      }
      x[r] = V2<T>{a0, a1};
    }
  } else {
#pragma unroll
    for (int r = 0; r < PT; ++r) {
      const int i = u + r * TH;
      const int row = r < PT / 2 ? 2 * i : 2 * N - 1 - 2 * i;
      x[r] = *reinterpret_cast<const V2<T>*>(spec + (long)row * N + k0);
    }
  }
  // the rows' box-data pairs, once per block (the same for every column), while the column
  // loads are in flight
  if (!FR && rowinfo != nullptr) {
    constexpr int PER = (N + P * TH - 1) / (P * TH);
    V2<T> v[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int t = (int)threadIdx.x + i * P * TH;
      if (t < N) v[i] = ldg2(rowinfo + t);
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int t = (int)threadIdx.x + i * P * TH;
      if (t < N) st2(sRow + t, v[i]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < PT; ++r) {
    V2<T> v = x[r];
    if (!FR && rowinfo != nullptr) {
      const int i = u + r * TH;
      const V2<T> ri = ld2(sRow + (r < PT / 2 ? 2 * i : 2 * N - 1 - 2 * i));
      if (ri.x == ri.x) v = V2<T>{ri.x * s0.x + ri.y * sN.x, ri.x * s0.y + ri.y * sN.y};
    }
    if (!dct && r >= PT / 2) v = V2<T>{-v.x, -v.y};
    x[r] = v;
  }
  rg_dft<PT, false>(x);
#pragma unroll
  for (int r = 0; r < PT; ++r) st2(buf + pidx(PT * u + r), x[r]);
  __syncthreads();

  // ---- middle stages
  srange<1, NST - 1>([&](auto si) { stage_fwd<T, LOGN, PT, decltype(si)::value>(buf, x, u, sT); });

  // ---- last stage: radix RL, span NSL; the outputs stay in registers, x[b RL + r] = bin j_b + r NSL
  sfor<G>([&](auto bi) {
    constexpr int b = decltype(bi)::value;
    const int j = last_j<LOGN, PT, b>(u);
#pragma unroll
    for (int r = 0; r < RL; ++r) x[b * RL + r] = ld2(buf + pidx(j + r * NSL));
#pragma unroll
    for (int r = 1; r < RL; ++r) x[b * RL + r] = cmul(x[b * RL + r], twid<T, LOGN, PT, NST - 1, false>(sT, r, j));
    rg_dft_at<RL, false, b * RL>(x);
  });

  // ---- bin pairs: (b, r) with (b + G/2, RL-1-r); thread 0's butterflies 0 (bins r NSL) and
  // G/2 (bins NSL/2 + r NSL) pair within themselves
  sfor<G / 2>([&](auto bi) {
    constexpr int b = decltype(bi)::value;
    if (b > 0 || u != 0) {
      const int jl = last_j<LOGN, PT, b>(u), jh = last_j<LOGN, PT, b + G / 2>(u);
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        if (r < RL / 2)
          bin_pair<T>(jl + r * NSL, N, dct, tab, sLam, lx0, lx1, r0, r1, x[b * RL + r], x[(b + G / 2) * RL + RL - 1 - r]);
        else
          bin_pair<T>(jh + (RL - 1 - r) * NSL, N, dct, tab, sLam, lx0, lx1, r0, r1, x[(b + G / 2) * RL + RL - 1 - r],
                      x[b * RL + r]);
      }
    }
  });
  if (u == 0) {
    {
      V2<T> a = x[0], bb = x[0];
      bin_pair<T>(0, N, dct, tab, sLam, lx0, lx1, r0, r1, a, bb);
      x[0] = a;
      a = x[RL / 2];
      bb = a;
      bin_pair<T>(N / 2, N, dct, tab, sLam, lx0, lx1, r0, r1, a, bb);
      x[RL / 2] = a;
    }
#pragma unroll
    for (int r = 1; r < RL / 2; ++r) bin_pair<T>(r * NSL, N, dct, tab, sLam, lx0, lx1, r0, r1, x[r], x[RL - r]);
#pragma unroll
    for (int r = 0; r < RL / 2; ++r)
      bin_pair<T>(NSL / 2 + r * NSL, N, dct, tab, sLam, lx0, lx1, r0, r1, x[(G / 2) * RL + r],
                  x[(G / 2) * RL + RL - 1 - r]);
  }

  // ---- adjoint of the last stage: back to the positions it read (this thread's own)
  sfor<G>([&](auto bi) {
    constexpr int b = decltype(bi)::value;
    const int j = last_j<LOGN, PT, b>(u);
    rg_dft_at<RL, true, b * RL>(x);
#pragma unroll
    for (int r = 1; r < RL; ++r) x[b * RL + r] = cmul(x[b * RL + r], twid<T, LOGN, PT, NST - 1, true>(sT, r, j));
#pragma unroll
    for (int r = 0; r < RL; ++r) st2(buf + pidx(j + r * NSL), x[b * RL + r]);
  });
  __syncthreads();

  // ---- adjoints of the middle stages, last to first
  srange<1, NST - 1>([&](auto si) { stage_inv<T, LOGN, PT, NST - 1 - decltype(si)::value>(buf, x, u, sT); });

  // ---- adjoint of stage 0: positions 16 u + r -> points u + r N/16 -> rows, scaled by 1/N
#pragma unroll
  for (int r = 0; r < PT; ++r) x[r] = ld2(buf + pidx(PT * u + r));
  rg_dft<PT, true>(x);
  constexpr T invN = (T)1 / (T)N;
#pragma unroll
  for (int r = 0; r < PT; ++r) {
    const int i = u + r * TH;
    const int row = r < PT / 2 ? 2 * i : 2 * N - 1 - 2 * i;
    const T sc = (!dct && r >= PT / 2) ? -invN : invN;
    st2(reinterpret_cast<V2<T>*>(spec + (long)row * N + k0), V2<T>{x[r].x * sc, x[r].y * sc});
  }
}

template <typename T>
struct FftSel {
  void (*kernel)(int, const V2<T>*, const T*, const T*, T, T*, const T*, const V2<T>*, RowSrc, const int*) = nullptr;
  int threads = 0, pairs = 0;
  size_t smem = 0;  // without the FR node arrays
};

template <typename T, int LOGN, int P, bool FR, int PT>
FftSel<T> fft_sel() {
  FftSel<T> s;
  s.kernel = k_col_fft<T, LOGN, P, FR, PT>;
  s.threads = P * FPlan<LOGN, PT>::TH;
  s.pairs = P;
  s.smem = fft_smem<T, LOGN, P, PT>() + (FR ? sizeof(int) * ((1 << LOGN) + 2) : 0);
  return s;
}

// largest dynamic shared memory of one block on sm_103a
constexpr size_t FFT_SMEM_MAX = 227 * 1024;

// an instantiation exists for P pairs per block when N/2 pairs allow it, its shared memory fits
// and (for P > 2 PMIN) the block holds at most 4096 points (256 threads of 16, 512 of 8)
template <typename T, int LOGN, int P, int PT>
constexpr bool fft_fits() {
  return P <= (1 << LOGN) / 2 && fft_smem<T, LOGN, P, PT>() <= FFT_SMEM_MAX &&
         (P <= 2 * pairs_min<LOGN, PT>() || P * (1 << LOGN) <= 4096);
}

// the kernel for N = 2^logN with the largest instantiated pair count (PMIN, 2 PMIN, 4 PMIN) that
// does not exceed `want`, or PMIN; no kernel when even PMIN does not fit. The FR form (rows
// formed in the kernel) and the 8-point form exist in float32 only, and not together; the
// 8-point form for N <= 1024 (above it the 16-point form measured faster).
template <typename T, int LOGN, bool FR, int PT>
FftSel<T> fft_sel_n(int want) {
  constexpr int P0 = pairs_min<LOGN, PT>();
  if constexpr ((FR || PT == 8) && (sizeof(T) != 4 || (FR && PT == 8) || (PT == 8 && LOGN > 10))) {
    return FftSel<T>{};
  } else {
    if constexpr (fft_fits<T, LOGN, 4 * P0, PT>()) {
      if (want >= 4 * P0) return fft_sel<T, LOGN, 4 * P0, FR, PT>();
    }
    if constexpr (fft_fits<T, LOGN, 2 * P0, PT>()) {
      if (want >= 2 * P0) return fft_sel<T, LOGN, 2 * P0, FR, PT>();
    }
    if constexpr (fft_fits<T, LOGN, P0, PT>()) return fft_sel<T, LOGN, P0, FR, PT>();
    return FftSel<T>{};
  }
}

template <typename T, bool FR, int PT>
FftSel<T> fft_select_pt(int logN, int want) {
  switch (logN) {
    case 5: return fft_sel_n<T, 5, FR, PT>(want);
    case 6: return fft_sel_n<T, 6, FR, PT>(want);
    case 7: return fft_sel_n<T, 7, FR, PT>(want);
    case 8: return fft_sel_n<T, 8, FR, PT>(want);
    case 9: return fft_sel_n<T, 9, FR, PT>(want);
    case 10: return fft_sel_n<T, 10, FR, PT>(want);
    case 11: return fft_sel_n<T, 11, FR, PT>(want);
    case 12: return fft_sel_n<T, 12, FR, PT>(want);
    default: return FftSel<T>{};
  }
}

// points per thread 8 where that form exists (pt = 8), else 16
template <typename T, bool FR>
FftSel<T> fft_select(int logN, int want, int pt = 16) {
  if (pt == 8) {
    const FftSel<T> s = fft_select_pt<T, FR, 8>(logN, want);
    if (s.kernel != nullptr) return s;
  }
  return fft_select_pt<T, FR, 16>(logN, want);
}

// KFBI_OPT_COL_POINTS: 0 chooses 8 points per thread up to N = 1024 (twice the warps of the
// 16-point form; measured 5-38 % faster there) and 16 above (5-7 % faster there)
inline int fft_points(const kfbi_ctx* c) { return c->col_pt != 0 ? c->col_pt : (c->logN <= 10 ? 8 : 16); }

// pair count asked for: the context's KFBI_OPT_COL_PAIRS, else the largest instantiated one
// (4 PMIN up to N = 1024, 2 PMIN above: 2P float32 columns of 4 bytes per row segment, a whole
// 32-byte sector at 4 PMIN; measured fastest from N = 512 to 4096)
inline int fft_want(const kfbi_ctx* c) { return c->col_P > 0 ? c->col_P : 64; }

}  // namespace

bool col_fft_supported(int logN, bool fp32) {
  return fp32 ? fft_select<float, false>(logN, 1).kernel != nullptr
              : fft_select<double, false>(logN, 1).kernel != nullptr;
}

// the FR kernel's node arrays: sv for the capacity, and the sine table for as many nodes as the
// rest of the block's shared memory holds (at most the capacity)
static bool rows_layout(const kfbi_ctx* c, FftSel<float>* sel, RowSrc* rs, size_t* smem) {
  *sel = fft_select<float, true>(c->logN, fft_want(c), fft_points(c));
  if (sel->kernel == nullptr) return false;
  const int cap = (c->cap_irr + 1) & ~1;  // even: the sine table after sv stays 8-byte aligned
  const size_t base = sel->smem + sizeof(float) * (size_t)cap;
  if (base > FFT_SMEM_MAX) return false;
  const size_t per = sizeof(float) * 2 * (size_t)sel->pairs;
  const size_t room = (FFT_SMEM_MAX - base) / per;
  rs->cap = cap;
  rs->tab = (int)(room < (size_t)cap ? room : (size_t)cap);
  *smem = base + per * (size_t)rs->tab;
  return true;
}

bool col_fft_rows_fit(const kfbi_ctx* c) {
  FftSel<float> sel;
  RowSrc rs;
  size_t smem = 0;
  return rows_layout(c, &sel, &rs, &smem);
}

kfbi_status col_fft_launch(kfbi_ctx* c, bool fp32, void* spec, const void* rowinfo, const int* skip, bool pdl,
                           const RowSrc* rows) {
  const int N = c->N, dct = c->boxbc == KFBI_BOX_NEUMANN0;
  if (!col_fft_supported(c->logN, fp32)) return KFBI_ERR_ARG;
  if (fp32) {
    RowSrc rs{};
    FftSel<float> s;
    size_t smem = 0;
    if (rows != nullptr) {
      rs = *rows;
      if (!rows_layout(c, &s, &rs, &smem)) return KFBI_ERR_ARG;
    } else {
      s = fft_select<float, false>(c->logN, fft_want(c), fft_points(c));
      smem = s.smem;
    }
    KFBI_TRY(launch_k(pdl, s.kernel, dim3(N / (2 * s.pairs)), dim3(s.threads), smem, c->stream, dct,
                      (const V2<float>*)c->twN_f, (const float*)c->sintab_f, (const float*)c->lam_f, (float)c->kappa,
                      (float*)spec, (const float*)nullptr, (const V2<float>*)rowinfo, rs, skip));
  } else {
    if (rows != nullptr) return KFBI_ERR_ARG;
    const FftSel<double> s = fft_select<double, false>(c->logN, fft_want(c));
    KFBI_TRY(launch_k(pdl, s.kernel, dim3(N / (2 * s.pairs)), dim3(s.threads), s.smem, c->stream, dct,
                      (const V2<double>*)c->twN, (const double*)c->sintab, (const double*)c->lam, c->kappa,
                      (double*)spec, (const double*)c->rinv, (const V2<double>*)rowinfo, RowSrc{}, skip));
  }
  return KFBI_OK;
}

kfbi_status col_fft_setup_attributes() {
  for (int lg = 5; lg <= 12; ++lg)
    for (int want = 1; want <= 64; want *= 2) {
      for (int pt = 8; pt <= 16; pt += 8) {
        const FftSel<float> f = fft_select<float, false>(lg, want, pt);
        if (f.kernel != nullptr)
          KFBI_TRY(cudaFuncSetAttribute(f.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f.smem));
        const FftSel<float> fr = fft_select<float, true>(lg, want, pt);
        if (fr.kernel != nullptr)
          KFBI_TRY(cudaFuncSetAttribute(fr.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FFT_SMEM_MAX));
      }
      const FftSel<double> d = fft_select<double, false>(lg, want);
      if (d.kernel != nullptr)
        KFBI_TRY(cudaFuncSetAttribute(d.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)d.smem));
    }
  return KFBI_OK;
}

}  // namespace kfbi
