// Pieces of the fast grid solve shared by the column-solve kernels (kfbi_apply.cu,
// kfbi_colfft.cu): the sine of the DCT/DST rotations, the Makhoul reordering that turns a
// DCT-II (or DST-II) of length N into a complex FFT of length N, its pre- and
// post-processing, and DFTs of compile-time length held in registers.
#pragma once

#include <utility>

#include "kfbi_fft.cuh"

namespace kfbi {

__device__ __forceinline__ float fdiv_t(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv_t(double a, double b) { return a / b; }

// sin(pi m / (2N)) for an integer m (4N-periodic): the table in float64; in float32 the SFU
// sine after exact integer reduction of the argument to (-pi, pi] (absolute error < 4e-7)
__device__ __forceinline__ double tsin(const double* tab, int m, int N, float) { return tab[m & (4 * N - 1)]; }
__device__ __forceinline__ float tsin(const float*, int m, int N, float scale) {
  int r = m & (4 * N - 1);
  if (r > 2 * N) r -= 4 * N;
  return __sinf((float)r * scale);
}

// position of sample j in the Makhoul reordering v[n] = x[2n], v[N-1-n] = x[2n+1]
__device__ __forceinline__ int mk_pos(int j, int N) { return (j & 1) ? N - 1 - (j >> 1) : (j >> 1); }
// row of the grid that Makhoul position p holds (inverse of mk_pos)
__device__ __forceinline__ int mk_row(int p, int N) { return p < N / 2 ? 2 * p : 2 * N - 1 - 2 * p; }

// pi / (2N) in float32, the argument unit of tsin
__device__ __forceinline__ float qscale(int N) { return 1.57079632679489662f / (float)N; }

// DCT-II from the FFT of the reordered pair (sequence a in .x, b in .y), at m and N - m:
// V_a[m] = (Z[m] + conj Z[N-m]) / 2, V_b[m] = (Z[m] - conj Z[N-m]) / (2i),
// X'[m] = Re(e^{-i pi m / (2N)} V[m]); V[N-m] = conj V[m] for each real sequence.
// For DST-II the caller stored (-1)^j x_j and mode l is DCT index N-1-l.
// (c, s) = (cos, sin)(pi m / (2N)); the rotation at N - m is (sin, cos) of the same angle.
template <typename T>
__device__ __forceinline__ void dct_post_v(V2<T> Z, V2<T> Zr, T c, T s, V2<T>& Xm, V2<T>& XNm) {
  V2<T> Va{(T)0.5 * (Z.x + Zr.x), (T)0.5 * (Z.y - Zr.y)};
  V2<T> Vb{(T)0.5 * (Z.y + Zr.y), (T)-0.5 * (Z.x - Zr.x)};
  Xm = V2<T>{c * Va.x + s * Va.y, c * Vb.x + s * Vb.y};
  XNm = V2<T>{s * Va.x - c * Va.y, s * Vb.x - c * Vb.y};
}
template <typename T>
__device__ __forceinline__ void dct_post(const V2<T>* z, int N, int m, T c, T s, V2<T>& Xm, V2<T>& XNm) {
  dct_post_v<T>(z[m], z[(N - m) & (N - 1)], c, s, Xm, XNm);
}

// inverse of dct_post: V[m] = e^{i pi m/(2N)} (G[m] - i G[N-m]) per sequence, packed a + i b
template <typename T>
__device__ __forceinline__ void dct_pre(int N, int m, T c, T s, V2<T> Gm, V2<T> GNm, V2<T>& Zm, V2<T>& ZNm) {
  V2<T> Va{c * Gm.x + s * GNm.x, s * Gm.x - c * GNm.x};
  V2<T> Vb{c * Gm.y + s * GNm.y, s * Gm.y - c * GNm.y};
  Zm = V2<T>{Va.x - Vb.y, Va.y + Vb.x};
  V2<T> Wa{s * GNm.x + c * Gm.x, c * GNm.x - s * Gm.x};
  V2<T> Wb{s * GNm.y + c * Gm.y, c * GNm.y - s * Gm.y};
  ZNm = V2<T>{Wa.x - Wb.y, Wa.y + Wb.x};
}

// (cos, sin)(pi m / (2N)) from the sine table (float64) or the SFU (float32)
template <typename T>
__device__ __forceinline__ void dct_cs(const T* tab, int N, int m, T& c, T& s) {
  c = tsin(tab, m + N, N, qscale(N));
  s = tsin(tab, m, N, qscale(N));
}

// --------------------------------------------------------------------------- register DFTs
// sine and cosine of 2 pi k / M for compile-time k, M (Taylor series after reduction to
// [-pi, pi]; evaluated by the compiler)
constexpr double CT_PI = 3.14159265358979323846;
constexpr double ct_angle(int k, int M) {
  int r = k % M;
  if (2 * r > M) r -= M;
  return 2.0 * CT_PI * (double)r / (double)M;
}
constexpr double ct_sin(double x) {
  double t = x, s = x;
  for (int i = 1; i < 24; ++i) {
    t = -t * x * x / ((2.0 * i) * (2.0 * i + 1.0));
    s += t;
  }
  return s;
}
constexpr double ct_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int i = 1; i < 24; ++i) {
    t = -t * x * x / ((2.0 * i - 1.0) * (2.0 * i));
    s += t;
  }
  return s;
}

using V2f = V2<float>;

// b times e^{-2 pi i K / M} (forward) or e^{+2 pi i K / M} (inverse), K and M constants
template <int K, int M, bool INV, typename T>
__device__ __forceinline__ V2<T> ct_twiddle(V2<T> b) {
  if constexpr (K % M == 0) {
    return b;
  } else if constexpr (4 * (K % M) == M) {
    return INV ? V2<T>{-b.y, b.x} : V2<T>{b.y, -b.x};
  } else if constexpr (2 * (K % M) == M) {
    return V2<T>{-b.x, -b.y};
  } else if constexpr (4 * (K % M) == 3 * M) {
    return INV ? V2<T>{b.y, -b.x} : V2<T>{-b.y, b.x};
  } else {
    constexpr T c = (T)ct_cos(ct_angle(K, M));
    constexpr T s = (T)(INV ? ct_sin(ct_angle(K, M)) : -ct_sin(ct_angle(K, M)));
    return V2<T>{b.x * c - b.y * s, b.x * s + b.y * c};
  }
}

// one radix-2 Stockham stage of span NS on R points held in registers: item j takes x[j] and
// x[j + R/2], multiplies the second by w^{(j mod NS)} (w = e^{-+ 2 pi i / (2 NS)}) and writes the
// sum and difference to y[(j / NS) 2 NS + j mod NS] and the same + NS
template <int R, int NS, bool INV, int J, typename T>
__device__ __forceinline__ void rg_bfly(const V2<T> (&x)[R], V2<T> (&y)[R]) {
  constexpr int jm = J % NS;
  constexpr int o = (J / NS) * 2 * NS + jm;
  const V2<T> a = x[J];
  const V2<T> b = ct_twiddle<jm, 2 * NS, INV>(x[J + R / 2]);
  y[o] = V2<T>{a.x + b.x, a.y + b.y};
  y[o + NS] = V2<T>{a.x - b.x, a.y - b.y};
}
template <int R, int NS, bool INV, typename T, int... J>
__device__ __forceinline__ void rg_stage(const V2<T> (&x)[R], V2<T> (&y)[R], std::integer_sequence<int, J...>) {
  (rg_bfly<R, NS, INV, J>(x, y), ...);
}
// length-R DFT (R a power of two) of the points x[0..R) in place, natural order in and out
// (the inverse without the 1/R)
template <int R, bool INV, int NS = 1, typename T>
__device__ __forceinline__ void rg_dft(V2<T> (&x)[R]) {
  if constexpr (NS < R) {
    V2<T> y[R];
    rg_stage<R, NS, INV>(x, y, std::make_integer_sequence<int, R / 2>{});
#pragma unroll
    for (int i = 0; i < R; ++i) x[i] = y[i];
    rg_dft<R, INV, 2 * NS>(x);
  }
}
// the same on the sub-array x[O .. O + R) of a longer register array
template <int R, bool INV, int O, int L, typename T>
__device__ __forceinline__ void rg_dft_at(V2<T> (&x)[L]) {
  V2<T> t[R];
#pragma unroll
  for (int i = 0; i < R; ++i) t[i] = x[O + i];
  rg_dft<R, INV>(t);
#pragma unroll
  for (int i = 0; i < R; ++i) x[O + i] = t[i];
}
template <int R, bool INV, int L, typename T, int... Q>
__device__ __forceinline__ void rg_dft_each(V2<T> (&x)[L], std::integer_sequence<int, Q...>) {
  (rg_dft_at<R, INV, Q * R, L>(x), ...);
}

}  // namespace kfbi
