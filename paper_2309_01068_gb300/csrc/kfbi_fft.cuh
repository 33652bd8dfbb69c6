// Complex values and the shared-memory Stockham FFT, used by the grid transforms
// (kfbi_apply.cu) and by the fine sampling of the interface (kfbi_geometry.cu).
#pragma once

namespace kfbi {

template <typename T>
struct V2 {
  T x, y;
};

template <typename T>
__device__ __forceinline__ V2<T> cmul(V2<T> a, V2<T> b) {
  return V2<T>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ V2<T> cadd(V2<T> a, V2<T> b) {
  return V2<T>{a.x + b.x, a.y + b.y};
}
template <typename T>
__device__ __forceinline__ V2<T> csub(V2<T> a, V2<T> b) {
  return V2<T>{a.x - b.x, a.y - b.y};
}

// --------------------------------------------------------------------------- FFT core
// Stockham autosort FFT of P length-N sequences in shared memory (natural order in and
// out): one radix-2 stage when log2 N is odd, then radix-4 stages. Stage with span Ns and
// radix R: item j reads src[j + r N/R], multiplies by w^{r (j mod Ns) N/(Ns R)}, does the
// R-point DFT and writes dst[(j/Ns) Ns R + (j mod Ns) + r Ns]. stw holds, stage by stage,
// w^{r jm N / (4 Ns)} at [off + (r-1) Ns + jm] (w = e^{-2 pi i / N}, r = 1..3, off advancing by
// 3 Ns per stage) so that neighbouring threads read neighbouring twiddles; the inverse
// conjugates them (no 1/N). Returns the buffer with the result.
template <typename T>
__device__ V2<T>* fft_stockham(V2<T>* a, V2<T>* b, int P, int N, int logN, const V2<T>* stw, bool inverse) {
  V2<T>* src = a;
  V2<T>* dst = b;
  int Ns = 1;
  if (logN & 1) {
    const int h = N >> 1;
    for (int t = threadIdx.x; t < P * h; t += blockDim.x) {
      int p = t >> (logN - 1), j = t & (h - 1);
      const V2<T>* s = src + (long)p * N;
      V2<T>* d = dst + (long)p * N;
      V2<T> v0 = s[j], v1 = s[j + h];
      d[2 * j] = cadd(v0, v1);
      d[2 * j + 1] = csub(v0, v1);
    }
    __syncthreads();
    V2<T>* tmp = src; src = dst; dst = tmp;
    Ns = 2;
  }
  const int q = N >> 2;
  const int lq = logN - 2;
  int off = 0;
  for (; Ns < N; off += 3 * Ns, Ns <<= 2) {
    const int lNs = __ffs(Ns) - 1;
    for (int t = threadIdx.x; t < P * q; t += blockDim.x) {
      int p = t >> lq, j = t & (q - 1);
      const V2<T>* s = src + (long)p * N;
      V2<T>* d = dst + (long)p * N;
      int jm = j & (Ns - 1);
      V2<T> v0 = s[j], v1 = s[j + q], v2 = s[j + 2 * q], v3 = s[j + 3 * q];
      if (jm != 0) {
        V2<T> w1 = stw[off + jm], w2 = stw[off + Ns + jm], w3 = stw[off + 2 * Ns + jm];
        if (inverse) { w1.y = -w1.y; w2.y = -w2.y; w3.y = -w3.y; }
        v1 = cmul(v1, w1);
        v2 = cmul(v2, w2);
        v3 = cmul(v3, w3);
      }
      V2<T> a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3), t3 = csub(v1, v3);
      V2<T> a3 = inverse ? V2<T>{-t3.y, t3.x} : V2<T>{t3.y, -t3.x};  // (+/- i)(v1 - v3)
      int o = ((j >> lNs) << (lNs + 2)) + jm;
      d[o] = cadd(a0, a2);
      d[o + Ns] = cadd(a1, a3);
      d[o + 2 * Ns] = csub(a0, a2);
      d[o + 3 * Ns] = csub(a1, a3);
    }
    __syncthreads();
    V2<T>* tmp = src; src = dst; dst = tmp;
  }
  return src;
}

// The same transform for a size fixed at compile time (N = 2^LOGN): every stage's span,
// twiddle offset and index arithmetic become constants.
template <typename T, int LOGN, bool INV>
__device__ __forceinline__ V2<T>* fft_ct(V2<T>* a, V2<T>* b, int P, const V2<T>* stw) {
  constexpr int N = 1 << LOGN;
  constexpr int q = N >> 2, lq = LOGN - 2;
  constexpr int LNS0 = LOGN & 1;
  constexpr int NST = (LOGN - LNS0) / 2;
  V2<T>* src = a;
  V2<T>* dst = b;
  if constexpr (LNS0 != 0) {
    constexpr int h = N >> 1;
    for (int t = threadIdx.x; t < P * h; t += blockDim.x) {
      const int p = t >> (LOGN - 1), j = t & (h - 1);
      const V2<T>* s = src + p * N;
      V2<T>* d = dst + p * N;
      const V2<T> v0 = s[j], v1 = s[j + h];
      d[2 * j] = cadd(v0, v1);
      d[2 * j + 1] = csub(v0, v1);
    }
    __syncthreads();
    V2<T>* tmp = src; src = dst; dst = tmp;
  }
#pragma unroll
  for (int st = 0; st < NST; ++st) {
    const int lNs = LNS0 + 2 * st, Ns = 1 << lNs;
    const int off = (1 << LNS0) * ((1 << (2 * st)) - 1);
    for (int t = threadIdx.x; t < P * q; t += blockDim.x) {
      const int p = t >> lq, j = t & (q - 1);
      const V2<T>* s = src + p * N;
      V2<T>* d = dst + p * N;
      const int jm = j & (Ns - 1);
      V2<T> v0 = s[j], v1 = s[j + q], v2 = s[j + 2 * q], v3 = s[j + 3 * q];
      if (jm != 0) {
        V2<T> w1 = stw[off + jm], w2 = stw[off + Ns + jm], w3 = stw[off + 2 * Ns + jm];
        if (INV) {
          w1.y = -w1.y;
          w2.y = -w2.y;
          w3.y = -w3.y;
        }
        v1 = cmul(v1, w1);
        v2 = cmul(v2, w2);
        v3 = cmul(v3, w3);
      }
      const V2<T> a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3), t3 = csub(v1, v3);
      const V2<T> a3 = INV ? V2<T>{-t3.y, t3.x} : V2<T>{t3.y, -t3.x};
      const int o = ((j >> lNs) << (lNs + 2)) + jm;
      d[o] = cadd(a0, a2);
      d[o + Ns] = cadd(a1, a3);
      d[o + 2 * Ns] = csub(a0, a2);
      d[o + 3 * Ns] = csub(a1, a3);
    }
    __syncthreads();
    V2<T>* tmp = src; src = dst; dst = tmp;
  }
  return src;
}

// number of staged twiddles of fft_stockham for N = 2^logN (at most N)
__host__ __device__ inline int staged_count(int N, int logN) {
  int c = 0;
  for (int Ns = (logN & 1) ? 2 : 1; Ns < N; Ns <<= 2) c += 3 * Ns;
  return c;
}

// staged twiddles of fft_stockham for a length-n transform built from the roots
// roots[m] = e^{2 pi i m / n}: entry off + (r - 1) Ns + jm of the stage with span Ns holds
// w^{r jm n / (4 Ns)}, w = e^{-2 pi i / n} = conj roots[1]
__device__ __forceinline__ void stage_twiddles_from_roots(const double2* roots, V2<double>* stw, int n, int logn) {
  const int cnt = staged_count(n, logn);
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    int off = 0, Ns = (logn & 1) ? 2 : 1;
    while (t >= off + 3 * Ns) {
      off += 3 * Ns;
      Ns <<= 2;
    }
    const int r = (t - off) / Ns + 1, jm = (t - off) - (r - 1) * Ns;
    const double2 w = roots[(long)r * jm * (n / (4 * Ns))];
    stw[t] = V2<double>{w.x, -w.y};
  }
}

}  // namespace kfbi
