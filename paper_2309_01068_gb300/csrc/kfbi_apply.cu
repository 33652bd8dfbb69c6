// The KFBI apply (Sec. 4): jumps at crossings and nodes (App. A.1), corrected five-point
// right-hand side (Sec. 4.2), free-space box data (Sec. 4.1), the fast DST/DCT solve and
// the jump-corrected 6-point interpolation (Sec. 4.3). Every kernel is templated on the
// grid arithmetic type T (double for KFBI_FP64, float for the inner applies of
// KFBI_MIXED); interface inputs and outputs stay float64.
#include <cmath>
#include <mutex>

#include "kfbi_internal.cuh"

namespace kfbi {

template <typename T>
struct V2 {
  T x, y;
};

template <typename T>
__device__ __forceinline__ V2<T> cmul(V2<T> a, V2<T> b) {
  return V2<T>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

__device__ __forceinline__ void sincos_t(double a, double* s, double* c) { sincos(a, s, c); }
__device__ __forceinline__ void sincos_t(float a, float* s, float* c) { sincosf(a, s, c); }

template <typename T>
__device__ __forceinline__ T wsum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// --------------------------------------------------------------------------- density
// c_k = (1/n) sum_j phi_j e^{-2 pi i k j / n} (k = 0..n/2) in T; the warp of k = 0 also
// forms int phi ds = sum_j phi_j s_a,j 2 pi / n (trapezoidal rule).
template <typename T>
__global__ void k_dens_coef(const double* phi, int n, const double2* tw, const Stencil* st, V2<T>* coef,
                            double* dint, const int* skip) {
  if (*skip) return;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  int nk = n / 2 + 1;
  if (warp >= nk) return;
  int k = warp;
  T re = 0, im = 0;
  for (int j = lane; j < n; j += 32) {
    T v = (T)phi[j];
    double2 w = tw[(int)(((long)k * j) % n)];
    re += v * (T)w.x;
    im -= v * (T)w.y;
  }
  re = wsum(re);
  im = wsum(im);
  if (lane == 0) coef[k] = V2<T>{re / (T)n, im / (T)n};
  if (k == 0 && dint != nullptr) {
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s += phi[j] * st[j].w;
    s = wsum(s);
    if (lane == 0) *dint = s;
  }
}

// f, f', f'' of the density interpolant at alpha (warp-cooperative, see trig_warp)
template <typename T>
__device__ __forceinline__ void dens_eval(const V2<T>* c, int n, double alpha, int lane, T& f, T& f1, T& f2) {
  const int K = (n - 1) / 2;
  const int chunk = (K + 31) / 32;
  int k0 = 1 + lane * chunk;
  int k1 = min(K + 1, k0 + chunk);
  T a = 0, b = 0, d = 0;
  if (k0 < k1) {
    double es, ec, ss, sc;
    sincos((double)k0 * alpha, &es, &ec);
    sincos(alpha, &ss, &sc);
    T er = (T)ec, ei = (T)es, sr = (T)sc, si = (T)ss;
    for (int k = k0; k < k1; ++k) {
      V2<T> ck = c[k];
      T re = ck.x * er - ck.y * ei;
      T im = ck.x * ei + ck.y * er;
      a += re;
      b -= (T)k * im;
      d -= (T)k * (T)k * re;
      T t = er * sr - ei * si;
      ei = er * si + ei * sr;
      er = t;
    }
  }
  a = (T)2 * wsum(a);
  b = (T)2 * wsum(b);
  d = (T)2 * wsum(d);
  a += c[0].x;
  if ((n & 1) == 0) {
    double m = 0.5 * n;
    T nyq = c[n / 2].x;
    double s, co;
    sincos(m * alpha, &s, &co);
    a += nyq * (T)co;
    b -= (T)m * nyq * (T)s;
    d -= (T)(m * m) * nyq * (T)co;
  }
  f = a;
  f1 = b;
  f2 = d;
}

// jumps ([u], [u_x], [u_y], [u_xx], [u_yy], [u_xy]) at every target (App. A.1, Table 2)
template <typename T>
__global__ void k_target_jumps(const V2<T>* coef, int n, int ntg, const TargetGeo* tg, int layer, double kappa,
                               T* J, const int* skip) {
  if (*skip) return;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= ntg) return;
  const TargetGeo& g = tg[warp];
  T f, f1, f2;
  dens_eval<T>(coef, n, g.alpha, lane, f, f1, f2);
  if (lane != 0) return;
  T Phi, Phia, Phiaa, Psi, Psia;
  if (layer == KFBI_DOUBLE) {
    Phi = f; Phia = f1; Phiaa = f2; Psi = 0; Psia = 0;
  } else {
    Phi = 0; Phia = 0; Phiaa = 0; Psi = -f; Psia = -f1;
  }
  T xa = (T)g.xa, ya = (T)g.ya, xaa = (T)g.xaa, yaa = (T)g.yaa, sa = (T)g.sa, saa = (T)g.saa;
  T is2 = (T)1 / (sa * sa);
  T ux = (xa * Phia + ya * sa * Psi) * is2;
  T uy = (ya * Phia - xa * sa * Psi) * is2;
  T b0 = Phiaa - xaa * ux - yaa * uy;
  T b1 = saa * Psi + sa * Psia - yaa * ux + xaa * uy;
  T b2 = (T)kappa * Phi;
  T* o = J + (long)warp * 6;
  o[0] = Phi;
  o[1] = ux;
  o[2] = uy;
  o[3] = (T)g.A3i[0] * b0 + (T)g.A3i[1] * b1 + (T)g.A3i[2] * b2;
  o[4] = (T)g.A3i[3] * b0 + (T)g.A3i[4] * b1 + (T)g.A3i[5] * b2;
  o[5] = (T)g.A3i[6] * b0 + (T)g.A3i[7] * b1 + (T)g.A3i[8] * b2;
}

// C at every irregular node: sum over crossed arms of sign * (J0 + d J1 + d^2/2 J2) / h^2,
// J1, J2 = [u_x], [u_xx] on horizontal arms and [u_y], [u_yy] on vertical arms (Sec. 4.2)
template <typename T>
__global__ void k_corrections(int nirr, const IrrNode* irr, const T* J, double inv_h2, T* cval, const int* skip) {
  if (*skip) return;
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nirr) return;
  const IrrNode& node = irr[q];
  T acc = 0;
  for (int a = 0; a < 4; ++a) {
    int t = node.target[a];
    if (t < 0) continue;
    const T* j = J + (long)t * 6;
    T d = (T)node.d[a];
    T j1 = a < 2 ? j[1] : j[2];
    T j2 = a < 2 ? j[3] : j[4];
    acc += j[0] + d * j1 + (T)0.5 * d * d * j2;
  }
  cval[q] = (T)(node.sign * inv_h2) * acc;
}

// Free-space box data (Sec. 4.1): g(p) = (1/n) sum_l phi_l (X_l - p).(y_a, -x_a)_l / |X_l - p|^2
// at the 4N face midpoints, stored pre-scaled as the right-hand side term -2 g / h^2.
template <typename T>
__global__ void k_box_data(const double* phi, int n, const double* xy, const TargetGeo* tg_nodes, int N,
                           double xmin, double xmax, double ymin, double ymax, double h, T* boxg, const int* skip) {
  if (*skip) return;
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= 4 * N) return;
  int face = warp / N, idx = warp - face * N;
  double px, py;
  if (face == 0) { px = xmin; py = grid_coord(ymin, h, idx); }
  else if (face == 1) { px = xmax; py = grid_coord(ymin, h, idx); }
  else if (face == 2) { px = grid_coord(xmin, h, idx); py = ymin; }
  else { px = grid_coord(xmin, h, idx); py = ymax; }
  T acc = 0;
  T tpx = (T)px, tpy = (T)py;
  for (int l = lane; l < n; l += 32) {
    T dx = (T)xy[2 * l] - tpx, dy = (T)xy[2 * l + 1] - tpy;
    T num = dx * (T)tg_nodes[l].ya - dy * (T)tg_nodes[l].xa;
    acc += (T)phi[l] * num / (dx * dx + dy * dy);
  }
  acc = wsum(acc);
  if (lane == 0) boxg[warp] = (T)(-2.0 / (h * h * (double)n)) * acc;
}

// --------------------------------------------------------------------------- row transforms
// Sparse forward transform along x of one row (Sec. 4.2 right-hand side is zero away
// from irregular nodes and, for free-space box data, the boundary cells):
//   spec[j][k] = sum_i C[j][i] S_k(i),  S_k(i) = sin(pi (k+1)(2i+1)/(2N)) (DST-II) or
//   cos(pi k (2i+1)/(2N)) (DCT-II), from the table sin(pi m / (2N)), m mod 4N.
template <typename T>
__global__ void k_row_forward(int N, int dct, const int* row_ptr, const IrrNode* irr, const T* cval,
                              const T* boxg, const T* tab, T* spec, const int* skip) {
  if (*skip) return;
  extern __shared__ unsigned char smem_raw[];
  int* si = (int*)smem_raw;
  T* sv = (T*)(smem_raw + sizeof(int) * 1024);
  int j = blockIdx.y;
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int mask = 4 * N - 1;
  int b = row_ptr[j], e = row_ptr[j + 1];
  T acc = 0;
  // irregular-node entries, staged through shared memory in chunks
  for (int c0 = b; c0 < e; c0 += 1024) {
    int cnt = min(1024, e - c0);
    __syncthreads();
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      si[t] = 2 * irr[c0 + t].i + 1;
      sv[t] = cval[c0 + t];
    }
    __syncthreads();
    if (k < N) {
      if (dct)
        for (int t = 0; t < cnt; ++t) acc += sv[t] * tab[(k * si[t] + N) & mask];
      else
        for (int t = 0; t < cnt; ++t) acc += sv[t] * tab[((k + 1) * si[t]) & mask];
    }
  }
  if (boxg != nullptr && k < N) {
    // west (i = 0) and east (i = N-1) faces of this row
    T w = boxg[j], ea = boxg[N + j];
    if (dct) {
      acc += w * tab[(k + N) & mask] + ea * tab[(k * (2 * N - 1) + N) & mask];
    } else {
      acc += w * tab[(k + 1) & mask] + ea * tab[((k + 1) * (2 * N - 1)) & mask];
    }
    if (j == 0 || j == N - 1) {  // south / north face: a dense row
      const T* g = boxg + (j == 0 ? 2 * N : 3 * N);
      if (dct)
        for (int i = 0; i < N; ++i) acc += g[i] * tab[(k * (2 * i + 1) + N) & mask];
      else
        for (int i = 0; i < N; ++i) acc += g[i] * tab[((k + 1) * (2 * i + 1)) & mask];
    }
  }
  if (k < N) spec[(long)j * N + k] = acc;
}

// --------------------------------------------------------------------------- FFT core
// In-place radix-2 decimation-in-frequency FFT of P length-N sequences in shared memory,
// natural order in, bit-reversed order out. tw[m] = e^{-2 pi i m / N}, m < N/2; the
// inverse uses the conjugate twiddles (no 1/N scaling here).
template <typename T>
__device__ void fft_dif(V2<T>* z, int P, int N, int logN, const V2<T>* tw, bool inverse) {
  const int halfN = N >> 1;
  for (int lh = logN - 1, ls = 0; lh >= 0; --lh, ++ls) {
    const int half = 1 << lh;
    for (int t = threadIdx.x; t < P * halfN; t += blockDim.x) {
      int p = t >> (logN - 1);
      int b = t & (halfN - 1);
      int grp = b >> lh, pos = b & (half - 1);
      int i0 = (grp << (lh + 1)) + pos, i1 = i0 + half;
      V2<T>* zz = z + (long)p * N;
      V2<T> a = zz[i0], c = zz[i1];
      V2<T> w = tw[pos << ls];
      if (inverse) w.y = -w.y;
      zz[i0] = V2<T>{a.x + c.x, a.y + c.y};
      zz[i1] = cmul(V2<T>{a.x - c.x, a.y - c.y}, w);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int bitrev(int k, int logN) { return (int)(__brev((unsigned)k) >> (32 - logN)); }

// position of sample j in the Makhoul reordering v[n] = x[2n], v[N-1-n] = x[2n+1]
__device__ __forceinline__ int mk_pos(int j, int N) { return (j & 1) ? N - 1 - (j >> 1) : (j >> 1); }

// Forward real-to-real transform of pair p (sequence a in .x, b in .y) already reordered
// and FFT'd in z (bit-reversed). For m in [0, N/2] the thread handling m also handles N-m.
// X'[m] = Re(e^{-i pi m/(2N)} V[m]) is the DCT-II of the stored sequence; for DST-II the
// caller stored (-1)^j x_j and mode l corresponds to m = N-1-l.
template <typename T>
__device__ __forceinline__ void dct_post(const V2<T>* z, int N, int logN, int m, const T* tab, V2<T>& Xm,
                                         V2<T>& XNm) {
  const int mask = 4 * N - 1;
  int mN = (N - m) & (N - 1);
  V2<T> Z = z[bitrev(m, logN)];
  V2<T> Zr = z[bitrev(mN, logN)];
  // V_a[m] = (Z[m] + conj Z[N-m]) / 2, V_b[m] = (Z[m] - conj Z[N-m]) / (2i)
  V2<T> Va{(T)0.5 * (Z.x + Zr.x), (T)0.5 * (Z.y - Zr.y)};
  V2<T> Vb{(T)0.5 * (Z.y + Zr.y), (T)-0.5 * (Z.x - Zr.x)};
  T c = tab[(m + N) & mask], s = tab[m & mask];  // cos, sin of pi m / (2N)
  Xm = V2<T>{c * Va.x + s * Va.y, c * Vb.x + s * Vb.y};
  // the same for N - m (V[N-m] = conj V[m] for each real sequence)
  V2<T> Vra{Va.x, -Va.y}, Vrb{Vb.x, -Vb.y};
  T c2 = tab[((N - m) + N) & mask], s2 = tab[(N - m) & mask];
  XNm = V2<T>{c2 * Vra.x + s2 * Vra.y, c2 * Vrb.x + s2 * Vrb.y};
}

// Inverse preprocessing: from G (DCT-domain coefficients of a and b at m and N-m) build
// V[m] = e^{i pi m/(2N)} (G[m] - i G[N-m]) for each sequence and pack a + i b.
template <typename T>
__device__ __forceinline__ void dct_pre(int N, int m, const T* tab, V2<T> Gm, V2<T> GNm, V2<T>& Zm, V2<T>& ZNm) {
  const int mask = 4 * N - 1;
  T c = tab[(m + N) & mask], s = tab[m & mask];
  // sequence a: (Gm.x - i GNm.x) * (c + i s)
  V2<T> Va{c * Gm.x + s * GNm.x, s * Gm.x - c * GNm.x};
  V2<T> Vb{c * Gm.y + s * GNm.y, s * Gm.y - c * GNm.y};
  Zm = V2<T>{Va.x - Vb.y, Va.y + Vb.x};
  if (m == 0) {  // G[N] = 0
    Va = V2<T>{Gm.x, 0};
    Vb = V2<T>{Gm.y, 0};
    Zm = V2<T>{Va.x - Vb.y, Va.y + Vb.x};
  }
  int mm = N - m;
  T c2 = tab[(mm + N) & mask], s2 = tab[mm & mask];
  V2<T> Wa{c2 * GNm.x + s2 * Gm.x, s2 * GNm.x - c2 * Gm.x};
  V2<T> Wb{c2 * GNm.y + s2 * Gm.y, s2 * GNm.y - c2 * Gm.y};
  ZNm = V2<T>{Wa.x - Wb.y, Wa.y + Wb.x};
}

// --------------------------------------------------------------------------- column solve
// For each column k of spec (x-mode k): forward transform along y, divide by
// lam_y(l) + lam_x(k) - kappa, inverse transform along y. A block owns CP column pairs;
// pair p holds columns (k0 + 2p, k0 + 2p + 1) as the real and imaginary parts of one
// complex FFT. spec is overwritten with the result.
template <typename T>
__global__ void k_col_solve(int N, int logN, int CP, int dct, const V2<T>* tw, const T* tab, const T* lam,
                            double kappa, T* spec, const int* skip) {
  if (*skip) return;
  extern __shared__ unsigned char smem_raw[];
  V2<T>* z = (V2<T>*)smem_raw;
  const int k0 = blockIdx.x * (2 * CP);
  const int W = 2 * CP;
  // load + reorder (+ (-1)^j for DST)
  for (int t = threadIdx.x; t < N * W; t += blockDim.x) {
    int j = t / W, c = t - j * W;
    T v = spec[(long)j * N + k0 + c];
    if (!dct && (j & 1)) v = -v;
    int p = c >> 1;
    T* dst = (T*)&z[(long)p * N + mk_pos(j, N)];
    dst[c & 1] = v;
  }
  __syncthreads();
  fft_dif<T>(z, CP, N, logN, tw, false);
  // post-process, divide, pre-process; stage through registers because output positions
  // are read by other threads
  const int halfN = N >> 1;
  const int per = (CP * (halfN + 1) + blockDim.x - 1) / blockDim.x;
  V2<T> outA[8], outB[8];
  int outP[8], outM[8];
  int cnt = 0;
  for (int t = threadIdx.x; t < CP * (halfN + 1); t += blockDim.x) {
    int p = t / (halfN + 1), m = t - p * (halfN + 1);
    const V2<T>* zz = z + (long)p * N;
    V2<T> Xm, XNm;
    dct_post<T>(zz, N, logN, m, tab, Xm, XNm);
    T lx0 = lam[k0 + 2 * p], lx1 = lam[k0 + 2 * p + 1];
    // eigen-mode index along y of DCT-domain index m
    int lm = dct ? m : N - 1 - m;
    int lNm = dct ? ((N - m) & (N - 1)) : m - 1;  // for m = 0, N-m = N is not a mode
    T ly = lam[lm];
    V2<T> Gm{Xm.x / (ly + lx0 - (T)kappa), Xm.y / (ly + lx1 - (T)kappa)};
    V2<T> GNm{0, 0};
    if (m > 0) {
      T ly2 = lam[lNm];
      GNm = V2<T>{XNm.x / (ly2 + lx0 - (T)kappa), XNm.y / (ly2 + lx1 - (T)kappa)};
    }
    if (m == halfN) GNm = Gm;
    V2<T> Zm, ZNm;
    dct_pre<T>(N, m, tab, Gm, GNm, Zm, ZNm);
    if (cnt < 8) {
      outA[cnt] = Zm;
      outB[cnt] = ZNm;
      outP[cnt] = p;
      outM[cnt] = m;
    }
    ++cnt;
  }
  (void)per;
  __syncthreads();
  for (int q = 0; q < cnt && q < 8; ++q) {
    V2<T>* zz = z + (long)outP[q] * N;
    int m = outM[q];
    zz[m] = outA[q];
    if (m > 0 && m < halfN) zz[N - m] = outB[q];
  }
  __syncthreads();
  fft_dif<T>(z, CP, N, logN, tw, true);
  const T invN = (T)1 / (T)N;
  for (int t = threadIdx.x; t < N * W; t += blockDim.x) {
    int j = t / W, c = t - j * W;
    int p = c >> 1;
    const T* src = (const T*)&z[(long)p * N + bitrev(mk_pos(j, N), logN)];
    T v = src[c & 1] * invN;
    if (!dct && (j & 1)) v = -v;
    spec[(long)j * N + k0 + c] = v;
  }
}

// Probe values: inverse transform along x evaluated only at the interpolation points,
//   u[j][i] = (2/N) sum_k w_k spec[j][k] sin(pi (k+1)(2i+1)/(2N)), w_{N-1} = 1/2  (DST-III)
//   u[j][i] = (1/N) (spec[j][0] + 2 sum_{k>=1} spec[j][k] cos(pi k (2i+1)/(2N)))  (DCT-III)
// one block per grid row, one warp per probe of that row.
template <typename T>
__global__ void k_probe_values(int N, int dct, const int* prow_ptr, const int* probe_i, const T* spec, const T* tab,
                               T* pval, const int* skip) {
  if (*skip) return;
  int j = blockIdx.x;
  int b = prow_ptr[j], e = prow_ptr[j + 1];
  if (b == e) return;
  extern __shared__ unsigned char smem_raw[];
  T* row = (T*)smem_raw;
  for (int k = threadIdx.x; k < N; k += blockDim.x) row[k] = spec[(long)j * N + k];
  __syncthreads();
  const int mask = 4 * N - 1;
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = b + wid; q < e; q += nw) {
    int m = 2 * probe_i[q] + 1;
    T acc = 0;
    if (dct) {
      for (int k = lane; k < N; k += 32) acc += (k == 0 ? (T)0.5 : (T)1) * row[k] * tab[(k * m + N) & mask];
    } else {
      for (int k = lane; k < N; k += 32) acc += (k == N - 1 ? (T)0.5 : (T)1) * row[k] * tab[((k + 1) * m) & mask];
    }
    acc = wsum(acc);
    if (lane == 0) pval[q] = acc * ((T)2 / (T)N);
  }
}

// Dense transforms along x of row pairs (for grid output and the plain box solve).
// forward: spec[j][.] = DST-II/DCT-II of rhs[j][.] (rhs float64);
// inverse: out[j][.] = exact inverse of spec[j][.] (out float64).
template <typename T>
__global__ void k_row_dense(int N, int logN, int dct, int inverse, const V2<T>* tw, const T* tab,
                            const double* rhs, T* spec, double* out) {
  extern __shared__ unsigned char smem_raw[];
  V2<T>* z = (V2<T>*)smem_raw;
  const int j0 = 2 * blockIdx.x;  // rows j0 (real part), j0+1 (imag part)
  const int halfN = N >> 1;
  if (!inverse) {
    for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
      int r = t / N, i = t - r * N;
      T v = (T)rhs[(long)(j0 + r) * N + i];
      if (!dct && (i & 1)) v = -v;
      ((T*)&z[mk_pos(i, N)])[r] = v;
    }
    __syncthreads();
    fft_dif<T>(z, 1, N, logN, tw, false);
    for (int m = threadIdx.x; m <= halfN; m += blockDim.x) {
      V2<T> Xm, XNm;
      dct_post<T>(z, N, logN, m, tab, Xm, XNm);
      // DCT index m -> mode (DCT: m; DST: N-1-m)
      int km = dct ? m : N - 1 - m;
      spec[(long)j0 * N + km] = Xm.x;
      spec[(long)(j0 + 1) * N + km] = Xm.y;
      if (m > 0 && m < halfN) {
        int kNm = dct ? N - m : m - 1;
        spec[(long)j0 * N + kNm] = XNm.x;
        spec[(long)(j0 + 1) * N + kNm] = XNm.y;
      }
    }
  } else {
    for (int m = threadIdx.x; m <= halfN; m += blockDim.x) {
      int km = dct ? m : N - 1 - m;
      V2<T> Gm{spec[(long)j0 * N + km], spec[(long)(j0 + 1) * N + km]};
      V2<T> GNm{0, 0};
      if (m > 0) {
        int kNm = dct ? N - m : m - 1;
        GNm = V2<T>{spec[(long)j0 * N + kNm], spec[(long)(j0 + 1) * N + kNm]};
      }
      V2<T> Zm, ZNm;
      dct_pre<T>(N, m, tab, Gm, GNm, Zm, ZNm);
      z[m] = Zm;
      if (m > 0 && m < halfN) z[N - m] = ZNm;
    }
    __syncthreads();
    fft_dif<T>(z, 1, N, logN, tw, true);
    const T invN = (T)1 / (T)N;
    for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
      int r = t / N, i = t - r * N;
      T v = ((const T*)&z[bitrev(mk_pos(i, N), logN)])[r] * invN;
      if (!dct && (i & 1)) v = -v;
      out[(long)(j0 + r) * N + i] = (double)v;
    }
  }
}

// --------------------------------------------------------------------------- interpolation
// Per node (Sec. 4.3): b_m = u(q_m) + [q_m in Omega-] C(q_m), v+ = r0.b, grad v+ = (r1.b, r2.b);
// value (v+ + v-)/2 = v+ - [v]/2; dnormal = n.(grad v+ - [grad v]/2). The result is written as
//   out = a x + b value + c int(x) ds   (a, b, c select the boundary integral operator)
template <typename T>
__global__ void k_interp(int n, const Stencil* st, const T* pval, const T* Jn, const double* x_in,
                         const double* eps_v, double ca, double cb, double cc, const double* dint, double* out,
                         double* dnormal, const int* skip) {
  if (*skip) return;
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const Stencil& S = st[p];
  const T* J = Jn ? Jn + (long)p * 6 : nullptr;
  T v = 0, gx = 0, gy = 0;
  for (int m = 0; m < 6; ++m) {
    T u = pval[S.probe[m]];
    if (J != nullptr && S.minus[m]) {
      T dx = (T)S.dx[m], dy = (T)S.dy[m];
      u += J[0] + dx * J[1] + dy * J[2] + (T)0.5 * dx * dx * J[3] + dx * dy * J[5] + (T)0.5 * dy * dy * J[4];
    }
    v += (T)S.r0[m] * u;
    gx += (T)S.r1[m] * u;
    gy += (T)S.r2[m] * u;
  }
  double val = (double)v, dn = 0.0;
  if (J != nullptr) {
    val -= 0.5 * (double)J[0];
    gx -= (T)0.5 * J[1];
    gy -= (T)0.5 * J[2];
  }
  dn = S.nx * (double)gx + S.ny * (double)gy;
  double a = eps_v != nullptr ? eps_v[p] : ca;
  double xin = x_in != nullptr ? x_in[p] : 0.0;
  double o = a * xin + cb * val;
  if (dint != nullptr) o += cc * (*dint);
  out[p] = o;
  if (dnormal != nullptr) dnormal[p] = dn;
}

// --------------------------------------------------------------------------- host side
template <typename T>
static int col_pairs_per_block() {
  return sizeof(T) == 8 ? 2 : 4;
}

template <typename T>
static kfbi_status launch_col_solve(kfbi_ctx* c, T* spec, const int* skip) {
  const int N = c->N;
  int CP = col_pairs_per_block<T>();
  if (2 * CP > N) CP = N / 2;
  // the register staging in k_col_solve holds at most 8 (m, N-m) pairs per thread
  while (CP > 1 && CP * (N / 2 + 1) > 8 * 1024) CP /= 2;
  size_t smem = sizeof(V2<T>) * (size_t)CP * N;
  const T* tab = sizeof(T) == 8 ? (const T*)c->sintab : (const T*)c->sintab_f;
  const T* lam = sizeof(T) == 8 ? (const T*)c->lam : (const T*)c->lam_f;
  const V2<T>* tw = sizeof(T) == 8 ? (const V2<T>*)c->twN : (const V2<T>*)c->twN_f;
  KFBI_TRY(cudaFuncSetAttribute(k_col_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int threads = 256;
  while (CP * (N / 2 + 1) > 8 * threads && threads < 1024) threads *= 2;
  const bool rec = c->timing && c->timing_used < TIMING_CAP;
  if (rec) KFBI_TRY(cudaEventRecord(c->tev[2 * c->timing_used], c->stream));
  k_col_solve<T><<<N / (2 * CP), threads, smem, c->stream>>>(N, c->logN, CP, c->boxbc == KFBI_BOX_NEUMANN0, tw,
                                                            tab, lam, c->kappa, spec, skip);
  launched(c, 1);
  if (rec) {
    KFBI_TRY(cudaEventRecord(c->tev[2 * c->timing_used + 1], c->stream));
    c->tprec[c->timing_used] = sizeof(T) == 4 ? 1 : 0;
    c->timing_used += 1;
  }
  return KFBI_OK;
}

template <typename T>
static kfbi_status apply_t(kfbi_ctx* c, int layer, const double* density, double* values, double* dnormal,
                           double* grid, int bie_kind, const double* eps_v, const int* skip) {
  cudaStream_t s = c->stream;
  const int N = c->N, n = c->n, ncr = c->n_cross, ntg = ncr + n;
  const bool dct = c->boxbc == KFBI_BOX_NEUMANN0;
  const T* tab = sizeof(T) == 8 ? (const T*)c->sintab : (const T*)c->sintab_f;
  V2<T>* coef = (V2<T>*)c->dcoef;
  T* J = (T*)c->jumps;
  T* cval = (T*)c->cval;
  T* boxg = (T*)c->boxg;
  T* spec = (T*)c->spec;
  T* pval = (T*)c->probe_val;
  const int nk = n / 2 + 1;
  bool want_int = bie_kind == KFBI_BIE_HS_EXTERIOR_MDL;
  launched(c, 5 + (c->n_irr > 0) + (c->boxbc == KFBI_BOX_FREESPACE_DL) + (grid != nullptr));  // col solve counts itself
  k_dens_coef<T><<<cdiv((long)nk * 32, 256), 256, 0, s>>>(density, n, (const double2*)c->twn, c->stencil, coef,
                                                          want_int ? c->dint : nullptr, skip);
  k_target_jumps<T><<<cdiv((long)ntg * 32, 256), 256, 0, s>>>(coef, n, ntg, c->tgeo, layer, c->kappa, J, skip);
  if (c->n_irr > 0)
    k_corrections<T><<<cdiv(c->n_irr, 256), 256, 0, s>>>(c->n_irr, c->irr, J, 1.0 / (c->h * c->h), cval, skip);
  bool fs = c->boxbc == KFBI_BOX_FREESPACE_DL;
  if (fs)
    k_box_data<T><<<cdiv((long)4 * N * 32, 256), 256, 0, s>>>(density, n, c->xy, c->tgeo + ncr, N, c->xmin, c->xmax,
                                                              c->ymin, c->ymax, c->h, boxg, skip);
  dim3 g1(cdiv(N, 256), N);
  size_t sm1 = 1024 * (sizeof(int) + sizeof(T));
  k_row_forward<T><<<g1, 256, sm1, s>>>(N, dct, c->row_ptr, c->irr, cval, fs ? boxg : nullptr, tab, spec, skip);
  KFBI_CHECK(launch_col_solve<T>(c, spec, skip));
  size_t sm2 = sizeof(T) * N;
  k_probe_values<T><<<N, 256, sm2, s>>>(N, dct, c->prow_ptr, c->probe_i, spec, tab, pval, skip);
  if (grid != nullptr) {
    size_t sm3 = sizeof(V2<T>) * N;
    const V2<T>* tw = sizeof(T) == 8 ? (const V2<T>*)c->twN : (const V2<T>*)c->twN_f;
    KFBI_TRY(cudaFuncSetAttribute(k_row_dense<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
    k_row_dense<T><<<N / 2, 256, sm3, s>>>(N, c->logN, dct, 1, tw, tab, nullptr, spec, grid);
  }
  double ca = 0.0, cb = 1.0, cc = 0.0;
  const double* ev = nullptr;
  const double* xin = nullptr;
  if (bie_kind == KFBI_BIE_INTERIOR_DL) { ca = 0.5; xin = density; }
  else if (bie_kind == KFBI_BIE_HS_EXTERIOR_MDL) { ca = -0.5; cc = 1.0; xin = density; }
  else if (bie_kind == KFBI_BIE_STEFAN_SL) { cb = -1.0; ev = eps_v; xin = density; }
  k_interp<T><<<cdiv(n, 128), 128, 0, s>>>(n, c->stencil, pval, J + (long)ncr * 6, xin, ev, ca, cb, cc,
                                           want_int ? c->dint : nullptr, values, dnormal, skip);
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

// bie_kind < 0: plain layer potential
kfbi_status apply_enqueue(kfbi_ctx* c, int layer, bool fp32, const double* density, double* values, double* dnormal,
                          double* grid, int bie_kind, const double* eps_v, const int* skip) {
  if (skip == nullptr) skip = c->zero_flag;
  if (fp32) return apply_t<float>(c, layer, density, values, dnormal, grid, bie_kind, eps_v, skip);
  return apply_t<double>(c, layer, density, values, dnormal, grid, bie_kind, eps_v, skip);
}

template <typename T>
static kfbi_status grid_solve_t(kfbi_ctx* c, const double* rhs, double* u) {
  cudaStream_t s = c->stream;
  const int N = c->N;
  const bool dct = c->boxbc == KFBI_BOX_NEUMANN0;
  const T* tab = sizeof(T) == 8 ? (const T*)c->sintab : (const T*)c->sintab_f;
  const V2<T>* tw = sizeof(T) == 8 ? (const V2<T>*)c->twN : (const V2<T>*)c->twN_f;
  T* spec = (T*)c->spec;
  size_t sm3 = sizeof(V2<T>) * N;
  KFBI_TRY(cudaFuncSetAttribute(k_row_dense<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
  k_row_dense<T><<<N / 2, 256, sm3, s>>>(N, c->logN, dct, 0, tw, tab, rhs, spec, nullptr);
  launched(c, 2);
  KFBI_CHECK(launch_col_solve<T>(c, spec, c->zero_flag));
  k_row_dense<T><<<N / 2, 256, sm3, s>>>(N, c->logN, dct, 1, tw, tab, nullptr, spec, u);
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

kfbi_status grid_solve_enqueue(kfbi_ctx* c, const double* rhs, double* u) {
  return grid_solve_t<double>(c, rhs, u);
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
  k_interp<double><<<cdiv(c->n, 128), 128, 0, s>>>(c->n, c->stencil, pval, nullptr, nullptr, nullptr, 0.0, 1.0, 0.0,
                                                    nullptr, values, nullptr, c->zero_flag);
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

// --------------------------------------------------------------------------- allocation-free solve
// kfbi_grid_solve_noalloc: the plain box solve of kfbi_grid_solve for callers that cannot
// allocate device memory (see include/kfbi.h). Its scratch lives in one file-scope device
// array: one slot holding the column kernel's skip flag (cleared by every call before the
// kernel reads it), then the spectral grid (N^2), the sine table (4N), the eigenvalues (N) and
// the FFT twiddles (N). Every call rewrites all of it before reading it. The array is shared
// by every call in the process.
constexpr int NOALLOC_MAX_N = 512;
constexpr size_t NOALLOC_HEAD = 32;  // doubles reserved for flags, keeps the grid 256-byte aligned
constexpr size_t NOALLOC_DOUBLES = NOALLOC_HEAD + (size_t)NOALLOC_MAX_N * NOALLOC_MAX_N + 6 * (size_t)NOALLOC_MAX_N;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

__global__ void k_noalloc_tables(int N, double h, int neumann, double* tab, double* lam, double* tw, int* flag) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m == 0) *flag = 0;
  if (m < 4 * N) tab[m] = sinpi((double)m / (2.0 * N));
  if (m < N) {
    double sk = sinpi(((double)m + (neumann ? 0.0 : 1.0)) / (2.0 * N));
    lam[m] = -4.0 * sk * sk / (h * h);
  }
  if (m < N / 2) {
    double sn, cs;
    sincospi(2.0 * (double)m / (double)N, &sn, &cs);
    tw[2 * m] = cs;
    tw[2 * m + 1] = -sn;
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
  k_noalloc_tables<<<cdiv(4L * N, 256), 256, 0, s>>>(N, h, dct, tab, lam, tw, flag);
  size_t sm_row = sizeof(V2<double>) * N;
  k_row_dense<double><<<N / 2, 256, sm_row, s>>>(N, logN, dct, 0, (const V2<double>*)tw, tab, rhs, spec, nullptr);
  int CP = 2;
  if (2 * CP > N) CP = N / 2;
  int threads = 256;
  while (CP * (N / 2 + 1) > 8 * threads && threads < 1024) threads *= 2;
  size_t sm_col = sizeof(V2<double>) * (size_t)CP * N;
  k_col_solve<double><<<N / (2 * CP), threads, sm_col, s>>>(N, logN, CP, dct, (const V2<double>*)tw, tab, lam, kappa,
                                                             spec, flag);
  k_row_dense<double><<<N / 2, 256, sm_row, s>>>(N, logN, dct, 1, (const V2<double>*)tw, tab, nullptr, spec, u);
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

}  // namespace kfbi

extern "C" kfbi_status kfbi_grid_solve_noalloc(int N, double h, double kappa, int boxbc, const double* rhs, double* u,
                                               void* stream) {
  if (N < 16 || (N & (N - 1)) != 0 || rhs == nullptr || u == nullptr) return KFBI_ERR_ARG;
  if (N > kfbi::NOALLOC_MAX_N) return KFBI_ERR_CAPACITY;
  if (!(h > 0.0) || !(kappa >= 0.0) || boxbc < KFBI_BOX_DIRICHLET0 || boxbc > KFBI_BOX_FREESPACE_DL)
    return KFBI_ERR_ARG;
  if (boxbc == KFBI_BOX_NEUMANN0 && kappa == 0.0) return KFBI_ERR_SINGULAR;
  return kfbi::grid_solve_noalloc_impl(N, h, kappa, boxbc, rhs, u, (cudaStream_t)stream);
}
