// Learned warm start of GMRES: per-node interface features, a 47-H-H-1 ReLU network with
// bfloat16 weights and float32 accumulation, its hand-written backward pass and Adam.
// The paper solves each boundary integral equation by GMRES from a given initial density
// (Sec. 4); the network only supplies that initial density, GMRES still iterates to the
// requested tolerance.
//
// Parameters (float32 master copy, flat): W1 [H][F] | b1 [H] | W2 [H][H] | b2 [H] | w3 [H] | b3;
// the bfloat16 copies of W1, W2, w3 (refreshed by every Adam step) feed the kernels.
#include <cuda_bf16.h>

#include <cmath>

#include "kfbi_internal.cuh"

struct kfbi_mlp {
  int F = KFBI_MLP_FEATURES;
  int H = 0;
  int max_rows = 0;
  int P = 0;  // parameter count
  int oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, ow3 = 0, ob3 = 0;
  cudaStream_t stream = nullptr;
  float* master = nullptr;          // [P]
  __nv_bfloat16* wq = nullptr;      // [P] bfloat16 copy (only the W1, W2, w3 ranges are used)
  float* grad = nullptr;            // [P]
  float* adam_m = nullptr;          // [P]
  float* adam_v = nullptr;          // [P]
  float* h1 = nullptr;              // [max_rows][H] activations of layer 1 (training)
  float* h2 = nullptr;              // [max_rows][H]
  float* dz1 = nullptr;             // [max_rows][H]
  float* dz2 = nullptr;             // [max_rows][H]
  float* xg = nullptr;              // [max_rows][F] gathered inputs (training)
  float* dy = nullptr;              // [max_rows]
  float* y = nullptr;               // [max_rows]
  float* loss_part = nullptr;       // [max_rows / MLP_ROWS + 1]
  float* loss = nullptr;            // [1]
  float* host_loss = nullptr;       // pinned [1]
  float* feat = nullptr;            // [max_rows][F] features for kfbi_warmstart_predict
  double* scale = nullptr;          // [1] rms of the right-hand side
  int step = 0;                     // Adam steps taken
  bool tc = true;                   // the H x H layer on the tensor cores (kfbi_tc_gemm path)
  float* w2f = nullptr;             // [H][H] the bfloat16 W2 as float32 (tensor-core operand)
  float* z2 = nullptr;              // [max_rows][H] pre-activations of layer 2 (tensor-core path)
  int* tc_err = nullptr;            // [1] completion-wait flag of the tensor-core contractions
};

namespace kfbi {

constexpr int MLP_ROWS = 16;    // rows per block of the forward/backward kernels
constexpr int MLP_MAX_H = 256;  // hidden width limit (one thread per hidden unit)
constexpr int MLP_MAXF = 48;    // input width bound for the register copy of a W1 row

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// --------------------------------------------------------------------------- forward/backward
// One block of H threads handles MLP_ROWS rows; thread i owns hidden unit i of both layers.
// W1 row i lives in registers, W2 in shared memory (row stride H + 2 bfloat16, an odd number
// of 32-bit words, so that the row-wise reads of the forward pass and the column-wise reads
// of the backward pass are both free of bank conflicts).
//   forward:  z1 = W1 x + b1, h1 = relu(z1), z2 = W2 h1 + b2, h2 = relu(z2), y = w3.h2 + b3
//   backward: dy = 2 (y - t) / R, dz2 = dy w3 [z2 > 0], dz1 = (W2^T dz2) [z1 > 0]
// With target == nullptr only y is produced. rows of the input are idx[r] when idx != nullptr.
__global__ void __launch_bounds__(MLP_MAX_H) k_mlp_rows(int F, int H, const float* X, const int* idx, int rows,
                                                         const float* target, const __nv_bfloat16* wq,
                                                         const float* master, int oW1, int ob1, int oW2, int ob2,
                                                         int ow3, int ob3, float inv_rows, float* y, float* xg,
                                                         float* h1g, float* h2g, float* dz1g, float* dz2g, float* dyg,
                                                         float* loss_part) {
  extern __shared__ unsigned char smem_raw[];
  const int ld = H + 2;
  __nv_bfloat16* sW2 = (__nv_bfloat16*)smem_raw;                     // [H][ld]
  float* sx = (float*)(smem_raw + sizeof(__nv_bfloat16) * (size_t)H * ld);  // [MLP_ROWS][F]
  float* sh1 = sx + MLP_ROWS * F;                                     // [MLP_ROWS][H]
  float* sd = sh1 + MLP_ROWS * H;                                     // [MLP_ROWS][H] dz2
  __shared__ float red[MLP_ROWS][MLP_MAX_H / 32];
  __shared__ float sy[MLP_ROWS], sdy[MLP_ROWS];
  const int i = threadIdx.x;
  const int r0 = blockIdx.x * MLP_ROWS;
  const int nr = min(MLP_ROWS, rows - r0);
  for (int t = i; t < H * H; t += H) {
    const int a = t / H, b = t - a * H;
    sW2[a * ld + b] = wq[oW2 + t];
  }
  for (int t = i; t < nr * F; t += H) {
    const int r = t / F, f = t - r * F;
    const int row = idx != nullptr ? idx[r0 + r] : r0 + r;
    const float v = X[(long)row * F + f];
    sx[r * F + f] = v;
    if (xg != nullptr) xg[(long)(r0 + r) * F + f] = v;
  }
  float w1[MLP_MAXF];
#pragma unroll
  for (int f = 0; f < MLP_MAXF; ++f) w1[f] = f < F ? bf(wq[oW1 + i * F + f]) : 0.0f;
  const float b1 = master[ob1 + i], b2 = master[ob2 + i], w3 = bf(wq[ow3 + i]);
  __syncthreads();
  // layer 1
  float z1[MLP_ROWS];
#pragma unroll
  for (int r = 0; r < MLP_ROWS; ++r) {
    float a = b1;
    if (r < nr) {
#pragma unroll
      for (int f = 0; f < MLP_MAXF; ++f)
        if (f < F) a = fmaf(sx[r * F + f], w1[f], a);
    }
    z1[r] = a;
    sh1[r * H + i] = fmaxf(a, 0.0f);
  }
  __syncthreads();
  // layer 2: row i of W2 against the MLP_ROWS activations
  float z2[MLP_ROWS];
#pragma unroll
  for (int r = 0; r < MLP_ROWS; ++r) z2[r] = b2;
  const __nv_bfloat162* wrow = (const __nv_bfloat162*)(sW2 + i * ld);
  for (int k = 0; k < H; k += 2) {
    const float2 w = __bfloat1622float2(wrow[k >> 1]);
#pragma unroll
    for (int r = 0; r < MLP_ROWS; ++r) {
      const float2 h = *(const float2*)(sh1 + r * H + k);
      z2[r] = fmaf(h.x, w.x, fmaf(h.y, w.y, z2[r]));
    }
  }
  // layer 3: y = w3 . relu(z2) + b3 (warp shuffles, then across warps)
  const int lane = i & 31, wid = i >> 5, nw = H >> 5;
#pragma unroll
  for (int r = 0; r < MLP_ROWS; ++r) {
    float p = fmaxf(z2[r], 0.0f) * w3;
    for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
    if (lane == 0) red[r][wid] = p;
  }
  __syncthreads();
  if (i < MLP_ROWS) {
    float a = master[ob3];
    for (int q = 0; q < nw; ++q) a += red[i][q];
    sy[i] = a;
    if (i < nr) y[r0 + i] = a;
  }
  __syncthreads();
  if (target == nullptr) return;
  // backward
  if (i < MLP_ROWS) {
    float d = 0.0f, l = 0.0f;
    if (i < nr) {
      const int row = idx != nullptr ? idx[r0 + i] : r0 + i;
      const float e = sy[i] - target[row];
      d = 2.0f * e * inv_rows;
      l = e * e;
      dyg[r0 + i] = d;
    }
    sdy[i] = d;
    red[i][0] = l;
  }
  __syncthreads();
  if (i == 0) {
    float l = 0.0f;
    for (int r = 0; r < MLP_ROWS; ++r) l += red[r][0];
    loss_part[blockIdx.x] = l;
  }
#pragma unroll
  for (int r = 0; r < MLP_ROWS; ++r) {
    const float d2 = z2[r] > 0.0f ? sdy[r] * w3 : 0.0f;
    sd[r * H + i] = d2;
    if (r < nr) {
      h1g[(long)(r0 + r) * H + i] = sh1[r * H + i];
      h2g[(long)(r0 + r) * H + i] = fmaxf(z2[r], 0.0f);
      dz2g[(long)(r0 + r) * H + i] = d2;
    }
  }
  __syncthreads();
  // dz1[:, i] = (W2^T dz2)[i] [z1 > 0]: column i of W2
  float acc[MLP_ROWS];
#pragma unroll
  for (int r = 0; r < MLP_ROWS; ++r) acc[r] = 0.0f;
  for (int k = 0; k < H; ++k) {
    const float w = bf(sW2[k * ld + i]);
#pragma unroll
    for (int r = 0; r < MLP_ROWS; ++r) acc[r] = fmaf(sd[r * H + k], w, acc[r]);
  }
#pragma unroll
  for (int r = 0; r < MLP_ROWS; ++r)
    if (r < nr) dz1g[(long)(r0 + r) * H + i] = z1[r] > 0.0f ? acc[r] : 0.0f;
}

// --------------------------------------------------------------------------- weight gradients
// G[a][b] = sum_r A[r][a] B[r][b] for b < KB, and G[a][KB] = sum_r A[r][a] (bias column), over
// all rows in a fixed order: one block per 32 x 32 tile of G, rows in chunks of 32.
struct GradJob {
  const float* A;  // [rows][HA]
  const float* B;  // [rows][KB]
  int HA, KB;
  float* Gw;       // [HA][KB] weight gradient
  float* Gb;       // [HA] bias gradient
  int tiles_a, tiles_b, first_block;
};

__global__ void k_mlp_wgrad(GradJob j0, GradJob j1, GradJob j2, int rows) {
  const GradJob& J = blockIdx.x >= j2.first_block ? j2 : (blockIdx.x >= j1.first_block ? j1 : j0);
  const int t = blockIdx.x - J.first_block;
  const int ta = t / J.tiles_b, tb = t - ta * J.tiles_b;
  const int a0 = ta * 32, b0 = tb * 32;
  __shared__ float sA[32][33], sB[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 256 threads: ty = 0..7
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int rr = 0; rr < rows; rr += 32) {
    for (int q = ty; q < 32; q += 8) {
      const int r = rr + q;
      const int a = a0 + tx, b = b0 + tx;
      sA[q][tx] = (r < rows && a < J.HA) ? J.A[(long)r * J.HA + a] : 0.0f;
      sB[q][tx] = r < rows ? (b < J.KB ? J.B[(long)r * J.KB + b] : (b == J.KB ? 1.0f : 0.0f)) : 0.0f;
    }
    __syncthreads();
#pragma unroll 4
    for (int q = 0; q < 32; ++q) {
      const float bv = sB[q][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fmaf(sA[q][ty + 8 * u], bv, acc[u]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int a = a0 + ty + 8 * u, b = b0 + tx;
    if (a >= J.HA) continue;
    if (b < J.KB) J.Gw[(long)a * J.KB + b] = acc[u];
    else if (b == J.KB) J.Gb[a] = acc[u];
  }
}

// total loss (mean) from the per-block partials, fixed order
__global__ void k_mlp_loss(const float* part, int nb, float inv_rows, float* loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float l = 0.0f;
  for (int b = 0; b < nb; ++b) l += part[b];
  *loss = l * inv_rows;
}

// --------------------------------------------------------------------------- Adam
// m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps);
// the bfloat16 copy of the weights is refreshed from the new master value.
__global__ void k_mlp_adam(int P, float* p, const float* g, float* m, float* v, __nv_bfloat16* wq, float lr,
                           float beta1, float beta2, float eps, float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  const float gk = g[k];
  const float mk = beta1 * m[k] + (1.0f - beta1) * gk;
  const float vk = beta2 * v[k] + (1.0f - beta2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  const float pk = p[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
  p[k] = pk;
  wq[k] = __float2bfloat16_rn(pk);
}

__global__ void k_mlp_quantise(int P, const float* p, __nv_bfloat16* wq) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < P) wq[k] = __float2bfloat16_rn(p[k]);
}

// --------------------------------------------------------------------------- features
// One block per interface. Node geometry from the float64 target data; float32 arithmetic.
// Features of node j: rotated curvature modes khat_k e^{i k alpha_j} l (k < 16, Re and Im),
// kappa_j l, normal, s_j / L (trapezoidal), g_j / rms(g), centred position / l, l = L / 2 pi,
// rotated data modes ghat_k e^{i k alpha_j} / rms(g) (k < 4).
constexpr int FEAT_THREADS = 1024;
constexpr int FEAT_MAX_N = 8192;

__global__ void __launch_bounds__(FEAT_THREADS) k_ws_features(int n, const TargetGeo* geo, const double* xy,
                                                               const double2* twn, const double* rhs, float* feat,
                                                               double* scale) {
  extern __shared__ float fsm[];
  float* kap = fsm;        // [n]
  float* sa = kap + n;     // [n]
  float* cum = sa + n;     // [n] arclength at node j
  __shared__ float red[4][FEAT_THREADS / 32];
  __shared__ float modes[2 * KFBI_MLP_MODES];
  __shared__ float gmodes[2 * KFBI_MLP_DATA_MODES];
  __shared__ float tot[4];
  __shared__ float chunk_tot[FEAT_THREADS];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  float s_sa = 0.0f, s_x = 0.0f, s_y = 0.0f, s_g = 0.0f;
  for (int j = tid; j < n; j += FEAT_THREADS) {
    const TargetGeo& g = geo[j];
    const float xa = (float)g.xa, ya = (float)g.ya, xaa = (float)g.xaa, yaa = (float)g.yaa, s = (float)g.sa;
    kap[j] = (xa * yaa - ya * xaa) / (s * s * s);
    sa[j] = s;
    s_sa += s;
    s_x += (float)xy[2 * j];
    s_y += (float)xy[2 * j + 1];
    const float gj = (float)rhs[j];
    s_g += gj * gj;
  }
  float v[4] = {s_sa, s_x, s_y, s_g};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float a = v[q];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) red[q][wid] = a;
  }
  __syncthreads();
  if (tid < 4) {
    float a = 0.0f;
    for (int q = 0; q < FEAT_THREADS / 32; ++q) a += red[tid][q];
    tot[tid] = a;
  }
  // curvature modes khat_k = (1/n) sum_m kappa_m e^{-i k alpha_m}: warp k
  if (wid < KFBI_MLP_MODES) {
    const int k = wid;
    float re = 0.0f, im = 0.0f;
    for (int m = lane; m < n; m += 32) {
      const double2 e = twn[((long)k * m) % n];
      re += kap[m] * (float)e.x;
      im -= kap[m] * (float)e.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
      modes[2 * k] = re / (float)n;
      modes[2 * k + 1] = im / (float)n;
    }
  } else if (wid < KFBI_MLP_MODES + KFBI_MLP_DATA_MODES) {
    // data modes ghat_k = (1/n) sum_m g_m e^{-i k alpha_m}
    const int k = wid - KFBI_MLP_MODES;
    float re = 0.0f, im = 0.0f;
    for (int m = lane; m < n; m += 32) {
      const double2 e = twn[((long)k * m) % n];
      const float gm = (float)rhs[m];
      re += gm * (float)e.x;
      im -= gm * (float)e.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
      gmodes[2 * k] = re / (float)n;
      gmodes[2 * k + 1] = im / (float)n;
    }
  }
  // arclength at the nodes: trapezoidal increments, scanned over contiguous chunks
  const int per = (n + FEAT_THREADS - 1) / FEAT_THREADS;
  const int b = tid * per, e = min(n, b + per);
  const float dal = 2.0f * 3.14159265358979f / (float)n;
  float run = 0.0f;
  for (int j = b; j < e; ++j)
    if (j + 1 < n) run += 0.5f * (sa[j] + sa[j + 1]) * dal;
  chunk_tot[tid] = run;
  __syncthreads();
  if (tid == 0) {
    float a = 0.0f;
    for (int q = 0; q < FEAT_THREADS; ++q) {
      const float c = chunk_tot[q];
      chunk_tot[q] = a;
      a += c;
    }
  }
  __syncthreads();
  run = chunk_tot[tid];
  for (int j = b; j < e; ++j) {
    cum[j] = run;
    if (j + 1 < n) run += 0.5f * (sa[j] + sa[j + 1]) * dal;
  }
  __syncthreads();
  const float L = tot[0] * dal;
  const float ell = L / (2.0f * 3.14159265358979f);
  const float xm = tot[1] / (float)n, ym = tot[2] / (float)n;
  const float rms = sqrtf(tot[3] / (float)n);
  if (tid == 0) *scale = (double)rms;
  for (int j = tid; j < n; j += FEAT_THREADS) {
    float* o = feat + (long)j * KFBI_MLP_FEATURES;
    for (int k = 0; k < KFBI_MLP_MODES; ++k) {
      const double2 e = twn[((long)k * j) % n];
      const float c = (float)e.x, s = (float)e.y;
      const float mr = modes[2 * k], mi = modes[2 * k + 1];
      o[2 * k] = (mr * c - mi * s) * ell;
      o[2 * k + 1] = (mr * s + mi * c) * ell;
    }
    const TargetGeo& g = geo[j];
    const float xa = (float)g.xa, ya = (float)g.ya;
    o[32] = kap[j] * ell;
    o[33] = ya / sa[j];
    o[34] = -xa / sa[j];
    o[35] = cum[j] / L;
    o[36] = rms > 0.0f ? (float)rhs[j] / rms : 0.0f;
    o[37] = ((float)xy[2 * j] - xm) / ell;
    o[38] = ((float)xy[2 * j + 1] - ym) / ell;
    for (int k = 0; k < KFBI_MLP_DATA_MODES; ++k) {
      const double2 e = twn[((long)k * j) % n];
      const float c = (float)e.x, s = (float)e.y;
      const float mr = gmodes[2 * k], mi = gmodes[2 * k + 1];
      const float inv = rms > 0.0f ? 1.0f / rms : 0.0f;
      o[39 + 2 * k] = (mr * c - mi * s) * inv;
      o[40 + 2 * k] = (mr * s + mi * c) * inv;
    }
  }
}

// density = scale * y (float64 output)
__global__ void k_ws_scale(int n, const float* y, const double* scale, double* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = *scale * (double)y[j];
}

// --------------------------------------------------------------------------- tensor-core path
// The same network with its H x H layer as a tensor-core contraction (kfbi_gemm.cu):
//   layer 1 (k_mlp_l1):   z1 = W1 x + b1, h1 = relu(z1), x gathered by idx
//   layer 2 (tc_gemm):    z2 = h1 W2^T (W2 as the float32 value of its bfloat16 copy)
//   layer 3 (k_mlp_l3):   h2 = relu(z2 + b2), y = w3.h2 + b3; training: dy, dz2 = dy w3 [z2 > 0]
//   backward (tc_gemm):   dz1 = (dz2 W2) [h1 > 0];  dW2 = dz2^T h1 (tc_gemm over the rows)
// The remaining gradients (W1, b1, b2, w3, b3) and the loss come from k_mlp_wgrad / k_mlp_loss.
__global__ void k_mlp_l1(int F, int H, const float* X, const int* idx, int rows, const __nv_bfloat16* wq,
                         const float* master, int oW1, int ob1, float* xg, float* h1) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)rows * H) return;
  const int r = (int)(t / H), i = (int)(t - (long)r * H);
  const int row = idx != nullptr ? idx[r] : r;
  const float* x = X + (long)row * F;
  float a = master[ob1 + i];
  for (int f = 0; f < F; ++f) a = fmaf(x[f], bf(wq[oW1 + i * F + f]), a);
  h1[t] = fmaxf(a, 0.0f);
  if (xg != nullptr)
    for (int f = i; f < F; f += H) xg[(long)r * F + f] = x[f];
}

// one warp per row: h2 = relu(z2 + b2), y = w3 . h2 + b3; with a target also the loss part,
// dy = 2 (y - t) / R and dz2 = dy w3 [z2 > 0]
__global__ void k_mlp_l3(int H, const float* z2, int rows, const float* target, const int* idx,
                         const __nv_bfloat16* wq, const float* master, int ob2, int ow3, int ob3, float inv_rows,
                         float* y, float* h2g, float* dz2g, float* dyg, float* loss_row) {
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (r >= rows) return;
  const float* z = z2 + (long)r * H;
  float acc = 0.0f;
  for (int a = lane; a < H; a += 32) {
    const float h = fmaxf(z[a] + master[ob2 + a], 0.0f);
    acc = fmaf(h, bf(wq[ow3 + a]), acc);
    if (h2g != nullptr) h2g[(long)r * H + a] = h;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  const float yr = acc + master[ob3];
  if (lane == 0) y[r] = yr;
  if (target == nullptr) return;
  const int row = idx != nullptr ? idx[r] : r;
  const float e = yr - target[row];
  const float d = 2.0f * e * inv_rows;
  if (lane == 0) {
    dyg[r] = d;
    loss_row[r] = e * e;
  }
  for (int a = lane; a < H; a += 32) {
    const float zz = z[a] + master[ob2 + a];
    dz2g[(long)r * H + a] = zz > 0.0f ? d * bf(wq[ow3 + a]) : 0.0f;
  }
}

__global__ void k_mlp_relu_mask(long count, const float* h1, float* dz1) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count && !(h1[t] > 0.0f)) dz1[t] = 0.0f;
}

__global__ void k_mlp_w2f(int count, const __nv_bfloat16* w, float* f) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) f[t] = bf(w[t]);
}

// loss over the rows in a fixed order (tensor-core path: one loss value per row)
__global__ void k_mlp_loss_rows(const float* per_row, int rows, float inv_rows, float* loss) {
  __shared__ float sh[32];
  float a = 0.0f;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) a += per_row[r];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    *loss = t * inv_rows;
  }
}

// --------------------------------------------------------------------------- host side
static size_t rows_smem_h(int F, int H) {
  return sizeof(__nv_bfloat16) * (size_t)H * (H + 2) + sizeof(float) * ((size_t)MLP_ROWS * F + 2 * (size_t)MLP_ROWS * H);
}
static size_t rows_smem(const kfbi_mlp* m) { return rows_smem_h(m->F, m->H); }
// the kernel's shared-memory limit is process-wide: set for the widest network
static size_t rows_smem_max() { return rows_smem_h(KFBI_MLP_FEATURES, MLP_MAX_H); }

static TcGemmArgs tc_args(kfbi_mlp* m) {
  TcGemmArgs g;
  g.terms = 3;
  g.error = m->tc_err;
  return g;
}

// forward (and, with a target, the per-row backward quantities) through the tensor-core layer
static kfbi_status run_rows_tc(kfbi_mlp* m, const float* X, const int* idx, int rows, const float* target, float* y) {
  const int H = m->H, F = m->F;
  const bool train = target != nullptr;
  k_mlp_l1<<<cdiv((long)rows * H, 256), 256, 0, m->stream>>>(F, H, X, idx, rows, m->wq, m->master, m->oW1, m->ob1,
                                                             train ? m->xg : nullptr, m->h1);
  TcGemmArgs g = tc_args(m);
  g.terms = 4;  // W2 is exact in bfloat16: h1 carried to float32 accuracy
  g.A = m->h1;
  g.lda = H;
  g.B = m->w2f;
  g.ldb = H;
  g.C = m->z2;
  g.ldc = H;
  g.M = rows;
  g.N = H;
  g.K = H;
  KFBI_CHECK(tc_gemm(g, m->stream));
  k_mlp_l3<<<cdiv((long)rows * 32, 256), 256, 0, m->stream>>>(
      H, m->z2, rows, target, idx, m->wq, m->master, m->ob2, m->ow3, m->ob3, 1.0f / (float)rows, y,
      train ? m->h2 : nullptr, m->dz2, m->dy, m->loss_part);
  if (train) {
    // dz1 = (dz2 W2) [h1 > 0]: B(n = b, k = a) = W2[a][b]
    TcGemmArgs b = tc_args(m);
    b.terms = 4;
    b.A = m->dz2;
    b.lda = H;
    b.B = m->w2f;
    b.ldb = H;
    b.transB = 1;
    b.C = m->dz1;
    b.ldc = H;
    b.M = rows;
    b.N = H;
    b.K = H;
    KFBI_CHECK(tc_gemm(b, m->stream));
    k_mlp_relu_mask<<<cdiv((long)rows * H, 256), 256, 0, m->stream>>>((long)rows * H, m->h1, m->dz1);
  }
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

static kfbi_status run_rows(kfbi_mlp* m, const float* X, const int* idx, int rows, const float* target, float* y) {
  if (m->tc) return run_rows_tc(m, X, idx, rows, target, y);
  const int nb = cdiv(rows, MLP_ROWS);
  const bool train = target != nullptr;
  k_mlp_rows<<<nb, m->H, rows_smem(m), m->stream>>>(
      m->F, m->H, X, idx, rows, target, m->wq, m->master, m->oW1, m->ob1, m->oW2, m->ob2, m->ow3, m->ob3,
      1.0f / (float)rows, y, train ? m->xg : nullptr, m->h1, m->h2, m->dz1, m->dz2, m->dy, m->loss_part);
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

static kfbi_status run_grads(kfbi_mlp* m, const float* X, const float* target, const int* idx, int rows,
                             float* grad) {
  KFBI_CHECK(run_rows(m, X, idx, rows, target, m->y));
  const int H = m->H, F = m->F;
  if (m->tc) {
    // dW2[a][b] = sum_r dz2[r][a] h1[r][b] on the tensor cores; b2, W1, b1, w3, b3 below
    TcGemmArgs g = tc_args(m);
    g.A = m->dz2;
    g.lda = H;
    g.transA = 1;
    g.B = m->h1;
    g.ldb = H;
    g.transB = 1;
    g.C = grad + m->oW2;
    g.ldc = H;
    g.M = H;
    g.N = H;
    g.K = rows;
    KFBI_CHECK(tc_gemm(g, m->stream));
    GradJob j0{m->dz2, m->h1, H, 0, grad + m->oW2, grad + m->ob2, cdiv(H, 32), 1, 0};  // bias column only
    GradJob j1{m->dz1, m->xg, H, F, grad + m->oW1, grad + m->ob1, cdiv(H, 32), cdiv(F + 1, 32), 0};
    GradJob j2{m->dy, m->h2, 1, H, grad + m->ow3, grad + m->ob3, 1, cdiv(H + 1, 32), 0};
    j1.first_block = j0.tiles_a * j0.tiles_b;
    j2.first_block = j1.first_block + j1.tiles_a * j1.tiles_b;
    const int blocks = j2.first_block + j2.tiles_a * j2.tiles_b;
    k_mlp_wgrad<<<blocks, 256, 0, m->stream>>>(j0, j1, j2, rows);
    k_mlp_loss_rows<<<1, 1024, 0, m->stream>>>(m->loss_part, rows, 1.0f / (float)rows, m->loss);
    KFBI_TRY(cudaGetLastError());
    return KFBI_OK;
  }
  GradJob j0{m->dz2, m->h1, H, H, grad + m->oW2, grad + m->ob2, cdiv(H, 32), cdiv(H + 1, 32), 0};
  GradJob j1{m->dz1, m->xg, H, F, grad + m->oW1, grad + m->ob1, cdiv(H, 32), cdiv(F + 1, 32), 0};
  GradJob j2{m->dy, m->h2, 1, H, grad + m->ow3, grad + m->ob3, 1, cdiv(H + 1, 32), 0};
  j1.first_block = j0.tiles_a * j0.tiles_b;
  j2.first_block = j1.first_block + j1.tiles_a * j1.tiles_b;
  const int blocks = j2.first_block + j2.tiles_a * j2.tiles_b;
  k_mlp_wgrad<<<blocks, 256, 0, m->stream>>>(j0, j1, j2, rows);
  k_mlp_loss<<<1, 32, 0, m->stream>>>(m->loss_part, cdiv(rows, MLP_ROWS), 1.0f / (float)rows, m->loss);
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

static kfbi_status read_loss(kfbi_mlp* m, float* loss) {
  if (loss == nullptr) return KFBI_OK;
  KFBI_TRY(cudaMemcpyAsync(m->host_loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
  KFBI_TRY(cudaStreamSynchronize(m->stream));
  *loss = *m->host_loss;
  return KFBI_OK;
}

}  // namespace kfbi

using namespace kfbi;

static void mlp_free(kfbi_mlp* m) {
  void* ptrs[] = {m->master, m->wq, m->grad, m->adam_m, m->adam_v, m->h1, m->h2, m->dz1, m->dz2, m->xg,
                  m->dy, m->y, m->loss_part, m->loss, m->feat, m->scale, m->w2f, m->z2, m->tc_err};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (m->host_loss) cudaFreeHost(m->host_loss);
  delete m;
}

template <typename T>
static kfbi_status mlp_alloc(T** p, size_t count) {
  KFBI_TRY(cudaMalloc((void**)p, sizeof(T) * (count > 0 ? count : 1)));
  KFBI_TRY(cudaMemset(*p, 0, sizeof(T) * (count > 0 ? count : 1)));
  return KFBI_OK;
}

extern "C" {

kfbi_status kfbi_mlp_create(int hidden, int max_rows, kfbi_mlp** out) {
  if (out == nullptr || hidden < 32 || hidden > MLP_MAX_H || hidden % 32 != 0 || max_rows < 1) return KFBI_ERR_ARG;
  *out = nullptr;
  kfbi_mlp* m = new kfbi_mlp();
  m->H = hidden;
  m->max_rows = max_rows;
  const int F = m->F, H = hidden;
  m->oW1 = 0;
  m->ob1 = H * F;
  m->oW2 = m->ob1 + H;
  m->ob2 = m->oW2 + H * H;
  m->ow3 = m->ob2 + H;
  m->ob3 = m->ow3 + H;
  m->P = m->ob3 + 1;
  const size_t P = m->P, R = max_rows;
  kfbi_status st = KFBI_OK;
  if ((st = mlp_alloc(&m->master, P)) != KFBI_OK || (st = mlp_alloc(&m->wq, P)) != KFBI_OK ||
      (st = mlp_alloc(&m->grad, P)) != KFBI_OK || (st = mlp_alloc(&m->adam_m, P)) != KFBI_OK ||
      (st = mlp_alloc(&m->adam_v, P)) != KFBI_OK || (st = mlp_alloc(&m->h1, R * H)) != KFBI_OK ||
      (st = mlp_alloc(&m->h2, R * H)) != KFBI_OK || (st = mlp_alloc(&m->dz1, R * H)) != KFBI_OK ||
      (st = mlp_alloc(&m->dz2, R * H)) != KFBI_OK || (st = mlp_alloc(&m->xg, R * F)) != KFBI_OK ||
      (st = mlp_alloc(&m->dy, R)) != KFBI_OK || (st = mlp_alloc(&m->y, R)) != KFBI_OK ||
      (st = mlp_alloc(&m->loss_part, R + 1)) != KFBI_OK || (st = mlp_alloc(&m->loss, 1)) != KFBI_OK ||
      (st = mlp_alloc(&m->feat, R * F)) != KFBI_OK || (st = mlp_alloc(&m->scale, 1)) != KFBI_OK ||
      (st = mlp_alloc(&m->w2f, (size_t)H * H)) != KFBI_OK || (st = mlp_alloc(&m->z2, R * H)) != KFBI_OK ||
      (st = mlp_alloc(&m->tc_err, 1)) != KFBI_OK) {
    mlp_free(m);
    return st;
  }
  cudaError_t e = cudaMallocHost((void**)&m->host_loss, sizeof(float));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_mlp_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_smem_max());
  if (e != cudaSuccess) {
    note_cuda_error(e, "kfbi_mlp_create", __FILE__, __LINE__);
    mlp_free(m);
    return KFBI_ERR_CUDA;
  }
  *out = m;
  return KFBI_OK;
}

void kfbi_mlp_destroy(kfbi_mlp* m) {
  if (m == nullptr) return;
  cudaStreamSynchronize(m->stream);
  mlp_free(m);
}

kfbi_status kfbi_mlp_set_stream(kfbi_mlp* m, void* stream) {
  if (m == nullptr) return KFBI_ERR_ARG;
  m->stream = (cudaStream_t)stream;
  return KFBI_OK;
}

kfbi_status kfbi_mlp_set_tensor_cores(kfbi_mlp* m, int enable) {
  if (m == nullptr) return KFBI_ERR_ARG;
  KFBI_TRY(cudaStreamSynchronize(m->stream));
  m->tc = enable != 0;
  if (m->tc) {
    k_mlp_w2f<<<cdiv(m->H * m->H, 256), 256, 0, m->stream>>>(m->H * m->H, m->wq + m->oW2, m->w2f);
    KFBI_TRY(cudaGetLastError());
  }
  return KFBI_OK;
}

kfbi_status kfbi_mlp_tc_error(kfbi_mlp* m, int* flag) {
  if (m == nullptr || flag == nullptr) return KFBI_ERR_ARG;
  KFBI_TRY(cudaMemcpyAsync(flag, m->tc_err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  KFBI_TRY(cudaStreamSynchronize(m->stream));
  return KFBI_OK;
}

kfbi_status kfbi_mlp_param_count(kfbi_mlp* m, int* count) {
  if (m == nullptr || count == nullptr) return KFBI_ERR_ARG;
  *count = m->P;
  return KFBI_OK;
}

kfbi_status kfbi_mlp_set_params(kfbi_mlp* m, const float* params) {
  if (m == nullptr || params == nullptr) return KFBI_ERR_ARG;
  const size_t bytes = sizeof(float) * m->P;
  KFBI_TRY(cudaMemcpyAsync(m->master, params, bytes, cudaMemcpyHostToDevice, m->stream));
  KFBI_TRY(cudaMemsetAsync(m->adam_m, 0, bytes, m->stream));
  KFBI_TRY(cudaMemsetAsync(m->adam_v, 0, bytes, m->stream));
  k_mlp_quantise<<<cdiv(m->P, 256), 256, 0, m->stream>>>(m->P, m->master, m->wq);
  k_mlp_w2f<<<cdiv(m->H * m->H, 256), 256, 0, m->stream>>>(m->H * m->H, m->wq + m->oW2, m->w2f);
  KFBI_TRY(cudaGetLastError());
  KFBI_TRY(cudaStreamSynchronize(m->stream));
  m->step = 0;
  return KFBI_OK;
}

kfbi_status kfbi_mlp_get_params(kfbi_mlp* m, float* params) {
  if (m == nullptr || params == nullptr) return KFBI_ERR_ARG;
  KFBI_TRY(cudaMemcpyAsync(params, m->master, sizeof(float) * m->P, cudaMemcpyDeviceToHost, m->stream));
  KFBI_TRY(cudaStreamSynchronize(m->stream));
  return KFBI_OK;
}

kfbi_status kfbi_mlp_forward(kfbi_mlp* m, const float* feat, int rows, float* y) {
  if (m == nullptr || feat == nullptr || y == nullptr || rows < 1 || rows > m->max_rows) return KFBI_ERR_ARG;
  return run_rows(m, feat, nullptr, rows, nullptr, y);
}

kfbi_status kfbi_mlp_gradients(kfbi_mlp* m, const float* feat, const float* target, const int* idx, int rows,
                               float* grad, float* loss) {
  if (m == nullptr || feat == nullptr || target == nullptr || rows < 1 || rows > m->max_rows) return KFBI_ERR_ARG;
  KFBI_CHECK(run_grads(m, feat, target, idx, rows, grad != nullptr ? grad : m->grad));
  return read_loss(m, loss);
}

kfbi_status kfbi_mlp_train_step(kfbi_mlp* m, const float* feat, const float* target, const int* idx, int rows,
                                float lr, float* loss) {
  if (m == nullptr || feat == nullptr || target == nullptr || rows < 1 || rows > m->max_rows || !(lr > 0.0f))
    return KFBI_ERR_ARG;
  KFBI_CHECK(run_grads(m, feat, target, idx, rows, m->grad));
  m->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)m->step), c2 = 1.0f - powf(b2, (float)m->step);
  k_mlp_adam<<<cdiv(m->P, 256), 256, 0, m->stream>>>(m->P, m->master, m->grad, m->adam_m, m->adam_v, m->wq, lr, b1,
                                                     b2, 1e-8f, c1, c2);
  if (m->tc) k_mlp_w2f<<<cdiv(m->H * m->H, 256), 256, 0, m->stream>>>(m->H * m->H, m->wq + m->oW2, m->w2f);
  KFBI_TRY(cudaGetLastError());
  return read_loss(m, loss);
}

kfbi_status kfbi_warmstart_features(kfbi_ctx* c, const double* rhs, float* feat, double* scale) {
  if (c == nullptr || rhs == nullptr || feat == nullptr || scale == nullptr) return KFBI_ERR_ARG;
  if (!c->have_iface) return KFBI_ERR_STATE;
  const int n = c->n;
  if (n > FEAT_MAX_N) return KFBI_ERR_CAPACITY;
  const size_t smem = sizeof(float) * 3 * (size_t)n;
  KFBI_TRY(cudaFuncSetAttribute(k_ws_features, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(float) * 3 * (size_t)FEAT_MAX_N)));
  KFBI_TRY(stream_enter(c));
  launched(c, 1);
  k_ws_features<<<1, FEAT_THREADS, smem, c->stream>>>(n, c->tgeo + c->n_cross, c->xy, (const double2*)c->twn, rhs,
                                                     feat, scale);
  KFBI_TRY(cudaGetLastError());
  KFBI_TRY(stream_exit(c));
  return KFBI_OK;
}

kfbi_status kfbi_warmstart_predict(kfbi_ctx* c, kfbi_mlp* m, const double* rhs, double* density) {
  if (c == nullptr || m == nullptr || rhs == nullptr || density == nullptr) return KFBI_ERR_ARG;
  if (!c->have_iface) return KFBI_ERR_STATE;
  const int n = c->n;
  if (n > m->max_rows || n > FEAT_MAX_N) return KFBI_ERR_CAPACITY;
  const size_t smem = sizeof(float) * 3 * (size_t)n;
  KFBI_TRY(cudaFuncSetAttribute(k_ws_features, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(float) * 3 * (size_t)FEAT_MAX_N)));
  // features, network and scaling all run on the context's stream
  KFBI_TRY(stream_enter(c));
  launched(c, 3);
  k_ws_features<<<1, FEAT_THREADS, smem, c->stream>>>(n, c->tgeo + c->n_cross, c->xy, (const double2*)c->twn, rhs,
                                                     m->feat, m->scale);
  cudaStream_t saved = m->stream;
  m->stream = c->stream;
  kfbi_status st = run_rows(m, m->feat, nullptr, n, nullptr, m->y);
  m->stream = saved;
  KFBI_CHECK(st);
  k_ws_scale<<<cdiv(n, 256), 256, 0, c->stream>>>(n, m->y, m->scale, density);
  KFBI_TRY(cudaGetLastError());
  KFBI_TRY(stream_exit(c));
  return KFBI_OK;
}

}  // extern "C"
