// Matrix-free restarted GMRES on the device (Sec. 4: one operator apply per iteration).
//
// The solve runs as a sequence of identical "bodies": one operator apply on the vector
// `gin`, followed by five small kernels that advance a device-side state machine
// (GmresCtl). In the Arnoldi phase a body orthogonalises w = A v_j against V[0..j] by two
// passes of classical Gram-Schmidt, appends the Hessenberg column, applies the Givens
// rotations and decides whether the cycle ends; at the end of a cycle it solves the
// small triangular system and updates x, and the next body's apply evaluates A x for the
// true residual, which decides convergence or a restart. Every decision is taken on the
// device; the host only enqueues bodies and polls the `done` flag between chunks. Once
// done, every kernel of a further body returns at entry (the apply kernels read the same
// flag), so extra bodies cost only their launches.
#include <cmath>
#include <cstddef>
#include <vector>

#include "kfbi_internal.cuh"

namespace kfbi {

enum : int { ACT_NONE = 0, ACT_NEXT_V = 1, ACT_UPDATE_X = 2, ACT_RESTART = 3 };

constexpr int GM_BLOCKS = 32;
constexpr int GM_THREADS = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
  }
  return t;  // valid in warp 0
}

// returns true in the one block that arrives last (all partials are visible to it)
__device__ __forceinline__ bool last_block(int* ticket) {
  __shared__ int is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = atomicAdd(ticket, 1);
    is_last = (t == (int)gridDim.x - 1);
  }
  __syncthreads();
  if (is_last) {
    __threadfence();
    if (threadIdx.x == 0) *ticket = 0;
  }
  return is_last;
}

__global__ void k_gm_init(GmresCtl* ctl, double tol, int max_iter, int m, int trust) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ctl->phase = PH_RESID;
  ctl->next_phase = PH_RESID;
  ctl->done = 0;
  ctl->action = ACT_NONE;
  ctl->j = 0;
  ctl->k_end = 0;
  ctl->its = 0;
  ctl->cycles = 0;
  ctl->max_iter = max_iter;
  ctl->m = m;
  ctl->status = KFBI_OK;
  ctl->ticket = 0;
  ctl->breakdown = 0;
  ctl->trust = trust;
  ctl->bodies = 0;
  ctl->tol = tol;
  ctl->bnorm = 0.0;
  ctl->beta = 0.0;
  ctl->hnorm = 0.0;
  ctl->res_est = 0.0;
}

// ||b||; with a zero initial guess the first Arnoldi vector is b / ||b|| (r = b needs no
// apply), otherwise gin = x and the first body evaluates A x for the initial residual
__global__ void k_gm_start(const double* b, double* x, double* gin, float* gin_f, double* V, float* Vf, int n,
                           GmresCtl* ctl, int zero_guess) {
  __shared__ double sh[32];
  __shared__ double bn;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += b[i] * b[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    bn = sqrt(s);
    ctl->bnorm = bn;
    if (s == 0.0) {
      ctl->phase = PH_DONE;
      ctl->status = KFBI_OK;
      ctl->done = 1;
    } else if (zero_guess) {
      ctl->beta = bn;
      ctl->g[0] = bn;
      for (int k = 1; k <= ctl->m; ++k) ctl->g[k] = 0.0;
      ctl->phase = PH_ARNOLDI;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double g;
    if (bn == 0.0) {
      x[i] = 0.0;
      g = 0.0;
    } else if (zero_guess) {
      x[i] = 0.0;
      g = b[i] / bn;
      V[i] = g;
      if (Vf) Vf[i] = (float)g;
    } else {
      g = x[i];
    }
    gin[i] = g;
    gin_f[i] = (float)g;
  }
}

// Gram-Schmidt coefficients (Arnoldi phase): block k computes h_k = V[k] . w for k <= j and
// accumulates it into the Hessenberg column (pass 0 sets, pass 1 adds). Residual phase
// (pass 0 only): r = b - A x split over the blocks, then ||r|| and the restart decision in
// the last block.
__global__ void k_gm_dots(GmresCtl* ctl, const double* V, int ldv, const double* w, const double* b, double* r,
                          int n, double* part, int pass) {
  if (ctl->done) return;
  __shared__ double sh[32];
  const int phase = ctl->phase;
  if (phase == PH_ARNOLDI) {
    const int j = ctl->j;
    const int k = blockIdx.x;
    if (k > j) return;
    const double* v = V + (long)k * ldv;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i] * w[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
      ctl->hcol[k] = s;
      double* Hc = ctl->H + (long)j * (ctl->m + 1);
      Hc[k] = pass == 0 ? s : Hc[k] + s;
    }
  } else if (phase == PH_RESID) {
    if (pass != 0) return;
    const int per = (n + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * per, i1 = min(n, i0 + per);
    double s = 0.0;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      double ri = b[i] - w[i];
      r[i] = ri;
      s += ri * ri;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x * (MAX_RESTART + 1)] = s;
    if (last_block(&ctl->ticket) && threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < (int)gridDim.x; ++q) t += part[q * (MAX_RESTART + 1)];
      double beta = sqrt(t);
      ctl->beta = beta;
      if (beta <= ctl->tol * ctl->bnorm) {
        ctl->status = KFBI_OK;
        ctl->next_phase = PH_DONE;
        ctl->action = ACT_NONE;
      } else if (ctl->its >= ctl->max_iter) {
        ctl->status = KFBI_ERR_NOT_CONVERGED;
        ctl->next_phase = PH_DONE;
        ctl->action = ACT_NONE;
      } else {
        ctl->g[0] = beta;
        for (int k = 1; k <= ctl->m; ++k) ctl->g[k] = 0.0;
        ctl->j = 0;
        ctl->next_phase = PH_ARNOLDI;
        ctl->action = ACT_RESTART;
      }
    }
  }
}

// w -= V[0..j] hcol over chunks of 32 entries: warp q of the block sums the Krylov vectors
// k = q, q + UPD_WARPS, ...; on the second pass also the partial ||w||^2 and, in the last block, the
// Hessenberg column, the Givens rotations and the end-of-cycle decision
constexpr int UPD_WARPS = 32;
__global__ void k_gm_update(GmresCtl* ctl, const double* V, int ldv, double* w, int n, double* part, int pass) {
  if (ctl->done) return;
  if (ctl->phase != PH_ARNOLDI) return;
  __shared__ double sh[32];
  __shared__ double hc[MAX_RESTART + 1];
  __shared__ double red[UPD_WARPS][33];
  const int j = ctl->j;
  for (int k = threadIdx.x; k <= j; k += blockDim.x) hc[k] = ctl->hcol[k];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  double acc = 0.0;
  if (i < n)
    for (int k = wid; k <= j; k += UPD_WARPS) acc += V[(long)k * ldv + i] * hc[k];
  red[wid][lane] = acc;
  __syncthreads();
  double s = 0.0;
  if (wid == 0 && i < n) {
    double tot = 0.0;
    for (int q = 0; q < UPD_WARPS; ++q) tot += red[q][lane];
    double v = w[i] - tot;
    w[i] = v;
    s = v * v;
  }
  if (pass == 0) return;
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x * (MAX_RESTART + 1)] = s;
  if (!last_block(&ctl->ticket)) return;
  // last block: Hessenberg column, Givens rotations, end-of-cycle decision. The column and
  // the rotations are staged in shared memory so the serial parts run from on-chip memory.
  __shared__ double scs[MAX_RESTART], ssn[MAX_RESTART], hcol[MAX_RESTART + 2];
  __shared__ int s_end;
  const int m = ctl->m;
  double* Hc = ctl->H + (long)j * (m + 1);
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    scs[i] = ctl->cs[i];
    ssn[i] = ctl->sn[i];
  }
  for (int i = threadIdx.x; i <= j; i += blockDim.x) hcol[i] = Hc[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)gridDim.x; ++q) t += part[q * (MAX_RESTART + 1)];
    double hn = sqrt(t);
    ctl->hnorm = hn;
    hcol[j + 1] = hn;
    int breakdown = hn == 0.0;
    for (int i = 0; i < j; ++i) {
      double a = hcol[i], bb = hcol[i + 1];
      hcol[i] = scs[i] * a + ssn[i] * bb;
      hcol[i + 1] = -ssn[i] * a + scs[i] * bb;
    }
    double den = hypot(hcol[j], hcol[j + 1]);
    double cj = hcol[j] / den, sj = hcol[j + 1] / den;
    ctl->cs[j] = cj;
    ctl->sn[j] = sj;
    hcol[j] = den;
    hcol[j + 1] = 0.0;
    double gj = ctl->g[j];
    ctl->g[j + 1] = -sj * gj;
    ctl->g[j] = cj * gj;
    ctl->its += 1;
    double res = fabs(ctl->g[j + 1]);
    ctl->res_est = res;
    bool end = res <= ctl->tol * ctl->bnorm || ctl->its >= ctl->max_iter || breakdown || j + 1 == m;
    ctl->breakdown = breakdown;
    if (end) {
      ctl->k_end = j + 1;
      ctl->cycles += 1;
      ctl->action = ACT_UPDATE_X;
      if (ctl->trust && res <= ctl->tol * ctl->bnorm) {
        ctl->status = KFBI_OK;
        ctl->beta = res;
        ctl->next_phase = PH_DONE;
      } else {
        ctl->next_phase = PH_RESID;
      }
    } else {
      ctl->next_phase = PH_ARNOLDI;
      ctl->action = ACT_NEXT_V;
    }
    s_end = end ? 1 : 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) Hc[i] = hcol[i];
  if (!s_end) return;
  // y = R^{-1} g by column-oriented back substitution: after y[i] is known, every thread
  // removes its contribution from the rows above (k sequential steps, parallel updates)
  __shared__ double gy[MAX_RESTART];
  const int k = j + 1;
  for (int i = threadIdx.x; i < k; i += blockDim.x) gy[i] = ctl->g[i];
  __syncthreads();
  for (int i = k - 1; i >= 0; --i) {
    const double* Hi = ctl->H + (long)i * (m + 1);
    double yi = gy[i] / (i == j ? hcol[i] : Hi[i]);
    __syncthreads();
    for (int q = threadIdx.x; q < i; q += blockDim.x) gy[q] -= Hi[q] * yi;
    if (threadIdx.x == 0) {
      gy[i] = yi;
      ctl->y[i] = yi;
    }
    __syncthreads();
  }
}

// elementwise follow-up of the decision, then the phase switch (last block)
__global__ void k_gm_finish(GmresCtl* ctl, double* V, int ldv, const double* w, const double* r, double* x,
                            double* gin, float* gin_f, int n) {
  if (ctl->done) return;
  const int act = ctl->action;
  const int j = ctl->j;
  if (act == ACT_NEXT_V) {
    double inv = 1.0 / ctl->hnorm;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      double v = w[i] * inv;
      V[(long)(j + 1) * ldv + i] = v;
      gin[i] = v;
      gin_f[i] = (float)v;
    }
  } else if (act == ACT_UPDATE_X) {
    const int k = ctl->k_end;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      double v = x[i];
      for (int q = 0; q < k; ++q) v += V[(long)q * ldv + i] * ctl->y[q];
      x[i] = v;
      gin[i] = v;
      gin_f[i] = (float)v;
    }
  } else if (act == ACT_RESTART) {
    double inv = 1.0 / ctl->beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      double v = r[i] * inv;
      V[i] = v;
      gin[i] = v;
      gin_f[i] = (float)v;
    }
  }
  if (last_block(&ctl->ticket) && threadIdx.x == 0) {
    if (act == ACT_NEXT_V) ctl->j = j + 1;
    ctl->phase = ctl->next_phase;
    ctl->action = ACT_NONE;
    if (ctl->phase == PH_DONE) ctl->done = 1;
  }
}

// r = b - y (outer residual of iterative refinement), ||r||^2 and ||b||^2 into out[0..1]
__global__ void k_resid(const double* b, const double* y, double* r, int n, double* out) {
  __shared__ double sh[32];
  double s = 0.0, t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double ri = b[i] - y[i];
    r[i] = ri;
    s += ri * ri;
    t += b[i] * b[i];
  }
  s = block_sum(s, sh);
  __syncthreads();
  t = block_sum(t, sh);
  if (threadIdx.x == 0) {
    out[0] = s;
    out[1] = t;
  }
}

__global__ void k_axpy_zero(double* x, double* d, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    x[i] += d[i];
    d[i] = 0.0;
  }
}

// Loop control of the graph form: counts bodies, stops the loop once the solve is done or
// the body count reaches `cap` (then the solve ends with KFBI_ERR_TIMEOUT).
__global__ void k_gm_cond(GmresCtl* ctl, cudaGraphConditionalHandle h, int cap) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int b = ++ctl->bodies;
  if (!ctl->done && b >= cap) {
    ctl->status = KFBI_ERR_TIMEOUT;
    ctl->phase = PH_DONE;
    ctl->done = 1;
  }
  cudaGraphSetConditional(h, ctl->done ? 0u : 1u);
}

// --------------------------------------------------------------------------- cluster form
// One GMRES body after the apply in a single launch of one thread-block cluster. CTA c of
// the cluster owns the rows [c R, (c + 1) R) of the Krylov basis and of every vector: it
// stages its slice of V[0..j] and of w in shared memory, forms its partial Gram-Schmidt
// coefficients, and every CTA sums the partials of all CTAs through distributed shared
// memory in the same order, so the Hessenberg column, the Givens rotations and every
// decision are identical in all CTAs without a broadcast. CTA 0 writes the control block.
// Float64 throughout; both Gram-Schmidt passes (CGS2) as in the multi-kernel form. The
// float64 pipe is narrow, so dependent float64 chains are kept short: the rotations of the
// new Hessenberg column run as a warp scan, sums as shuffle trees, and ||w||^2 after the
// second pass comes from the second pass's own reduction,
//   ||w' - V h2||^2 = ||w'||^2 - ||h2||^2   (V orthonormal, h2 = V^T w'),
// with an explicit reduction when that difference cancels (below half of ||w'||^2).
constexpr int GMF_THREADS = 512;
constexpr int GMF_PART = MAX_RESTART + 2;
// row stride of the partial-sum and receive buffers: a multiple of 16 bytes for either type
constexpr int GMF_PART_P = (GMF_PART + 3) & ~3;

// row stride of the staged V slice: >= R and 4 mod 16 doubles, so that the lane patterns of
// the dot and combine steps touch each shared-memory bank at most twice per warp access
__host__ __device__ inline int gmf_row_stride(int R) { return R + ((20 - R % 16) % 16); }

__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cl_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// barrier over every thread of every CTA in the cluster; orders shared-memory writes before
// it with distributed shared-memory reads after it
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// arrive without release semantics: no use orders memory through the barrier itself (the
// mbarriers' initialisation is published by fence.mbarrier_init, received copies complete on
// the receiver's mbarrier, remote loads have returned before the arrive), so the arrive need
// not wait for this thread's outstanding loads
__device__ __forceinline__ void cl_arrive() { asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory"); }
__device__ __forceinline__ void cl_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// ---- push reductions: every CTA copies its partial sums into a receive row of every CTA of
// the cluster (bulk copies, shared::cta -> shared::cluster) that complete the transaction
// count of the receiver's mbarrier; each CTA then waits on its own barrier only.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned cl_map(unsigned addr, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for phase 0 of a barrier; false when the bound ran out
constexpr int GMF_WAIT_TRIES = 1 << 22;
__device__ __forceinline__ bool mbar_wait0(unsigned long long* b) {
  for (int it = 0; it < GMF_WAIT_TRIES; ++it)
    if (mbar_try(b, 0)) return true;
  return false;
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_to_cluster(unsigned dst, unsigned src, unsigned bytes, unsigned mbar) {
  asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "r"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
// L elements rounded up to a multiple of 16 bytes
template <typename T>
__host__ __device__ inline int gmf_pad(int L) {
  constexpr int E = 16 / (int)sizeof(T);
  return (L + E - 1) / E * E;
}
// element offset of the receive rows in the dynamic shared memory (after sV, sH, sw)
__host__ __device__ inline size_t gmf_recv_off(int m, int Rp, int hs, int esz) {
  const size_t e = (size_t)(m + 1) * Rp + (hs ? (size_t)(m + 1) * (m + 1) : 0) + Rp;
  const size_t E = 16 / (size_t)esz;
  return (e + E - 1) / E * E;
}

// out[0..L) = sum over the cluster's CTAs (rank order, the same in every CTA) of part[0..L).
// part was written before a __syncthreads by threads that fenced their writes for the async
// proxy; recv holds cs rows of GMF_PART_P; mbar expects cs * gmf_pad(L) elements. A wait that
// runs out sets *err and the sums are not meaningful.
template <typename T>
__device__ __forceinline__ void cl_push_reduce(const T* part, T* recv, unsigned long long* mbar, T* out, int L,
                                               unsigned cs, unsigned rank, int* err) {
  if (threadIdx.x < cs) {
    const unsigned dst = cl_map(smem_u32(recv + (size_t)rank * GMF_PART_P), threadIdx.x);
    const unsigned mb = cl_map(smem_u32(mbar), threadIdx.x);
    bulk_to_cluster(dst, smem_u32(part), (unsigned)(gmf_pad<T>(L) * sizeof(T)), mb);
  }
  if (!*(volatile int*)err && !mbar_wait0(mbar)) *(volatile int*)err = 1;
  for (int idx = threadIdx.x; idx < L; idx += GMF_THREADS) {
    T v = recv[idx];
    for (unsigned r = 1; r < cs; ++r) v += recv[(size_t)r * GMF_PART_P + idx];
    out[idx] = v;
  }
  __syncthreads();
}
__device__ __forceinline__ double cl_load(const double* p, unsigned rank) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p), r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(r) : "memory");
  return v;
}
__device__ __forceinline__ float cl_load(const float* p, unsigned rank) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p), r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(r) : "memory");
  return v;
}
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }

// out[0..L) = sum over the cluster's CTAs (rank order) of part[0..L) in each CTA. Thread t
// loads entry t / cs of CTA t % cs; a half-warp (cs = 16) or an 8-lane group (cs = 8) sums
// its loads by a fixed shuffle tree.
template <typename T>
__device__ __forceinline__ void cl_reduce(const T* part, T* out, int L, unsigned cs) {
  cl_sync();
  const int lcs = __ffs((int)cs) - 1;  // cs is a power of two
  const int per = GMF_THREADS >> lcs;
  for (int base = 0; base < L; base += per) {
    const int idx = base + (int)(threadIdx.x >> lcs);
    const unsigned c = threadIdx.x & (cs - 1);
    T v = idx < L ? cl_load(part + idx, c) : (T)0;
    for (unsigned o = cs >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (c == 0 && idx < L) out[idx] = v;
  }
  __syncthreads();
}

// sum of v over the CTA by shuffle trees; the result is returned in every thread
template <typename T>
__device__ __forceinline__ T cta_sum(T v, T* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T t = lane < GMF_THREADS / 32 ? sh[lane] : (T)0;
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  __syncthreads();
  return t;
}

// largest power of two <= min(32, x) (x >= 1)
__device__ __forceinline__ int lanes_pow2(int x) {
  int g = 1;
  while (2 * g <= x && g < 32) g <<= 1;
  return g;
}

// p[k] = sum_i sV[k][i] w[i] for k < K over this CTA's rows, and p[K] = sum_i w[i]^2 when
// with_norm. G adjacent lanes share one k: lane g sums i = g, g + G, ... with four
// accumulators, then a shuffle tree over the G lanes.
template <typename T>
__device__ __forceinline__ void cta_dots(const T* sV, int Rp, const T* w, int len, int K, bool with_norm, T* p) {
  const int Kt = K + (with_norm ? 1 : 0);
  const int G = lanes_pow2(GMF_THREADS / Kt), lg = __ffs(G) - 1;
  const int total = Kt * G;
  for (int base = 0; base < total; base += GMF_THREADS) {
    const int t = base + (int)threadIdx.x;
    const int k = t >> lg, g = t & (G - 1);
    T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    if (t < total) {
      const T* row = k < K ? sV + k * Rp : w;
      int i = g;
      for (; i + 3 * G < len; i += 4 * G) {
        a0 += row[i] * w[i];
        a1 += row[i + G] * w[i + G];
        a2 += row[i + 2 * G] * w[i + 2 * G];
        a3 += row[i + 3 * G] * w[i + 3 * G];
      }
      for (; i < len; i += G) a0 += row[i] * w[i];
    }
    T v = (a0 + a1) + (a2 + a3);
    for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (t < total && g == 0) {
      p[k] = v;
      fence_proxy_async();  // p may be read next by a bulk copy
    }
  }
  __syncthreads();
}

// w[i] += sign * sum_k sV[k][i] h[k] over this CTA's rows. G adjacent lanes share one i:
// lane g sums k = g, g + G, ... with four accumulators, then a shuffle tree.
template <typename T>
__device__ __forceinline__ void cta_combine(const T* sV, int Rp, const T* h, int K, int len, T* w, T sign) {
  const int G = lanes_pow2(GMF_THREADS / (len > 0 ? len : 1)), lg = __ffs(G) - 1;
  const int total = len * G;
  for (int base = 0; base < total; base += GMF_THREADS) {
    const int t = base + (int)threadIdx.x;
    const int i = t >> lg, g = t & (G - 1);
    T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    if (t < total) {
      int k = g;
      for (; k + 3 * G < K; k += 4 * G) {
        a0 += sV[k * Rp + i] * h[k];
        a1 += sV[(k + G) * Rp + i] * h[k + G];
        a2 += sV[(k + 2 * G) * Rp + i] * h[k + 2 * G];
        a3 += sV[(k + 3 * G) * Rp + i] * h[k + 3 * G];
      }
      for (; k < K; k += G) a0 += sV[k * Rp + i] * h[k];
    }
    T v = (a0 + a1) + (a2 + a3);
    for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (t < total && g == 0) w[i] = fma(sign, v, w[i]);
  }
  __syncthreads();
}

// Applies the j previous Givens rotations to the column hc[0..j] in one warp. With the
// carried entry x_0 = hc[0], rotation i maps (x_i, hc[i+1]) to
//   out_i = c_i x_i + s_i hc[i+1],   x_{i+1} = -s_i x_i + c_i hc[i+1],
// an affine recurrence x_{i+1} = A_i x_i + B_i (A_i = -s_i, B_i = c_i hc[i+1]). Lane l takes
// the rotations [l C, (l+1) C), composes its maps, an inclusive shuffle scan composes the
// lanes' maps, and each lane replays its rotations from its starting x. On return hc[0..j-1]
// hold out_i and hc[j] holds x_j. Warp 0 only; j <= 32 * GIV_CHUNK.
constexpr int GIV_CHUNK = (MAX_RESTART + 31) / 32;
template <typename T>
__device__ __forceinline__ void givens_scan(T* hc, const T* cs_, const T* sn_, int j) {
  const int lane = threadIdx.x & 31;
  const int C = (j + 31) / 32;
  const int i0 = lane * C;
  T c[GIV_CHUNK], s[GIV_CHUNK], h[GIV_CHUNK];
  T A = 1, B = 0;
#pragma unroll
  for (int u = 0; u < GIV_CHUNK; ++u) {
    const int i = i0 + u;
    const bool ok = u < C && i < j;
    c[u] = ok ? cs_[i] : (T)1;
    s[u] = ok ? sn_[i] : (T)0;
    h[u] = ok ? hc[i + 1] : (T)0;
  }
  const T x0 = hc[0];
  __syncwarp();
#pragma unroll
  for (int u = 0; u < GIV_CHUNK; ++u) {
    if (u < C && i0 + u < j) {
      const T cb = c[u] * h[u];
      B = fma(-s[u], B, cb);
      A = -s[u] * A;
    }
  }
  // inclusive scan of lane maps: (A, B) <- (A, B) o (A', B') of lane l - d
  for (int d = 1; d < 32; d <<= 1) {
    const T Ap = __shfl_up_sync(0xffffffffu, A, d);
    const T Bp = __shfl_up_sync(0xffffffffu, B, d);
    if (lane >= d) {
      B = fma(A, Bp, B);
      A = A * Ap;
    }
  }
  // exclusive prefix applied to x_0 gives this lane's starting x
  T Ae = __shfl_up_sync(0xffffffffu, A, 1);
  T Be = __shfl_up_sync(0xffffffffu, B, 1);
  T x = lane == 0 ? x0 : fma(Ae, x0, Be);
#pragma unroll
  for (int u = 0; u < GIV_CHUNK; ++u) {
    const int i = i0 + u;
    if (u < C && i < j) {
      const T sh = s[u] * h[u], ch = c[u] * h[u];
      hc[i] = fma(c[u], x, sh);
      x = fma(-s[u], x, ch);
      if (i == j - 1) hc[j] = x;
    }
  }
  __syncwarp();
}

__device__ __forceinline__ void gmf_close(GmresCtl* ctl, unsigned rank, cudaGraphConditionalHandle hcond,
                                          int use_cond, int cap, int done) {
  if (rank != 0 || threadIdx.x != 0) return;
  const int b = ++ctl->bodies;
  if (!done && b >= cap) {
    ctl->status = KFBI_ERR_TIMEOUT;
    ctl->phase = PH_DONE;
    ctl->done = 1;
    done = 1;
  }
  if (use_cond) cudaGraphSetConditional(hcond, done ? 0u : 1u);
}

// sw[i] = A v at node i0 + i for i < len: formed here from the apply's probe values and
// jumps (ia.st != nullptr; the apply then stops before its interpolation kernel) or read from
// the apply's output w. Eight lanes per node for the former. Ends with __syncthreads.
template <typename T>
__device__ __forceinline__ InterpPre<T> gmf_w_pre(const InterpArgs<T>& ia, int i0, int len) {
  const int i = (int)(threadIdx.x >> 3);
  return ia.st != nullptr ? interp_pre(ia, i0 + i, (int)(threadIdx.x & 7), i < len) : InterpPre<T>{};
}
// pre: this thread's interp_pre for the first GMF_THREADS / 8 nodes (gmf_w_pre)
template <typename T>
__device__ __forceinline__ void gmf_w_slice(const InterpArgs<T>& ia, const InterpPre<T>& pre, const double* w, int i0,
                                            int len, T* sw) {
  if (ia.st != nullptr) {
    // 8 lanes per node (6 stencil points), GMF_THREADS / 8 nodes at a time
    const int m = threadIdx.x & 7;
    for (int base = 0; base < len; base += GMF_THREADS / 8) {
      const int i = base + (int)(threadIdx.x >> 3);
      const InterpPre<T> q = base == 0 ? pre : interp_pre(ia, i0 + i, m, i < len);
      const T v = interp_finish(ia, q, i0 + i, m, i < len);
      if (m == 0 && i < len) sw[i] = v;
    }
  } else {
    for (int i = threadIdx.x; i < len; i += GMF_THREADS) sw[i] = (T)w[i0 + i];
  }
  __syncthreads();
}

// Dynamic shared memory: sV[(m+1) Rp] | sH[(m+1)(m+1)] (hsmem) | sw[Rp], elements of T.
// T is the arithmetic of the Gram-Schmidt passes, the rotations and the update of x, and the
// type of the stored basis V: double, or float for the inner solve of the mixed-precision
// refinement (its operator is the float32 apply; the control block stays double).
template <typename T>
__global__ void __launch_bounds__(GMF_THREADS, 1) k_gm_cluster(GmresCtl* ctl, T* V, int ldv, const double* w,
                                                            const double* b, double* x, double* gin, float* gin_f,
                                                            int n, int R, int hsmem, int push, InterpArgs<T> ia,
                                                            cudaGraphConditionalHandle hcond, int use_cond, int cap) {
  extern __shared__ __align__(16) unsigned char gmf_dyn[];
  T* dsm = (T*)gmf_dyn;
  __shared__ __align__(16) T part[2][GMF_PART_P];
  __shared__ __align__(8) unsigned long long s_mbar[3];
  __shared__ int s_err;
  __shared__ T h1[GMF_PART], h2[GMF_PART], hcol[GMF_PART];
  __shared__ T scs[MAX_RESTART], ssn[MAX_RESTART], gy[MAX_RESTART + 1];
  __shared__ T red[GMF_THREADS / 32];
  __shared__ int s_done, s_phase, s_j, s_m, s_its, s_maxit, s_trust, s_cycles, s_end;
  __shared__ double s_tol, s_bnorm;
  __shared__ T s_gj, s_gj1, s_hn2, s_inv, s_rd;
  const unsigned rank = cl_rank(), cs = cl_size();
  const int Rp = gmf_row_stride(R);
  const int i0 = (int)rank * R;
  const int len = max(0, min(n, i0 + R) - i0);
  if (threadIdx.x == 0) {
    s_done = ctl->done;
    s_phase = ctl->phase;
    s_j = ctl->j;
    s_m = ctl->m;
    s_its = ctl->its;
    s_maxit = ctl->max_iter;
    s_trust = ctl->trust;
    s_cycles = ctl->cycles;
    s_tol = ctl->tol;
    s_bnorm = ctl->bnorm;
    s_err = 0;
  }
  __syncthreads();
  if (s_done) {
    pdl_wait();
    gmf_close(ctl, rank, hcond, use_cond, cap, 1);
    return;
  }
  const int m = s_m;
  T* sV = dsm;
  T* sH = sV + (size_t)(m + 1) * Rp;
  T* sw = sH + (hsmem ? (size_t)(m + 1) * (m + 1) : 0);
  const T tolb = (T)(s_tol * s_bnorm);
  int done = 0;
  if (s_phase == PH_RESID) {
    // r = b - A x, ||r||; restart from r / ||r|| unless converged or out of iterations
    const InterpPre<T> pre = gmf_w_pre(ia, i0, len);
    pdl_wait();
    gmf_w_slice(ia, pre, w, i0, len, sw);
    T ss = 0;
    for (int i = threadIdx.x; i < len; i += GMF_THREADS) {
      const T r = (T)(b[i0 + i] - (double)sw[i]);
      sw[i] = r;
      ss += r * r;
    }
    ss = cta_sum(ss, red);
    if (threadIdx.x == 0) part[0][0] = ss;
    cl_reduce(part[0], h1, 1, cs);
    cl_arrive();  // the last read of another CTA's shared memory is done
    if (threadIdx.x == 0) {
      const T q = h1[0];
      const T r = q > (T)0 ? rsqrt_t(q) : (T)0;
      s_gj = q * r;  // ||r||
      s_gj1 = r;     // 1 / ||r||
    }
    __syncthreads();
    const T beta = s_gj;
    int status = KFBI_OK;
    if (beta <= tolb) {
      done = 1;
    } else if (s_its >= s_maxit) {
      done = 1;
      status = KFBI_ERR_NOT_CONVERGED;
    } else {
      const T inv = s_gj1;
      for (int i = threadIdx.x; i < len; i += GMF_THREADS) {
        const T v = sw[i] * inv;
        V[i0 + i] = v;
        gin[i0 + i] = v;
        gin_f[i0 + i] = (float)v;
      }
    }
    if (rank == 0 && threadIdx.x == 0) {
      ctl->beta = beta;
      if (done) {
        ctl->status = status;
        ctl->phase = PH_DONE;
        ctl->done = 1;
      } else {
        ctl->g[0] = beta;
        for (int k = 1; k <= m; ++k) ctl->g[k] = 0.0;
        ctl->j = 0;
        ctl->phase = PH_ARNOLDI;
      }
      ctl->action = ACT_NONE;
    }
    cl_wait();  // no CTA leaves while another still reads its shared memory
    gmf_close(ctl, rank, hcond, use_cond, cap, done);
    return;
  }
  // Arnoldi step j: w = A v_j against V[0..j]. The global reads are issued together and
  // consumed afterwards (one memory round trip, not one per array): the rotations and g_j,
  // the first NB * GMF_THREADS values of the V slice, then the w slice.
  const int j = s_j;
  const int K = j + 1;
  const InterpPre<T> pre = gmf_w_pre(ia, i0, len);  // fixed with the interface: before the wait
  // push reductions (push = 1): receive rows for pass 1 (reused by the explicit norm) and
  // pass 2; the barriers expect every CTA's rows; the cluster barrier begun here tells the
  // other CTAs (before their first copy) that these barriers are initialised
  T* recv0 = dsm + gmf_recv_off(m, Rp, hsmem, (int)sizeof(T));
  T* recv1 = recv0 + (size_t)cs * GMF_PART_P;
  if (push) {
    if (threadIdx.x == 0) {
      mbar_init(&s_mbar[0], 1);
      mbar_init(&s_mbar[1], 1);
      mbar_init(&s_mbar[2], 1);
      fence_mbar_init();
      mbar_arrive_expect(&s_mbar[0], cs * (unsigned)(gmf_pad<T>(K) * sizeof(T)));
      mbar_arrive_expect(&s_mbar[1], cs * (unsigned)(gmf_pad<T>(K + 1) * sizeof(T)));
      mbar_arrive_expect(&s_mbar[2], cs * (unsigned)(gmf_pad<T>(1) * sizeof(T)));
    }
    cl_arrive();
  }
  {
    static_assert(MAX_RESTART <= GMF_THREADS, "one rotation per thread");
    constexpr int NB = 4;  // loads in flight per thread and pass (longer unrolls measured slower)
    const int tid = (int)threadIdx.x;
    const int tot = K * len;
    double cs_r = 0.0, sn_r = 0.0, gj_r = 0.0, w_r = 0.0;
    if (tid < j) {
      cs_r = ctl->cs[tid];
      sn_r = ctl->sn[tid];
    }
    if (tid == 0) gj_r = ctl->g[j];
    // element t of the slice is (k, i) = (t / len, t mod len); consecutive t of one thread
    // differ by GMF_THREADS = qs len + rs, so (k, i) advance without a division
    const int qs = len > 0 ? GMF_THREADS / len : 0, rs = GMF_THREADS - qs * len;
    int kk = len > 0 ? tid / len : 0, ii = tid - kk * len;
    for (int t0 = 0; t0 < tot; t0 += NB * GMF_THREADS) {
      T buf[NB];
      int so[NB];
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const int t = t0 + u * GMF_THREADS + tid;
        so[u] = -1;
        if (t < tot) {
          buf[u] = V[(long)kk * ldv + i0 + ii];
          so[u] = kk * Rp + ii;
        }
        kk += qs;
        ii += rs;
        if (ii >= len) {
          ii -= len;
          kk += 1;
        }
      }
      if (t0 == 0) {
        // V and the rotations were complete before the apply started; w is its output
        pdl_wait();
        if (ia.st == nullptr && tid < len) w_r = w[i0 + tid];
      }
#pragma unroll
      for (int u = 0; u < NB; ++u)
        if (so[u] >= 0) sV[so[u]] = buf[u];
    }
    if (tot == 0) pdl_wait();
    if (tid < j) {
      scs[tid] = (T)cs_r;
      ssn[tid] = (T)sn_r;
    }
    if (tid == 0) s_gj = (T)gj_r;
    if (ia.st == nullptr) {
      if (tid < len) sw[tid] = (T)w_r;
      for (int i = tid + GMF_THREADS; i < len; i += GMF_THREADS) sw[i] = (T)w[i0 + i];
    }
  }
  if (ia.st != nullptr) gmf_w_slice(ia, pre, w, i0, len, sw);
  __syncthreads();
  // two passes of classical Gram-Schmidt; the second also reduces ||w'||^2 (entry K). The
  // passes are a loop that is not unrolled: the second runs the first one's instructions again
  // (already fetched) instead of an inlined copy of its own
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    T* hp = pass == 0 ? h1 : h2;
    cta_dots(sV, Rp, sw, len, K, pass == 1, part[pass]);
    if (push) {
      if (pass == 0) cl_wait();  // every CTA's barriers are initialised
      cl_push_reduce(part[pass], pass == 0 ? recv0 : recv1, &s_mbar[pass], hp, K + pass, cs, rank, &s_err);
    } else {
      cl_reduce(part[pass], hp, K + pass, cs);
    }
    cta_combine(sV, Rp, hp, K, len, sw, (T)-1);
  }
  // concurrently: warp 0 forms ||w''||^2 = ||w'||^2 - ||h2||^2, warp 1 applies the previous
  // rotations to the Hessenberg column h1 + h2
  if (threadIdx.x < 32) {
    T q0 = 0, q1 = 0;
    int k = threadIdx.x;
    for (; k + 32 < K; k += 64) {
      q0 += h2[k] * h2[k];
      q1 += h2[k + 32] * h2[k + 32];
    }
    if (k < K) q0 += h2[k] * h2[k];
    const T q = warp_sum(q0 + q1);
    if (threadIdx.x == 0) s_hn2 = h2[K] - q;
  } else if (threadIdx.x < 64) {
    for (int k = threadIdx.x - 32; k < K; k += 32) hcol[k] = h1[k] + h2[k];
    __syncwarp();
    if (j > 0) givens_scan(hcol, scs, ssn, j);
  }
  __syncthreads();
  if (!(s_hn2 > (T)0.5 * h2[K])) {
    // cancellation (w nearly in the span of V): reduce ||w''||^2 explicitly
    T ss = 0;
    for (int i = threadIdx.x; i < len; i += GMF_THREADS) ss += sw[i] * sw[i];
    ss = cta_sum(ss, red);
    if (threadIdx.x == 0) {
      part[0][0] = ss;
      fence_proxy_async();
    }
    if (push) {
      // part[0] and recv0 are free: every CTA has received every pass-2 row, so every pass-1
      // copy has completed
      __syncthreads();
      cl_push_reduce(part[0], recv0, &s_mbar[2], &s_hn2, 1, cs, rank, &s_err);
    } else {
      cl_reduce(part[0], &s_hn2, 1, cs);
    }
  }
  cl_arrive();  // the last access to another CTA's shared memory is done
  // the new rotation from (hcol[j], ||w''||), with reciprocal square roots only:
  //   hn = ||w''||, den = sqrt(hcol[j]^2 + hn^2), c = hcol[j] / den, s = hn / den
  if (threadIdx.x == 0) {
    const T hn2 = s_hn2 > (T)0 ? s_hn2 : (T)0;
    const T rh = hn2 > (T)0 ? rsqrt_t(hn2) : (T)0;
    const T hn = hn2 * rh;
    const T a = hcol[j];
    const T d2 = fma(a, a, hn2);
    const T rd = d2 > (T)0 ? rsqrt_t(d2) : (T)0;
    const T den = d2 * rd;
    const int brk = hn2 == (T)0;
    const T cj = d2 > (T)0 ? a * rd : (T)1, sj = hn * rd;
    hcol[j] = den;
    hcol[j + 1] = 0;
    const T gj = s_gj;
    gy[j] = cj * gj;
    const T gj1 = -sj * gj;
    s_gj1 = gj1;
    s_inv = rh;
    s_rd = rd;
    const int its = s_its + 1;
    const T res = fabs(gj1);
    s_end = (res <= tolb || its >= s_maxit || brk || j + 1 == m) ? 1 : 0;
    if (rank == 0) {
      ctl->cs[j] = cj;
      ctl->sn[j] = sj;
      ctl->rinv[j] = rd;
      ctl->g[j] = gy[j];
      ctl->g[j + 1] = gj1;
      ctl->its = its;
      ctl->res_est = res;
      ctl->hnorm = hn;
      ctl->breakdown = brk;
    }
    if (s_err) {
      // a reduction wait ran out: stop the solve with the timeout status
      ctl->status = KFBI_ERR_TIMEOUT;
      ctl->phase = PH_DONE;
      ctl->done = 1;
    }
  }
  __syncthreads();
  if (rank == 0) {
    // Hessenberg column j (rotated), written by all threads
    double* Hc = ctl->H + (long)j * (m + 1);
    for (int k = threadIdx.x; k <= j + 1; k += GMF_THREADS) Hc[k] = hcol[k];
  }
  if (s_err) {
    done = 1;
  } else if (!s_end) {
    const T inv = s_inv;
    for (int i = threadIdx.x; i < len; i += GMF_THREADS) {
      const T v = sw[i] * inv;
      V[(long)(j + 1) * ldv + i0 + i] = v;
      gin[i0 + i] = v;
      gin_f[i0 + i] = (float)v;
    }
    if (rank == 0 && threadIdx.x == 0) {
      ctl->j = j + 1;
      ctl->phase = PH_ARNOLDI;
      ctl->action = ACT_NONE;
    }
  } else {
    // end of the cycle: y = R^{-1} g by column-oriented back substitution (every CTA, with
    // the stored reciprocals of the diagonal), then x += V y over this CTA's rows
    const T res = fabs(s_gj1);
    for (int i = threadIdx.x; i < j; i += GMF_THREADS) {
      gy[i] = (T)ctl->g[i];
      scs[i] = (T)ctl->rinv[i];
    }
    if (threadIdx.x == 0) scs[j] = s_rd;
    if (hsmem)
      for (int t = threadIdx.x; t < j * (m + 1); t += GMF_THREADS) sH[t] = (T)ctl->H[t];
    __syncthreads();
    for (int i = K - 1; i >= 0; --i) {
      const T yi = gy[i] * scs[i];
      __syncthreads();
      if (i == j || hsmem) {
        const T* Hi = i == j ? hcol : sH + (long)i * (m + 1);
        for (int q = threadIdx.x; q < i; q += GMF_THREADS) gy[q] = fma(-Hi[q], yi, gy[q]);
      } else {
        const double* Hi = ctl->H + (long)i * (m + 1);
        for (int q = threadIdx.x; q < i; q += GMF_THREADS) gy[q] = fma(-(T)Hi[q], yi, gy[q]);
      }
      if (threadIdx.x == 0) gy[i] = yi;
      __syncthreads();
    }
    // x += V y over this CTA's rows (w is no longer needed), then the next apply's input.
    // In float32 the product V y is formed alone and added to the float64 x.
    for (int i = threadIdx.x; i < len; i += GMF_THREADS) sw[i] = sizeof(T) == 8 ? (T)x[i0 + i] : (T)0;
    __syncthreads();
    cta_combine(sV, Rp, gy, K, len, sw, (T)1);
    for (int i = threadIdx.x; i < len; i += GMF_THREADS) {
      const double v = sizeof(T) == 8 ? (double)sw[i] : x[i0 + i] + (double)sw[i];
      x[i0 + i] = v;
      gin[i0 + i] = v;
      gin_f[i0 + i] = (float)v;
    }
    const bool conv = s_trust && res <= tolb;
    if (rank == 0)
      for (int i = threadIdx.x; i < K; i += GMF_THREADS) ctl->y[i] = gy[i];
    if (rank == 0 && threadIdx.x == 0) {
      ctl->k_end = K;
      ctl->cycles = s_cycles + 1;
      ctl->action = ACT_NONE;
      if (conv) {
        ctl->status = KFBI_OK;
        ctl->beta = res;
        ctl->phase = PH_DONE;
        ctl->done = 1;
      } else {
        ctl->phase = PH_RESID;
      }
    }
    done = conv ? 1 : 0;
  }
  cl_wait();  // no CTA leaves while another may still read or copy from its shared memory
  gmf_close(ctl, rank, hcond, use_cond, cap, done);
}
// --------------------------------------------------------------------------- device-driven refinement
__global__ void k_ir_init(IrCtl* ir, double tol, int max_iter, int max_sweeps, int cap_outer) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ir->done = 0;
  ir->status = KFBI_OK;
  ir->sweeps = 0;
  ir->total_its = 0;
  ir->total_cycles = 0;
  ir->inner_bodies = 0;
  ir->run_inner = 0;
  ir->outer_bodies = 0;
  ir->max_iter = max_iter;
  ir->max_sweeps = max_sweeps;
  ir->cap_outer = cap_outer;
  ir->tol = tol;
  ir->rel = 1.0;
}

// r = b - y (y = A64 x), ||r|| / ||b||, the decision of the sweep, and for another sweep the
// start of the inner float32 GMRES on A d = r from d = 0 (tolerance 0.5 tol / rel clamped to
// [1e-7, 0.5]; the inner GMRES trusts its Givens estimate). One block.
__global__ void k_ir_decide(IrCtl* ir, GmresCtl* g, const double* b, const double* y, double* r, double* V,
                            float* Vf, double* d, double* gin, float* gin_f, int n, int m,
                            cudaGraphConditionalHandle h_inner) {
  __shared__ double sh[32];
  __shared__ double s_rr;
  __shared__ int s_run;
  __shared__ double s_inv;
  double rr = 0.0, bb = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double ri = b[i] - y[i];
    r[i] = ri;
    rr += ri * ri;
    bb += b[i] * b[i];
  }
  rr = block_sum(rr, sh);
  if (threadIdx.x == 0) s_rr = rr;
  __syncthreads();
  bb = block_sum(bb, sh);
  if (threadIdx.x == 0) {
    rr = s_rr;
    const double rel = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    ir->rel = rel;
    ir->sweeps += 1;
    int run = 0;
    if (rel <= ir->tol) {
      ir->done = 1;
      ir->status = KFBI_OK;
    } else if (ir->total_its >= ir->max_iter || ir->sweeps > ir->max_sweeps) {
      ir->done = 1;
      ir->status = KFBI_ERR_NOT_CONVERGED;
    } else {
      run = 1;
      double inner = 0.5 * ir->tol / rel;
      inner = inner < 1e-7 ? 1e-7 : (inner > 0.5 ? 0.5 : inner);
      const double bn = sqrt(rr);
      g->phase = PH_ARNOLDI;
      g->next_phase = PH_ARNOLDI;
      g->done = 0;
      g->action = ACT_NONE;
      g->j = 0;
      g->k_end = 0;
      g->its = 0;
      g->cycles = 0;
      g->max_iter = ir->max_iter - ir->total_its;
      g->m = m;
      g->status = KFBI_OK;
      g->ticket = 0;
      g->breakdown = 0;
      g->trust = 1;
      g->bodies = 0;
      g->tol = inner;
      g->bnorm = bn;
      g->beta = bn;
      g->hnorm = 0.0;
      g->res_est = 0.0;
      g->g[0] = bn;
      for (int k = 1; k <= m; ++k) g->g[k] = 0.0;
      s_inv = 1.0 / bn;
    }
    ir->run_inner = run;
    s_run = run;
    cudaGraphSetConditional(h_inner, run ? 1u : 0u);
  }
  __syncthreads();
  if (!s_run) return;
  const double inv = s_inv;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = r[i] * inv;
    V[i] = v;
    if (Vf) Vf[i] = (float)v;
    gin[i] = v;
    gin_f[i] = (float)v;
    d[i] = 0.0;
  }
}

// after the inner GMRES: x += d, d = 0, iteration totals, the loop condition of the sweeps
__global__ void k_ir_finish(IrCtl* ir, const GmresCtl* g, double* x, double* d, int n,
                            cudaGraphConditionalHandle h_outer) {
  __shared__ int s_run;
  if (threadIdx.x == 0) s_run = ir->run_inner;
  __syncthreads();
  if (s_run)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      x[i] += d[i];
      d[i] = 0.0;
    }
  if (threadIdx.x != 0) return;
  if (s_run) {
    ir->total_its += g->its;
    ir->total_cycles += g->cycles;
    ir->inner_bodies += g->bodies;
    if (g->status == KFBI_ERR_TIMEOUT) {
      ir->done = 1;
      ir->status = KFBI_ERR_TIMEOUT;
    }
    ir->run_inner = 0;
  }
  ir->outer_bodies += 1;
  if (!ir->done && ir->outer_bodies >= ir->cap_outer) {
    ir->done = 1;
    ir->status = KFBI_ERR_TIMEOUT;
  }
  cudaGraphSetConditional(h_outer, ir->done ? 0u : 1u);
}

// --------------------------------------------------------------------------- host side
// Largest dynamic shared memory the cluster kernel of element type T may use (queried and
// set once per context; the attribute is the function's largest possible value, the same
// for every context).
template <typename T>
static size_t gmf_smem_limit(kfbi_ctx* c) {
  size_t& mx = c->gmf_smem_max[sizeof(T) == 4 ? 1 : 0];
  if (mx == 0) {
    cudaFuncAttributes fa{};
    int optin = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, k_gm_cluster<T>) != cudaSuccess) {
      cudaGetLastError();
      mx = 1;
      return 0;
    }
    size_t lim = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    if (cudaFuncSetAttribute(k_gm_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim) != cudaSuccess ||
        cudaFuncSetAttribute(k_gm_cluster<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      lim = 0;
    }
    mx = lim > 0 ? lim : 1;
  }
  return mx > 1 ? mx : 0;
}

static cudaLaunchConfig_t gmf_launch_config(kfbi_ctx* c, const kfbi_ctx::GmfConfig& g, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(g.cs, 1, 1);
  cfg.blockDim = dim3(GMF_THREADS, 1, 1);
  cfg.dynamicSmemBytes = g.smem;
  cfg.stream = c->stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = g.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = c->use_pdl ? 2 : 1;
  return cfg;
}

// Cluster form for n nodes and restart m: 16 CTAs (else 8) whose slices of V (and, when it
// fits, the Hessenberg matrix for the back substitution) fit in shared memory and that the
// device can co-schedule. cs = 0: the multi-kernel form.
template <typename T>
static kfbi_ctx::GmfConfig gmf_select_t(kfbi_ctx* c, int n, int m) {
  kfbi_ctx::GmfConfig& cache = sizeof(T) == 4 ? c->gmf32 : c->gmf;
  if (cache.n == n && cache.m == m) return cache;
  const size_t lim = gmf_smem_limit<T>(c);
  kfbi_ctx::GmfConfig pick{};
  pick.n = n;
  pick.m = m;
  for (int cs : {16, 8}) {
    if (pick.cs) break;
    if (c->force_cs != 0 && cs != c->force_cs) continue;
    const int R = cdiv(n, cs), Rp = gmf_row_stride(R);
    // push reductions first (their receive rows cost 2 cs GMF_PART_P elements), then the
    // Hessenberg matrix staged for the back substitution
    for (int opt = c->gmf_push ? 0 : 2; opt < 4 && !pick.cs; ++opt) {
      const int push = opt < 2 ? 1 : 0, hs = (opt & 1) ? 0 : 1;
      const size_t elems = push ? gmf_recv_off(m, Rp, hs, (int)sizeof(T)) + (size_t)2 * cs * GMF_PART_P
                                : (size_t)(m + 1) * Rp + (hs ? (size_t)(m + 1) * (m + 1) : 0) + Rp;
      const size_t smem = sizeof(T) * elems;
      if (smem > lim) continue;
      kfbi_ctx::GmfConfig g{n, m, cs, R, hs, smem, sizeof(T) == 4 ? 1 : 0, push};
      cudaLaunchAttribute attr[2];
      cudaLaunchConfig_t cfg = gmf_launch_config(c, g, attr);
      int nc = 0;
      if (cudaOccupancyMaxActiveClusters(&nc, k_gm_cluster<T>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        nc = 0;
      }
      if (nc >= 1) {
        pick = g;
        break;
      }
    }
  }
  cache = pick;
  return pick;
}

// inner = true: the inner solve of the mixed-precision refinement, whose Gram-Schmidt runs in
// float32 when the context allows it (KFBI_OPT_FP32_ARNOLDI) and has the float32 basis
kfbi_ctx::GmfConfig gmf_select(kfbi_ctx* c, int n, int m, bool inner) {
  kfbi_ctx::GmfConfig none{};
  if (!c->gm_cluster) return none;
  if (inner && c->arn32 && c->gVf != nullptr) {
    kfbi_ctx::GmfConfig g = gmf_select_t<float>(c, n, m);
    if (g.cs > 0) return g;
  }
  return gmf_select_t<double>(c, n, m);
}

static kfbi_status body(kfbi_ctx* c, int kind, bool fp32, const double* eps_v, const double* b, double* x,
                        const kfbi_ctx::GmfConfig& gf, cudaGraphConditionalHandle hcond, int use_cond, int cap) {
  cudaStream_t s = c->stream;
  const int n = c->n;
  const int* done = &c->gctl->done;
  int layer = kind == KFBI_BIE_STEFAN_SL ? KFBI_SINGLE : KFBI_DOUBLE;
  // the float32 Gram-Schmidt kernel forms A v itself from the apply's probe values and jumps
  // (the apply then stops before its interpolation kernel)
  const bool fuse = gf.cs > 0 && gf.f32 && fp32 && c->fuse_interp;
  KFBI_CHECK(apply_enqueue(c, layer, fp32, c->gin, c->gw, nullptr, nullptr, kind, eps_v, done, c->gin_f, fuse));
  const int ldv = c->max_nodes;
  if (gf.cs > 0) {
    cudaLaunchAttribute attr[2];
    cudaLaunchConfig_t cfg = gmf_launch_config(c, gf, attr);
    launched(c, 1);
    if (gf.f32) {
      const InterpArgs<float> ia = fuse ? interp_args_f32(c, kind, eps_v, c->gin_f) : InterpArgs<float>{};
      KFBI_TRY(cudaLaunchKernelEx(&cfg, k_gm_cluster<float>, c->gctl, c->gVf, ldv, (const double*)c->gw, b, x,
                                  c->gin, c->gin_f, n, gf.R, gf.hsmem, gf.push, ia, hcond, use_cond, cap));
    } else {
      KFBI_TRY(cudaLaunchKernelEx(&cfg, k_gm_cluster<double>, c->gctl, c->gV, ldv, (const double*)c->gw, b, x,
                                  c->gin, c->gin_f, n, gf.R, gf.hsmem, gf.push, InterpArgs<double>{}, hcond, use_cond,
                                  cap));
    }
    return KFBI_OK;
  }
  const int dblocks = c->gm_m + 1;
  const int ublocks = cdiv(n, 32);
  launched(c, 5);
  k_gm_dots<<<dblocks, GM_THREADS, 0, s>>>(c->gctl, c->gV, ldv, c->gw, b, c->gr, n, c->gpart, 0);
  k_gm_update<<<ublocks, 32 * UPD_WARPS, 0, s>>>(c->gctl, c->gV, ldv, c->gw, n, c->gpart, 0);
  k_gm_dots<<<dblocks, GM_THREADS, 0, s>>>(c->gctl, c->gV, ldv, c->gw, b, c->gr, n, c->gpart, 1);
  k_gm_update<<<ublocks, 32 * UPD_WARPS, 0, s>>>(c->gctl, c->gV, ldv, c->gw, n, c->gpart, 1);
  k_gm_finish<<<GM_BLOCKS, GM_THREADS, 0, s>>>(c->gctl, c->gV, ldv, c->gw, c->gr, x, c->gin, c->gin_f, n);
  if (use_cond) {
    launched(c, 1);
    k_gm_cond<<<1, 32, 0, s>>>(c->gctl, hcond, cap);
  }
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

int body_cap(int max_iter, int m) { return 2 * max_iter + 2 * (max_iter / m) + 8; }

// loop caps of a context: the derived ones unless KFBI_OPT_BODY_CAP / KFBI_OPT_SWEEP_CAP set them
static int ctx_body_cap(const kfbi_ctx* c, int max_iter, int m) {
  return c->body_cap_set > 0 ? c->body_cap_set : body_cap(max_iter, m);
}
static int ctx_sweep_cap(const kfbi_ctx* c) { return c->sweep_cap_set > 0 ? c->sweep_cap_set : IR_MAX_SWEEPS + 2; }

kfbi_status cap_begin(kfbi_ctx* c, cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd);
kfbi_status cap_end(kfbi_ctx* c, std::vector<cudaGraphNode_t>* sinks);
kfbi_status add_while(cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd, cudaGraphConditionalHandle h,
                             cudaGraphNode_t* node, cudaGraph_t* body);

// Adds to graph g (after deps) the GMRES loop of one solve: a conditional WHILE node whose
// body (captured from the context's stream) is one GMRES iteration that also sets the loop
// condition. k_gm_init and k_gm_start must run before it.
kfbi_status add_gmres_nodes(kfbi_ctx* c, cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd, int kind, bool fp32,
                            const double* eps_v, const double* b, double* x, int cap, const kfbi_ctx::GmfConfig& gf,
                            cudaGraphNode_t* node, int* body_launches) {
  cudaGraphConditionalHandle h;
  KFBI_TRY(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cudaGraph_t bodyg;
  KFBI_CHECK(add_while(g, deps, nd, h, node, &bodyg));
  KFBI_CHECK(cap_begin(c, bodyg, nullptr, 0));
  const long long l0 = c->launches;
  kfbi_status st = body(c, kind, fp32, eps_v, b, x, gf, h, 1, cap);
  *body_launches = (int)(c->launches - l0);
  c->launches = l0;  // capture launches nothing; replays are counted per body
  kfbi_status st2 = cap_end(c, nullptr);
  KFBI_CHECK(st);
  return st2;
}

static kfbi_status build_graph(kfbi_ctx* c, kfbi_ctx::SolveGraph& G, int kind, bool fp32, const double* eps_v,
                               const double* b, double* x, int cap, const kfbi_ctx::GmfConfig& gf) {
  if (G.exec) cudaGraphExecDestroy(G.exec);
  if (G.graph) cudaGraphDestroy(G.graph);
  G.exec = nullptr;
  G.graph = nullptr;
  G.version = -1;
  KFBI_TRY(cudaGraphCreate(&G.graph, 0));
  cudaGraphNode_t node;
  kfbi_status st = add_gmres_nodes(c, G.graph, nullptr, 0, kind, fp32, eps_v, b, x, cap, gf, &node, &G.body_launches);
  if (st == KFBI_OK && cudaGraphInstantiate(&G.exec, G.graph, 0) != cudaSuccess) st = KFBI_ERR_CUDA;
  if (st != KFBI_OK) {
    G.graph = nullptr;  // released without cudaGraphDestroy (see solve_ir_graph)
    G.exec = nullptr;
    cudaGetLastError();
    return st;
  }
  G.version = c->layout_version;
  return KFBI_OK;
}

int restart_length(int restart, int n) {
  int m = restart < n ? restart : n;
  if (m > MAX_RESTART) m = MAX_RESTART;
  return m < 1 ? 1 : m;
}

kfbi_status gmres_start_enqueue(kfbi_ctx* c, double tol, int max_iter, int m) {
  k_gm_init<<<1, 32, 0, c->stream>>>(c->gctl, tol, max_iter, m, 0);
  k_gm_start<<<1, 1024, 0, c->stream>>>(c->gb, c->gx, c->gin, c->gin_f, c->gV, nullptr, c->n, c->gctl, 0);
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

kfbi_status ir_start_enqueue(kfbi_ctx* c, double tol, int max_iter) {
  k_ir_init<<<1, 32, 0, c->stream>>>(c->irctl, tol, max_iter, IR_MAX_SWEEPS, ctx_sweep_cap(c));
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

// GMRES on A x = b with the apply precision `fp32`; b and x are context buffers (gb, gx) so
// that a cached graph stays valid; x holds the initial guess (ignored when zero_guess).
static kfbi_status gmres_run(kfbi_ctx* c, int kind, bool fp32, const double* eps_v, const double* b, double* x,
                             double tol, int max_iter, int restart, bool zero_guess, bool trust, int* its, int* cycles,
                             double* rel, int* status) {
  cudaStream_t s = c->stream;
  const int n = c->n;
  int m = restart < n ? restart : n;
  if (m > MAX_RESTART) m = MAX_RESTART;
  if (m < 1) m = 1;
  c->gm_m = m;
  const int cap = ctx_body_cap(c, max_iter, m);
  const kfbi_ctx::GmfConfig gf = gmf_select(c, n, m, fp32);
  c->gmf_last_cs = gf.cs;
  const size_t hdr = offsetof(GmresCtl, g);
  launched(c, 2);
  k_gm_init<<<1, 32, 0, s>>>(c->gctl, tol, max_iter, m, trust ? 1 : 0);
  k_gm_start<<<1, 1024, 0, s>>>(b, x, c->gin, c->gin_f, c->gV, gf.f32 ? c->gVf : nullptr, n, c->gctl,
                                zero_guess ? 1 : 0);
  bool graphed = false;
  if (c->use_graphs && !c->timing) {
    kfbi_ctx::SolveGraph& G = c->sgraph[kind][fp32 ? 1 : 0];
    kfbi_status st = KFBI_OK;
    if (G.exec == nullptr || G.version != c->layout_version || G.m != m || G.cs != gf.cs || G.pdl != c->use_pdl ||
        G.cfg != c->cfg_version || G.f32 != gf.f32 || G.cap != cap) {
      st = build_graph(c, G, kind, fp32, eps_v, b, x, cap, gf);
      G.cap = cap;
      G.m = m;
      G.cs = gf.cs;
      G.pdl = c->use_pdl;
      G.cfg = c->cfg_version;
      G.f32 = gf.f32;
    }
    if (st == KFBI_OK) st = box_table_join(c, s);
    if (st == KFBI_OK && cudaGraphLaunch(G.exec, s) == cudaSuccess) {
      graphed = true;
    } else {
      c->use_graphs = false;  // keep the stream-launched loop from now on
      cudaGetLastError();
    }
  }
  if (graphed) {
    KFBI_TRY(cudaMemcpyAsync(c->host_gctl, c->gctl, hdr, cudaMemcpyDeviceToHost, s));
    KFBI_TRY(cudaStreamSynchronize(s));
    // bodies replayed by the graph: one apply, the Gram-Schmidt kernel(s) and the loop test
    c->launches += (long long)c->host_gctl->bodies * c->sgraph[kind][fp32 ? 1 : 0].body_launches;
  } else {
    int launched_bodies = 0, chunk = 2;
    while (true) {
      for (int q = 0; q < chunk; ++q) KFBI_CHECK(body(c, kind, fp32, eps_v, b, x, gf, 0, 0, cap));
      launched_bodies += chunk;
      KFBI_TRY(cudaMemcpyAsync(c->host_gctl, c->gctl, hdr, cudaMemcpyDeviceToHost, s));
      KFBI_TRY(cudaStreamSynchronize(s));
      if (c->host_gctl->done) break;
      if (launched_bodies > cap) {  // backstop: the bodies themselves stop at the cap
        c->host_gctl->status = KFBI_ERR_TIMEOUT;
        break;
      }
      chunk = chunk < 8 ? chunk * 2 : 8;
    }
  }
  const GmresCtl* h = c->host_gctl;
  *its = h->its;
  *cycles = h->cycles;
  *rel = h->bnorm > 0 ? h->beta / h->bnorm : 0.0;
  *status = h->status;
  return KFBI_OK;
}

// ---- device-driven refinement as one graph: a WHILE node over the sweeps whose body is
//   [float64 apply of x] -> k_ir_decide -> WHILE node over the inner GMRES bodies -> k_ir_finish
// (nested conditional nodes), so a mixed-precision solve is one graph launch.
kfbi_status cap_begin(kfbi_ctx* c, cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd) {
  KFBI_TRY(cudaStreamBeginCaptureToGraph(c->stream, g, deps, nullptr, nd, cudaStreamCaptureModeRelaxed));
  c->capturing = true;
  return KFBI_OK;
}

// ends the capture; sinks (optional) receives the capture's last nodes
kfbi_status cap_end(kfbi_ctx* c, std::vector<cudaGraphNode_t>* sinks) {
  cudaError_t e = cudaSuccess;
  if (sinks != nullptr) {
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    e = cudaStreamGetCaptureInfo(c->stream, &cst, nullptr, nullptr, &deps, nullptr, &nd);
    if (e == cudaSuccess) sinks->assign(deps, deps + nd);
  }
  c->capturing = false;
  cudaGraph_t out = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(c->stream, &out);
  KFBI_TRY(e);
  KFBI_TRY(e2);
  return KFBI_OK;
}

kfbi_status add_while(cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd, cudaGraphConditionalHandle h,
                      cudaGraphNode_t* node, cudaGraph_t* body) {
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  KFBI_TRY(cudaGraphAddNode(node, g, deps, nullptr, nd, &cp));
  *body = cp.conditional.phGraph_out[0];
  return KFBI_OK;
}

// Adds the refinement loop of context c to graph g (a root node). The loop works on the
// context's copies ir_b (rhs) and ir_x (iterate), ir_dn (normal derivative of the last float64
// apply, when want_dn); k_ir_init must run before each launch.
kfbi_status add_ir_nodes(kfbi_ctx* c, cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd, int kind, bool want_dn,
                         int m, const kfbi_ctx::GmfConfig& gf, int cap_inner, cudaGraphNode_t* node,
                         int* inner_body_launches) {
  const int n = c->n;
  const double* ev = kind == KFBI_BIE_STEFAN_SL ? c->gev : nullptr;
  const int layer = kind == KFBI_BIE_STEFAN_SL ? KFBI_SINGLE : KFBI_DOUBLE;
  cudaGraphConditionalHandle h_outer, h_inner;
  KFBI_TRY(cudaGraphConditionalHandleCreate(&h_outer, g, 1, cudaGraphCondAssignDefault));
  KFBI_TRY(cudaGraphConditionalHandleCreate(&h_inner, g, 0, cudaGraphCondAssignDefault));
  cudaGraphNode_t n_outer, n_inner;
  cudaGraph_t b_outer, b_inner;
  KFBI_CHECK(add_while(g, deps, nd, h_outer, &n_outer, &b_outer));
  *node = n_outer;
  const long long l0 = c->launches;
  // sweep part 1: float64 apply of the iterate, residual and decision
  KFBI_CHECK(cap_begin(c, b_outer, nullptr, 0));
  kfbi_status st = apply_enqueue(c, layer, false, c->ir_x, c->tmp_vals, want_dn ? c->ir_dn : nullptr, nullptr, kind,
                                 ev, c->zero_flag, nullptr);
  if (st == KFBI_OK) {
    k_ir_decide<<<1, 1024, 0, c->stream>>>(c->irctl, c->gctl, c->ir_b, c->tmp_vals, c->gb, c->gV,
                                           gf.f32 ? c->gVf : nullptr, c->gx, c->gin, c->gin_f, n, m, h_inner);
    if (cudaGetLastError() != cudaSuccess) st = KFBI_ERR_CUDA;
  }
  std::vector<cudaGraphNode_t> sinks;
  kfbi_status st2 = cap_end(c, &sinks);
  KFBI_CHECK(st);
  KFBI_CHECK(st2);
  // inner GMRES loop
  KFBI_CHECK(add_while(b_outer, sinks.data(), sinks.size(), h_inner, &n_inner, &b_inner));
  KFBI_CHECK(cap_begin(c, b_inner, nullptr, 0));
  const long long l1 = c->launches;
  st = body(c, kind, true, ev, c->gb, c->gx, gf, h_inner, 1, cap_inner);
  *inner_body_launches = (int)(c->launches - l1);
  st2 = cap_end(c, nullptr);
  KFBI_CHECK(st);
  KFBI_CHECK(st2);
  // sweep part 2: x += d and the loop condition
  KFBI_CHECK(cap_begin(c, b_outer, &n_inner, 1));
  k_ir_finish<<<1, 256, 0, c->stream>>>(c->irctl, c->gctl, c->ir_x, c->gx, n, h_outer);
  st = cudaGetLastError() == cudaSuccess ? KFBI_OK : KFBI_ERR_CUDA;
  st2 = cap_end(c, nullptr);
  c->launches = l0;  // capture launches nothing
  KFBI_CHECK(st);
  return st2;
}

// One mixed-precision solve as a graph launch. *used = false: the graph form is unavailable
// (the caller runs the host-driven loop instead).
static kfbi_status solve_ir_graph(kfbi_ctx* c, int kind, const double* rhs, double tol, int max_iter, int restart,
                                  double* x, double* dnormal, kfbi_solve_info* out, bool* used) {
  *used = false;
  cudaStream_t s = c->stream;
  const int n = c->n;
  int m = restart < n ? restart : n;
  if (m > MAX_RESTART) m = MAX_RESTART;
  if (m < 1) m = 1;
  c->gm_m = m;
  const kfbi_ctx::GmfConfig gf = gmf_select(c, n, m, true);
  c->gmf_last_cs = gf.cs;
  const int cap = ctx_body_cap(c, max_iter, m);
  const int max_sweeps = IR_MAX_SWEEPS;
  kfbi_ctx::IrGraph& G = c->irgraph[kind][dnormal != nullptr ? 1 : 0];
  if (G.exec == nullptr || G.version != c->layout_version || G.m != m || G.cs != gf.cs || G.pdl != c->use_pdl ||
      G.cap != cap || G.cfg != c->cfg_version || G.f32 != gf.f32 || G.asw != c->apply_sweeps) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
    G.exec = nullptr;
    G.graph = nullptr;
    G.version = -1;
    kfbi_status st = cudaGraphCreate(&G.graph, 0) == cudaSuccess ? KFBI_OK : KFBI_ERR_CUDA;
    cudaGraphNode_t node;
    if (st == KFBI_OK)
      st = add_ir_nodes(c, G.graph, nullptr, 0, kind, dnormal != nullptr, m, gf, cap, &node, &G.inner_body_launches);
    if (st == KFBI_OK && cudaGraphInstantiate(&G.exec, G.graph, 0) != cudaSuccess) st = KFBI_ERR_CUDA;
    if (st != KFBI_OK) {
      // released without cudaGraphDestroy (a graph whose capture failed crashed the driver on
      // destruction); the host-driven loop takes over
      if (G.exec) cudaGraphExecDestroy(G.exec);
      G.exec = nullptr;
      G.graph = nullptr;
      cudaGetLastError();
      return KFBI_OK;  // not used
    }
    G.version = c->layout_version;
    G.m = m;
    G.cs = gf.cs;
    G.pdl = c->use_pdl;
    G.cap = cap;
    G.cfg = c->cfg_version;
    G.f32 = gf.f32;
    G.asw = c->apply_sweeps;
  }
  const size_t bytes = sizeof(double) * n;
  KFBI_TRY(cudaMemcpyAsync(c->ir_b, rhs, bytes, cudaMemcpyDeviceToDevice, s));
  KFBI_TRY(cudaMemcpyAsync(c->ir_x, x, bytes, cudaMemcpyDeviceToDevice, s));
  k_ir_init<<<1, 32, 0, s>>>(c->irctl, tol, max_iter, max_sweeps, ctx_sweep_cap(c));
  KFBI_TRY(cudaGetLastError());
  KFBI_CHECK(box_table_join(c, s));
  KFBI_TRY(cudaGraphLaunch(G.exec, s));
  *used = true;
  KFBI_TRY(cudaMemcpyAsync(x, c->ir_x, bytes, cudaMemcpyDeviceToDevice, s));
  if (dnormal != nullptr) KFBI_TRY(cudaMemcpyAsync(dnormal, c->ir_dn, bytes, cudaMemcpyDeviceToDevice, s));
  KFBI_TRY(cudaMemcpyAsync(c->host_irctl, c->irctl, sizeof(IrCtl), cudaMemcpyDeviceToHost, s));
  KFBI_TRY(cudaStreamSynchronize(s));
  const IrCtl& h = *c->host_irctl;
  c->launches += 1 + (long long)h.sweeps * (c->per_apply_launches[0] + 2) +
                 (long long)h.inner_bodies * G.inner_body_launches;
  out->iterations = h.total_its;
  out->restarts = h.total_cycles > h.sweeps - 1 ? h.total_cycles - (h.sweeps - 1) : 0;
  out->refinements = h.sweeps;
  out->rel_residual = h.rel;
  out->status = h.status;
  return KFBI_OK;
}

// dnormal (optional, mixed precision only): the refinement's float64 applies also write the
// normal derivative of the layer potential of the iterate; the last one belongs to the
// returned density. Set to nullptr on return when it was not produced.
kfbi_status solve_bie_impl(kfbi_ctx* c, int kind, const double* eps_v, const double* rhs, double tol, int max_iter,
                           int restart, double* x, kfbi_solve_info* info, double* dnormal) {
  cudaStream_t s = c->stream;
  const int n = c->n;
  const size_t bytes = sizeof(double) * n;
  const double* ev = nullptr;
  if (kind == KFBI_BIE_STEFAN_SL) {
    KFBI_TRY(cudaMemcpyAsync(c->gev, eps_v, bytes, cudaMemcpyDeviceToDevice, s));
    ev = c->gev;
  }
  kfbi_solve_info out{};
  // refined float64 applies of this solve (grids >= IR_APPLY_MIN_N): one correction sweep for
  // a tolerance of IR_ONE_SWEEP_TOL or looser; reset when the solve returns
  struct SweepScope {
    kfbi_ctx* c;
    ~SweepScope() { c->apply_sweeps = 0; }
  } sweep_scope{c};
  c->apply_sweeps = tol >= IR_ONE_SWEEP_TOL && c->grid_ir > 1 ? 1 : c->grid_ir;
  if (c->precision == KFBI_FP64) {
    int its = 0, cyc = 0, st = 0;
    double rel = 0.0;
    KFBI_TRY(cudaMemcpyAsync(c->gb, rhs, bytes, cudaMemcpyDeviceToDevice, s));
    KFBI_TRY(cudaMemcpyAsync(c->gx, x, bytes, cudaMemcpyDeviceToDevice, s));
    KFBI_CHECK(gmres_run(c, kind, false, ev, c->gb, c->gx, tol, max_iter, restart, false, false, &its, &cyc, &rel, &st));
    KFBI_TRY(cudaMemcpyAsync(x, c->gx, bytes, cudaMemcpyDeviceToDevice, s));
    out.iterations = its;
    out.restarts = cyc > 0 ? cyc - 1 : 0;
    out.refinements = 0;
    out.rel_residual = rel;
    out.status = st;
  } else {
    if (c->use_graphs && !c->timing) {
      bool used = false;
      KFBI_CHECK(solve_ir_graph(c, kind, rhs, tol, max_iter, restart, x, dnormal, &out, &used));
      if (used) {
        if (info) *info = out;
        return (kfbi_status)out.status;
      }
      c->use_graphs = false;  // keep the host-driven loops from now on
    }
    // iterative refinement: r = b - A64 x (float64 apply); solve A32 d = r by GMRES with
    // float32 grid applies from d = 0 to a tolerance the float32 operator resolves; x += d
    double* y = c->tmp_vals;                 // A64 x
    double* hres = (double*)c->host_counts;  // pinned scratch (2 doubles)
    int total_its = 0, total_cyc = 0, sweeps = 0, st = KFBI_OK;
    double rel = 1.0;
    const int max_sweeps = IR_MAX_SWEEPS;
    int layer = kind == KFBI_BIE_STEFAN_SL ? KFBI_SINGLE : KFBI_DOUBLE;
    while (true) {
      KFBI_CHECK(apply_enqueue(c, layer, false, x, y, dnormal, nullptr, kind, ev, nullptr));
      k_resid<<<1, 1024, 0, s>>>(rhs, y, c->gb, n, c->dint + 1);
      launched(c, 1);
      KFBI_TRY(cudaMemcpyAsync(hres, c->dint + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      KFBI_TRY(cudaStreamSynchronize(s));
      sweeps += 1;
      double rn = sqrt(hres[0]), bn = sqrt(hres[1]);
      rel = bn > 0 ? rn / bn : 0.0;
      if (rel <= tol) { st = KFBI_OK; break; }
      if (total_its >= max_iter || sweeps > max_sweeps) { st = KFBI_ERR_NOT_CONVERGED; break; }
      if (sweeps > ctx_sweep_cap(c)) { st = KFBI_ERR_TIMEOUT; break; }
      double inner = 0.5 * tol / rel;
      if (inner < 1e-7) inner = 1e-7;
      if (inner > 0.5) inner = 0.5;
      int its = 0, cyc = 0, ist = 0;
      double irel = 0.0;
      KFBI_CHECK(gmres_run(c, kind, true, ev, c->gb, c->gx, inner, max_iter - total_its, restart, true, true, &its,
                           &cyc, &irel, &ist));
      total_its += its;
      total_cyc += cyc;
      k_axpy_zero<<<cdiv(n, 256), 256, 0, s>>>(x, c->gx, n);
      launched(c, 1);
      if (ist == KFBI_ERR_TIMEOUT) { st = KFBI_ERR_TIMEOUT; break; }
    }
    out.iterations = total_its;
    out.restarts = total_cyc > sweeps - 1 ? total_cyc - (sweeps - 1) : 0;
    out.refinements = sweeps;
    out.rel_residual = rel;
    out.status = st;
  }
  if (info) *info = out;
  return (kfbi_status)out.status;
}

}  // namespace kfbi
