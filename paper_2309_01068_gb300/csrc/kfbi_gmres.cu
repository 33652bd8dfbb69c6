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
__global__ void k_gm_start(const double* b, double* x, double* gin, float* gin_f, double* V, int n, GmresCtl* ctl,
                           int zero_guess) {
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

// --------------------------------------------------------------------------- host side
static kfbi_status body(kfbi_ctx* c, int kind, bool fp32, const double* eps_v, const double* b, double* x) {
  cudaStream_t s = c->stream;
  const int n = c->n;
  const int* done = &c->gctl->done;
  int layer = kind == KFBI_BIE_STEFAN_SL ? KFBI_SINGLE : KFBI_DOUBLE;
  KFBI_CHECK(apply_enqueue(c, layer, fp32, c->gin, c->gw, nullptr, nullptr, kind, eps_v, done, c->gin_f));
  const int ldv = c->max_nodes;
  const int dblocks = c->gm_m + 1;
  const int ublocks = cdiv(n, 32);
  launched(c, 5);
  k_gm_dots<<<dblocks, GM_THREADS, 0, s>>>(c->gctl, c->gV, ldv, c->gw, b, c->gr, n, c->gpart, 0);
  k_gm_update<<<ublocks, 32 * UPD_WARPS, 0, s>>>(c->gctl, c->gV, ldv, c->gw, n, c->gpart, 0);
  k_gm_dots<<<dblocks, GM_THREADS, 0, s>>>(c->gctl, c->gV, ldv, c->gw, b, c->gr, n, c->gpart, 1);
  k_gm_update<<<ublocks, 32 * UPD_WARPS, 0, s>>>(c->gctl, c->gV, ldv, c->gw, n, c->gpart, 1);
  k_gm_finish<<<GM_BLOCKS, GM_THREADS, 0, s>>>(c->gctl, c->gV, ldv, c->gw, c->gr, x, c->gin, c->gin_f, n);
  KFBI_TRY(cudaGetLastError());
  return KFBI_OK;
}

static int body_cap(int max_iter, int m) { return 2 * max_iter + 2 * (max_iter / m) + 8; }

// Builds the graph of one solve: a conditional WHILE node whose body (captured from the
// stream) is one GMRES iteration followed by k_gm_cond.
static kfbi_status build_graph(kfbi_ctx* c, kfbi_ctx::SolveGraph& G, int kind, bool fp32, const double* eps_v,
                               const double* b, double* x, int cap) {
  if (G.exec) cudaGraphExecDestroy(G.exec);
  if (G.graph) cudaGraphDestroy(G.graph);
  G.exec = nullptr;
  G.graph = nullptr;
  G.version = -1;
  KFBI_TRY(cudaGraphCreate(&G.graph, 0));
  cudaGraphConditionalHandle h;
  KFBI_TRY(cudaGraphConditionalHandleCreate(&h, G.graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  KFBI_TRY(cudaGraphAddNode(&node, G.graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
  cudaStream_t s = c->stream;
  KFBI_TRY(cudaStreamBeginCaptureToGraph(s, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  c->capturing = true;
  const long long l0 = c->launches;
  kfbi_status st = body(c, kind, fp32, eps_v, b, x);
  if (st == KFBI_OK) k_gm_cond<<<1, 32, 0, s>>>(c->gctl, h, cap);
  c->launches = l0;  // capture launches nothing; replays are counted per body
  c->capturing = false;
  cudaGraph_t out = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &out);
  if (st != KFBI_OK) return st;
  KFBI_TRY(e);
  KFBI_TRY(cudaGetLastError());
  KFBI_TRY(cudaGraphInstantiate(&G.exec, G.graph, 0));
  G.version = c->iface_version;
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
  const int cap = body_cap(max_iter, m);
  const size_t hdr = offsetof(GmresCtl, g);
  launched(c, 2);
  k_gm_init<<<1, 32, 0, s>>>(c->gctl, tol, max_iter, m, trust ? 1 : 0);
  k_gm_start<<<1, 1024, 0, s>>>(b, x, c->gin, c->gin_f, c->gV, n, c->gctl, zero_guess ? 1 : 0);
  bool graphed = false;
  if (c->use_graphs && !c->timing) {
    kfbi_ctx::SolveGraph& G = c->sgraph[kind][fp32 ? 1 : 0];
    kfbi_status st = KFBI_OK;
    if (G.exec == nullptr || G.version != c->iface_version || G.m != m) {
      st = build_graph(c, G, kind, fp32, eps_v, b, x, cap);
      G.m = m;
    }
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
    // bodies replayed by the graph: one apply plus five Gram-Schmidt kernels and the loop test
    c->launches += (long long)c->host_gctl->bodies * (c->per_apply_launches[fp32 ? 1 : 0] + 6);
  } else {
    int launched_bodies = 0, chunk = 2;
    while (true) {
      for (int q = 0; q < chunk; ++q) KFBI_CHECK(body(c, kind, fp32, eps_v, b, x));
      launched_bodies += chunk;
      KFBI_TRY(cudaMemcpyAsync(c->host_gctl, c->gctl, hdr, cudaMemcpyDeviceToHost, s));
      KFBI_TRY(cudaStreamSynchronize(s));
      if (c->host_gctl->done) break;
      if (launched_bodies > cap) return KFBI_ERR_TIMEOUT;
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

kfbi_status solve_bie_impl(kfbi_ctx* c, int kind, const double* eps_v, const double* rhs, double tol, int max_iter,
                           int restart, double* x, kfbi_solve_info* info) {
  cudaStream_t s = c->stream;
  const int n = c->n;
  const size_t bytes = sizeof(double) * n;
  const double* ev = nullptr;
  if (kind == KFBI_BIE_STEFAN_SL) {
    KFBI_TRY(cudaMemcpyAsync(c->gev, eps_v, bytes, cudaMemcpyDeviceToDevice, s));
    ev = c->gev;
  }
  kfbi_solve_info out{};
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
    // iterative refinement: r = b - A64 x (float64 apply); solve A32 d = r by GMRES with
    // float32 grid applies from d = 0 to a tolerance the float32 operator resolves; x += d
    double* y = c->tmp_vals;                 // A64 x
    double* hres = (double*)c->host_counts;  // pinned scratch (2 doubles)
    int total_its = 0, total_cyc = 0, sweeps = 0, st = KFBI_OK;
    double rel = 1.0;
    const int max_sweeps = 12;
    int layer = kind == KFBI_BIE_STEFAN_SL ? KFBI_SINGLE : KFBI_DOUBLE;
    while (true) {
      KFBI_CHECK(apply_enqueue(c, layer, false, x, y, nullptr, nullptr, kind, ev, nullptr));
      k_resid<<<1, 1024, 0, s>>>(rhs, y, c->gb, n, c->dint + 1);
      launched(c, 1);
      KFBI_TRY(cudaMemcpyAsync(hres, c->dint + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      KFBI_TRY(cudaStreamSynchronize(s));
      sweeps += 1;
      double rn = sqrt(hres[0]), bn = sqrt(hres[1]);
      rel = bn > 0 ? rn / bn : 0.0;
      if (rel <= tol) { st = KFBI_OK; break; }
      if (total_its >= max_iter || sweeps > max_sweeps) { st = KFBI_ERR_NOT_CONVERGED; break; }
      double inner = 0.5 * tol / rel;
      if (inner < 1e-5) inner = 1e-5;
      if (inner > 0.5) inner = 0.5;
      int its = 0, cyc = 0, ist = 0;
      double irel = 0.0;
      KFBI_CHECK(gmres_run(c, kind, true, ev, c->gb, c->gx, inner, max_iter - total_its, restart, true, true, &its,
                           &cyc, &irel, &ist));
      if (ist == KFBI_ERR_TIMEOUT) return KFBI_ERR_TIMEOUT;
      total_its += its;
      total_cyc += cyc;
      k_axpy_zero<<<cdiv(n, 256), 256, 0, s>>>(x, c->gx, n);
      launched(c, 1);
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
