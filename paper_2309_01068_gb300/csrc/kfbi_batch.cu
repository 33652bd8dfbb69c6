// Many independent boundary integral equations in one CUDA graph (batched solves), and an
// autotuner for the launch shapes of each grid size. The paper solves one interface problem at
// a time (Sec. 4); a batch here runs the same per-instance method (the apply and GMRES of
// kfbi_solve_bie) for every instance, as independent branches of one graph launch.
//
// Branch of instance i: copies of its rhs and initial density into the instance's buffers,
// the start kernels of its solve, its solve loop (float64: the GMRES WHILE node; mixed: the
// refinement WHILE node with the inner GMRES WHILE node), and the copy of the density back.
// A final kernel gathers every instance's counters and status into one array, which the graph
// copies to pinned host memory: one launch and one synchronisation per batch solve.
#include <algorithm>
#include <chrono>
#include <map>
#include <vector>

#include "kfbi_internal.cuh"

namespace kfbi {

struct BatchRef {
  const GmresCtl* g;
  const IrCtl* ir;
};

struct BatchOut {
  int iterations, restarts, refinements, status, bodies, sweeps, pad0, pad1;
  double rel;
};

__global__ void k_batch_collect(const BatchRef* refs, int count, int mixed, BatchOut* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  BatchOut o{};
  if (refs[i].g == nullptr) {
    o.status = KFBI_ERR_STATE;
  } else if (mixed) {
    const IrCtl& r = *refs[i].ir;
    o.iterations = r.total_its;
    o.restarts = r.total_cycles > r.sweeps - 1 ? r.total_cycles - (r.sweeps - 1) : 0;
    o.refinements = r.sweeps;
    o.status = r.status;
    o.bodies = r.inner_bodies;
    o.sweeps = r.sweeps;
    o.rel = r.rel;
  } else {
    const GmresCtl& g = *refs[i].g;
    o.iterations = g.its;
    o.restarts = g.cycles > 0 ? g.cycles - 1 : 0;
    o.refinements = 0;
    o.status = g.status;
    o.bodies = g.bodies;
    o.rel = g.bnorm > 0.0 ? g.beta / g.bnorm : 0.0;
  }
  out[i] = o;
}

}  // namespace kfbi

using namespace kfbi;

struct kfbi_batch {
  int count = 0;
  int precision = KFBI_FP64;
  std::vector<kfbi_ctx*> ctx;
  cudaStream_t user = nullptr;   // caller's stream
  cudaStream_t own = nullptr;    // launch and capture stream
  cudaEvent_t ev = nullptr;
  BatchRef* d_refs = nullptr;
  BatchOut* d_out = nullptr;
  BatchOut* h_out = nullptr;     // pinned
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // what the cached graph was built for
  struct Key {
    long version;
    int cfg, m, cs, cap, n, f32;
    bool pdl;
    const double* rhs;
    double* x;
    bool operator==(const Key& o) const {
      return version == o.version && cfg == o.cfg && m == o.m && cs == o.cs && cap == o.cap && n == o.n &&
             f32 == o.f32 && pdl == o.pdl && rhs == o.rhs && x == o.x;
    }
  };
  std::vector<Key> keys;
  int key_kind = -1, key_max_iter = -1;
  double key_tol = -1.0;
  std::vector<int> body_launches;  // per instance, kernels per replayed (inner) body
};

static void batch_drop_graph(kfbi_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->keys.clear();
}

static kfbi_batch::Key batch_key(kfbi_ctx* c, int restart, int max_iter, const double* rhs, double* x) {
  kfbi_batch::Key k{};
  k.version = c->iface_version;
  k.cfg = c->cfg_version;
  k.n = c->have_iface ? c->n : 0;
  k.m = k.n > 0 ? restart_length(restart, k.n) : 0;
  const kfbi_ctx::GmfConfig gf = k.n > 0 ? gmf_select(c, k.n, k.m, c->precision == KFBI_MIXED) : kfbi_ctx::GmfConfig{};
  k.cs = gf.cs;
  k.f32 = gf.f32;
  k.cap = k.m > 0 ? body_cap(max_iter, k.m) : 0;
  k.pdl = false;
  k.rhs = rhs;
  k.x = x;
  return k;
}

// Builds the batch graph (see the file comment).
static kfbi_status batch_build(kfbi_batch* b, int kind, const double* const* rhs, double* const* x, double tol,
                               int max_iter, int restart) {
  batch_drop_graph(b);
  KFBI_TRY(cudaGraphCreate(&b->graph, 0));
  const bool mixed = b->precision == KFBI_MIXED;
  std::vector<cudaGraphNode_t> tails;
  std::vector<BatchRef> refs(b->count, BatchRef{nullptr, nullptr});
  b->body_launches.assign(b->count, 0);
  std::vector<kfbi_batch::Key> keys;
  kfbi_status st = KFBI_OK;
  for (int i = 0; i < b->count && st == KFBI_OK; ++i) {
    kfbi_ctx* c = b->ctx[i];
    keys.push_back(batch_key(c, restart, max_iter, rhs[i], x[i]));
    if (!c->have_iface || c->n < 1) continue;
    const kfbi_batch::Key& k = keys.back();
    const kfbi_ctx::GmfConfig gf = gmf_select(c, k.n, k.m, mixed);
    c->gm_m = k.m;
    c->gmf_last_cs = gf.cs;
    cudaStream_t saved = c->stream;
    const bool saved_pdl = c->use_pdl;
    c->stream = b->own;  // capture this instance's work through the batch's stream
    // no programmatic dependent launch inside a batch graph: on this driver the capture of a
    // programmatic edge into a graph that already holds other instances' loops was invalidated
    c->use_pdl = false;
    const size_t bytes = sizeof(double) * k.n;
    double* bdst = mixed ? c->ir_b : c->gb;
    double* xdst = mixed ? c->ir_x : c->gx;
    std::vector<cudaGraphNode_t> head;
    st = cap_begin(c, b->graph, nullptr, 0);
    if (st == KFBI_OK) {
      kfbi_status s1 = KFBI_OK;
      if (cudaMemcpyAsync(bdst, rhs[i], bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
          cudaMemcpyAsync(xdst, x[i], bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
        s1 = KFBI_ERR_CUDA;
      if (s1 == KFBI_OK) s1 = mixed ? ir_start_enqueue(c, tol, max_iter) : gmres_start_enqueue(c, tol, max_iter, k.m);
      st = cap_end(c, &head);
      if (s1 != KFBI_OK) st = s1;
    }
    cudaGraphNode_t loop{};
    if (st == KFBI_OK) {
      if (mixed)
        st = add_ir_nodes(c, b->graph, head.data(), head.size(), kind, false, k.m, gf, k.cap, &loop,
                          &b->body_launches[i]);
      else
        st = add_gmres_nodes(c, b->graph, head.data(), head.size(), kind, false, nullptr, c->gb, c->gx, k.cap, gf,
                             &loop, &b->body_launches[i]);
    }
    if (st == KFBI_OK) st = cap_begin(c, b->graph, &loop, 1);
    if (st == KFBI_OK) {
      kfbi_status s1 = cudaMemcpyAsync(x[i], xdst, bytes, cudaMemcpyDeviceToDevice, c->stream) == cudaSuccess
                           ? KFBI_OK
                           : KFBI_ERR_CUDA;
      std::vector<cudaGraphNode_t> tail;
      st = cap_end(c, &tail);
      if (s1 != KFBI_OK) st = s1;
      tails.insert(tails.end(), tail.begin(), tail.end());
    }
    c->stream = saved;
    c->use_pdl = saved_pdl;
    refs[i] = BatchRef{c->gctl, c->irctl};
  }
  if (st == KFBI_OK) {
    KFBI_TRY(cudaMemcpy(b->d_refs, refs.data(), sizeof(BatchRef) * b->count, cudaMemcpyHostToDevice));
    KFBI_TRY(cudaStreamBeginCaptureToGraph(b->own, b->graph, tails.empty() ? nullptr : tails.data(), nullptr,
                                           tails.size(), cudaStreamCaptureModeRelaxed));
    k_batch_collect<<<cdiv(b->count, 128), 128, 0, b->own>>>(b->d_refs, b->count, mixed ? 1 : 0, b->d_out);
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 =
        cudaMemcpyAsync(b->h_out, b->d_out, sizeof(BatchOut) * b->count, cudaMemcpyDeviceToHost, b->own);
    cudaGraph_t outg = nullptr;
    cudaError_t e3 = cudaStreamEndCapture(b->own, &outg);
    KFBI_TRY(e1);
    KFBI_TRY(e2);
    KFBI_TRY(e3);
    KFBI_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
    b->keys = keys;
    b->key_kind = kind;
    b->key_tol = tol;
    b->key_max_iter = max_iter;
  }
  if (st != KFBI_OK) {
    // a graph whose capture failed is released without cudaGraphDestroy: destroying such a
    // graph crashed inside the driver; the object is small and the failure path is rare
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->graph = nullptr;
    b->keys.clear();
    cudaGetLastError();
  }
  return st;
}

static kfbi_status batch_solve_impl(kfbi_batch* b, int kind, const double* const* rhs, double* const* x, double tol,
                                    int max_iter, int restart, kfbi_solve_info* infos) {
  bool fresh = b->exec != nullptr && b->key_kind == kind && b->key_tol == tol && b->key_max_iter == max_iter &&
               (int)b->keys.size() == b->count;
  for (int i = 0; fresh && i < b->count; ++i)
    fresh = b->keys[i] == batch_key(b->ctx[i], restart, max_iter, rhs[i], x[i]);
  if (!fresh) KFBI_CHECK(batch_build(b, kind, rhs, x, tol, max_iter, restart));
  KFBI_TRY(cudaEventRecord(b->ev, b->user));
  KFBI_TRY(cudaStreamWaitEvent(b->own, b->ev, 0));
  for (int i = 0; i < b->count; ++i) KFBI_CHECK(box_table_join(b->ctx[i], b->own));
  KFBI_TRY(cudaGraphLaunch(b->exec, b->own));
  KFBI_TRY(cudaStreamSynchronize(b->own));
  const bool mixed = b->precision == KFBI_MIXED;
  kfbi_status worst = KFBI_OK;
  for (int i = 0; i < b->count; ++i) {
    const BatchOut& o = b->h_out[i];
    kfbi_ctx* c = b->ctx[i];
    if (mixed)
      c->launches += 1 + (long long)o.sweeps * (c->per_apply_launches[0] + 2) + (long long)o.bodies * b->body_launches[i];
    else
      c->launches += 2 + (long long)o.bodies * b->body_launches[i];
    if (infos) {
      infos[i].iterations = o.iterations;
      infos[i].restarts = o.restarts;
      infos[i].refinements = o.refinements;
      infos[i].rel_residual = o.rel;
      infos[i].status = o.status;
    }
    if (o.status != KFBI_OK && (worst == KFBI_OK || worst == KFBI_ERR_NOT_CONVERGED)) worst = (kfbi_status)o.status;
  }
  return worst;
}

extern "C" {

kfbi_status kfbi_batch_create(int count, const kfbi_instance_desc* descs, int precision, kfbi_batch** out) {
  if (out == nullptr || descs == nullptr || count < 1 || (precision != KFBI_FP64 && precision != KFBI_MIXED))
    return KFBI_ERR_ARG;
  *out = nullptr;
  kfbi_batch* b = new kfbi_batch();
  b->count = count;
  b->precision = precision;
  b->ctx.assign(count, nullptr);
  kfbi_status st = KFBI_OK;
  for (int i = 0; i < count && st == KFBI_OK; ++i) {
    const kfbi_instance_desc& d = descs[i];
    st = kfbi_create(d.N, d.xmin, d.xmax, d.ymin, d.ymax, d.kappa, d.boxbc, precision, d.max_nodes, &b->ctx[i]);
  }
  if (st == KFBI_OK) {
    if (cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc((void**)&b->d_refs, sizeof(BatchRef) * count) != cudaSuccess ||
        cudaMalloc((void**)&b->d_out, sizeof(BatchOut) * count) != cudaSuccess ||
        cudaMallocHost((void**)&b->h_out, sizeof(BatchOut) * count) != cudaSuccess) {
      note_cuda_error(cudaGetLastError(), "kfbi_batch_create", __FILE__, __LINE__);
      st = KFBI_ERR_CUDA;
    }
  }
  if (st != KFBI_OK) {
    kfbi_batch_destroy(b);
    return st;
  }
  *out = b;
  return KFBI_OK;
}

void kfbi_batch_destroy(kfbi_batch* b) {
  if (b == nullptr) return;
  if (b->own) cudaStreamSynchronize(b->own);
  batch_drop_graph(b);
  for (kfbi_ctx* c : b->ctx)
    if (c) kfbi_destroy(c);
  if (b->d_refs) cudaFree(b->d_refs);
  if (b->d_out) cudaFree(b->d_out);
  if (b->h_out) cudaFreeHost(b->h_out);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->own) cudaStreamDestroy(b->own);
  delete b;
}

kfbi_status kfbi_batch_context(kfbi_batch* b, int i, kfbi_ctx** ctx) {
  if (b == nullptr || ctx == nullptr || i < 0 || i >= b->count) return KFBI_ERR_ARG;
  *ctx = b->ctx[i];
  return KFBI_OK;
}

kfbi_status kfbi_batch_set_stream(kfbi_batch* b, void* stream) {
  if (b == nullptr) return KFBI_ERR_ARG;
  b->user = (cudaStream_t)stream;
  return KFBI_OK;
}

kfbi_status kfbi_batch_solve(kfbi_batch* b, int kind, const double* const* rhs, double* const* density, double tol,
                             int max_iter, int restart, kfbi_solve_info* infos) {
  if (b == nullptr || rhs == nullptr || density == nullptr || !(tol > 0.0) || max_iter < 1 || restart < 1 ||
      restart > MAX_RESTART || (kind != KFBI_BIE_INTERIOR_DL && kind != KFBI_BIE_HS_EXTERIOR_MDL))
    return KFBI_ERR_ARG;
  for (int i = 0; i < b->count; ++i) {
    if (!b->ctx[i]->have_iface) return KFBI_ERR_STATE;
    if (rhs[i] == nullptr || density[i] == nullptr) return KFBI_ERR_ARG;
  }
  return batch_solve_impl(b, kind, rhs, density, tol, max_iter, restart, infos);
}

// Coordinate search over the launch shapes of each grid size N in the batch: the Gram-Schmidt
// form (16-CTA cluster, 8-CTA cluster, five kernels), the column pairs per block of the column
// transform (the kernel's default, 1, 2, 4) and, in the mixed form, the float32 column kernel
// (radix-16, four-step register FFTs, tensor-core contractions, radix-4). Each candidate is
// applied to every instance of that N
// and timed on the whole batch solve (second of two launches, so graph building is not
// timed); the fastest is kept. The solves run on scratch densities starting from zero.
kfbi_status kfbi_batch_autotune(kfbi_batch* b, int kind, const double* const* rhs, double tol, int max_iter,
                                int restart, double* best_ms) {
  if (b == nullptr || rhs == nullptr || !(tol > 0.0) || max_iter < 1 || restart < 1 || restart > MAX_RESTART)
    return KFBI_ERR_ARG;
  std::vector<double*> xs(b->count, nullptr);
  kfbi_status st = KFBI_OK;
  for (int i = 0; i < b->count && st == KFBI_OK; ++i) {
    kfbi_ctx* c = b->ctx[i];
    if (!c->have_iface) st = KFBI_ERR_STATE;
    else if (cudaMalloc((void**)&xs[i], sizeof(double) * c->n) != cudaSuccess) st = KFBI_ERR_CUDA;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (st == KFBI_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) st = KFBI_ERR_CUDA;
  auto run = [&](float* ms) -> kfbi_status {
    float best = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      for (int i = 0; i < b->count; ++i)
        if (cudaMemsetAsync(xs[i], 0, sizeof(double) * b->ctx[i]->n, b->own) != cudaSuccess) return KFBI_ERR_CUDA;
      KFBI_TRY(cudaEventRecord(e0, b->own));
      kfbi_status s = batch_solve_impl(b, kind, rhs, xs.data(), tol, max_iter, restart, nullptr);
      if (s != KFBI_OK && s != KFBI_ERR_NOT_CONVERGED) return s;
      KFBI_TRY(cudaEventRecord(e1, b->own));
      KFBI_TRY(cudaEventSynchronize(e1));
      float t = 0.0f;
      KFBI_TRY(cudaEventElapsedTime(&t, e0, e1));
      if (rep == 1) best = t;
    }
    *ms = best;
    return KFBI_OK;
  };
  std::map<int, std::vector<int>> classes;  // grid size -> instances
  for (int i = 0; i < b->count; ++i) classes[b->ctx[i]->N].push_back(i);
  auto apply = [&](const std::vector<int>& ids, int form, int pairs) {
    for (int i : ids) {
      kfbi_ctx* c = b->ctx[i];
      kfbi_set_option(c, KFBI_OPT_CLUSTER_GMRES, form == 2 ? 0 : 1);
      kfbi_set_option(c, KFBI_OPT_CLUSTER_SIZE, form == 0 ? 16 : (form == 1 ? 8 : 0));
      kfbi_set_option(c, KFBI_OPT_COL_PAIRS, pairs);
    }
  };
  float cur = 0.0f;
  if (st == KFBI_OK) st = run(&cur);
  const int forms[3] = {0, 1, 2}, pairs[4] = {0, 1, 2, 4};
  for (auto& kv : classes) {
    if (st != KFBI_OK) break;
    int best_form = 0, best_pairs = 0;
    apply(kv.second, best_form, best_pairs);
    if ((st = run(&cur)) != KFBI_OK) break;
    for (int f : forms) {
      if (f == best_form) continue;
      apply(kv.second, f, best_pairs);
      float t = 0.0f;
      if ((st = run(&t)) != KFBI_OK) break;
      if (t < cur) {
        cur = t;
        best_form = f;
      }
    }
    for (int p : pairs) {
      if (st != KFBI_OK || p == best_pairs) continue;
      apply(kv.second, best_form, p);
      float t = 0.0f;
      if ((st = run(&t)) != KFBI_OK) break;
      if (t < cur) {
        cur = t;
        best_pairs = p;
      }
    }
    apply(kv.second, best_form, best_pairs);
    // the float32 column transform: radix-16 register-resident kernel (0), four-step register
    // FFTs (1, N <= 1024), tensor-core contractions (2, N <= 256) or the radix-4 shared-memory
    // kernel (3); only the mixed form runs float32 applies
    if (b->precision == KFBI_MIXED && st == KFBI_OK) {
      auto apply_col = [&](int cf) {
        for (int i : kv.second) {
          kfbi_ctx* c = b->ctx[i];
          if (cf == 2 && kfbi_set_option(c, KFBI_OPT_COL_TC, 1) != KFBI_OK) return false;
          if (cf != 2) kfbi_set_option(c, KFBI_OPT_COL_TC, 0);
          kfbi_set_option(c, KFBI_OPT_COL_REG, cf == 1 ? 1 : 0);
          kfbi_set_option(c, KFBI_OPT_COL_RADIX4, cf == 3 ? 3 : 2);
        }
        return true;
      };
      int best_cf = 0;
      for (int cf = 1; cf <= 3 && st == KFBI_OK; ++cf) {
        if ((cf == 1 && kv.first > 1024) || (cf == 2 && kv.first > COL_TC_MAX_N)) continue;
        if (!apply_col(cf)) continue;
        float t = 0.0f;
        if ((st = run(&t)) != KFBI_OK) break;
        if (t < cur) {
          cur = t;
          best_cf = cf;
        }
      }
      apply_col(best_cf);
    }
  }
  if (best_ms) *best_ms = (double)cur;
  for (double* p : xs)
    if (p) cudaFree(p);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return st;
}

}  // extern "C"
