#include <algorithm>
// C ABI of libkfbi (include/kfbi.h): context lifetime, constant tables and the entry
// points that validate arguments and enqueue the kernels of the other translation units.
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "kfbi_internal.cuh"

namespace kfbi {

kfbi_status set_interface_impl(kfbi_ctx* c, int n, const double* xy);
kfbi_status solve_bie_impl(kfbi_ctx* c, int kind, const double* eps_v, const double* rhs, double tol, int max_iter,
                           int restart, double* x, kfbi_solve_info* info,
                           double* dnormal = nullptr);

static thread_local char g_last_error[512] = {0};

void note_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_last_error, sizeof g_last_error, "%s: %s (%s:%d)", cudaGetErrorName(e), what, file, line);
  if (getenv("KFBI_VERBOSE")) fprintf(stderr, "libkfbi: %s\n", g_last_error);
}

// sin(pi m / (2N)) for m < 4N; box eigenvalues -4 sin^2(pi (k + s) / (2N)) / h^2 with s = 1
// (Dirichlet-0, DST-II mode k) or s = 0 (Neumann-0, DCT-II mode k); FFT twiddles
// e^{-2 pi i m / N} for m < N.
// rinv[k][l] = 1 / (lam[l] + lam[k] - kappa)
__global__ void k_rinv(int N, const double* lam, double kappa, double* rinv) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)N * N) return;
  const int k = (int)(t / N), l = (int)(t - (long)k * N);
  rinv[t] = 1.0 / (lam[l] + lam[k] - kappa);
}

__global__ void k_init_tables(int N, double h, int neumann, double* tab, float* tab_f, double* lam, float* lam_f,
                              double* tw, float* tw_f) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < 4 * N) {
    double s = sinpi((double)m / (2.0 * N));
    tab[m] = s;
    tab_f[m] = (float)s;
  }
  if (m < N) {
    double sk = sinpi(((double)m + (neumann ? 0.0 : 1.0)) / (2.0 * N));
    double l = -4.0 * sk * sk / (h * h);
    lam[m] = l;
    lam_f[m] = (float)l;
  }
  if (m < N) {
    double s, c;
    sincospi(2.0 * (double)m / (double)N, &s, &c);
    tw[2 * m] = c;
    tw[2 * m + 1] = -s;
    tw_f[2 * m] = (float)c;
    tw_f[2 * m + 1] = (float)-s;
  }
}

__global__ void k_stage_twiddles(int N, int Ns, int off, const double* tw, double* out, float* out_f) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * Ns) return;
  int r = t / Ns + 1, jm = t - (r - 1) * Ns;
  long m = (long)r * jm * (N / (4 * Ns));  // < N
  out[2 * (off + t)] = tw[2 * m];
  out[2 * (off + t) + 1] = tw[2 * m + 1];
  out_f[2 * (off + t)] = (float)tw[2 * m];
  out_f[2 * (off + t) + 1] = (float)tw[2 * m + 1];
}

template <typename P>
static kfbi_status dalloc(P** p, size_t count) {
  KFBI_TRY(cudaMalloc((void**)p, sizeof(P) * (count > 0 ? count : 1)));
  return KFBI_OK;
}

kfbi_status ensure_cross_capacity(kfbi_ctx* c, int ncr) {
  if (ncr <= c->cap_cross) return KFBI_OK;
  int cap = ncr + ncr / 2 + 64;
  cudaStreamSynchronize(c->stream);
  cudaFree(c->cr_kind); cudaFree(c->cr_line); cudaFree(c->cr_seg); cudaFree(c->cr_first);
  cudaFree(c->cr_alpha); cudaFree(c->cr_xi); cudaFree(c->tgeo); cudaFree(c->tgeo_f); cudaFree(c->irr);
  cudaFree(c->tstart); cudaFree(c->tstart_f); cudaFree(c->jumps);
  cudaFree(c->irr_ci); cudaFree(c->arm_slot); cudaFree(c->arm_rev); cudaFree(c->arm_coef);
  cudaFree(c->corr_val); cudaFree(c->corr_pos);
  c->irr_ci = nullptr; c->arm_slot = nullptr; c->arm_rev = nullptr; c->arm_coef = nullptr;
  c->corr_val = nullptr; c->corr_pos = nullptr;
  c->cr_kind = c->cr_line = c->cr_seg = c->cr_first = nullptr;
  c->cr_alpha = c->cr_xi = nullptr;
  c->tgeo = nullptr; c->tgeo_f = nullptr; c->irr = nullptr;
  c->tstart = nullptr; c->tstart_f = nullptr; c->jumps = nullptr;
  c->cap_cross = c->cap_irr = 0;
  KFBI_CHECK(dalloc(&c->cr_kind, cap));
  KFBI_CHECK(dalloc(&c->cr_line, cap));
  KFBI_CHECK(dalloc(&c->cr_seg, cap));
  KFBI_CHECK(dalloc(&c->cr_first, cap));
  KFBI_CHECK(dalloc(&c->cr_alpha, cap));
  KFBI_CHECK(dalloc(&c->cr_xi, cap));
  KFBI_CHECK(dalloc(&c->tgeo, (size_t)cap + c->max_nodes));
  KFBI_CHECK(dalloc(&c->tgeo_f, (size_t)cap + c->max_nodes));
  int cap_irr = 2 * cap + 64;
  KFBI_CHECK(dalloc(&c->irr, cap_irr));
  KFBI_CHECK(dalloc(&c->irr_ci, cap_irr));
  KFBI_CHECK(dalloc(&c->arm_slot, 4 * (size_t)cap_irr));
  KFBI_CHECK(dalloc(&c->corr_val, cap_irr));
  KFBI_CHECK(dalloc(&c->corr_pos, cap_irr));
  KFBI_CHECK(dalloc(&c->arm_rev, 2 * (size_t)cap));
  KFBI_CHECK(dalloc(&c->arm_coef, 4 * (size_t)cap));
  KFBI_CHECK(dalloc(&c->tstart, 2 * (size_t)TSTART_STRIDE * ((size_t)cap + c->max_nodes)));
  KFBI_CHECK(dalloc(&c->tstart_f, 2 * (size_t)TSTART_STRIDE * ((size_t)cap + c->max_nodes)));
  KFBI_CHECK(dalloc(&c->jumps, 6 * ((size_t)cap + c->max_nodes)));
  c->cap_cross = cap;
  c->cap_irr = cap_irr;
  c->layout_version += 1;
  return KFBI_OK;
}

static void free_all(kfbi_ctx* c) {
  void* ptrs[] = {c->sintab, c->sintab_f, c->lam, c->lam_f, c->twN, c->twN_f, c->xy, c->twn, c->icoef, c->fine, c->twM,
                  c->seg_count, c->seg_off, c->cr_kind, c->cr_line, c->cr_seg, c->cr_first, c->cr_alpha, c->cr_xi,
                  c->tgeo, c->tgeo_f, c->rinv, c->stencil_f, c->dens_f, c->stw, c->stw_d, c->hcount, c->vcount, c->hid, c->vid, c->side, c->rowcnt, c->row_ptr, c->irr, c->stencil,
                  c->probe_mark, c->prow_cnt, c->prow_ptr, c->probe_i, c->probe_j, c->flags, c->counts, c->dcoef, c->dint,
                  c->boxg, c->facespec, c->spec, c->rowinfo, c->twn_f, c->tstart, c->tstart_f, c->jumps, c->npack, c->boxK, c->boxK_f,
                  c->npack_f, c->prow_list, c->probe_val, c->tmp_vals, c->gctl, c->gV, c->gVf, c->gpart, c->gw,
                  c->gin, c->gin_f, c->gb, c->gx, c->gr, c->zero_flag, c->irctl, c->ir_b, c->ir_x, c->ir_dn,
                  c->col_fwd, c->col_inv, c->col_tmp, c->col_tc_err, c->irr_ci, c->arm_slot, c->arm_rev,
                  c->arm_coef, c->corr_val, c->corr_pos, c->ir_grid};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->host_counts) cudaFreeHost(c->host_counts);
  if (c->host_gctl) cudaFreeHost(c->host_gctl);
  if (c->host_irctl) cudaFreeHost(c->host_irctl);
  for (auto& row : c->irgraph)
    for (auto& g : row) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.graph) cudaGraphDestroy(g.graph);
    }
  for (auto& row : c->sgraph)
    for (auto& g : row) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.graph) cudaGraphDestroy(g.graph);
    }
  if (c->gev) cudaFree(c->gev);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_boxK) cudaEventDestroy(c->ev_boxK);
  if (c->ev_boxK0) cudaEventDestroy(c->ev_boxK0);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->aux) cudaStreamDestroy(c->aux);
  if (c->own) cudaStreamDestroy(c->own);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->tev) {
    for (int i = 0; i < 2 * TIMING_CAP; ++i)
      if (c->tev[i]) cudaEventDestroy(c->tev[i]);
    delete[] c->tev;
  }
  delete[] c->tprec;
}

static kfbi_status create_impl(int N, double xmin, double xmax, double ymin, double ymax, double kappa, int boxbc,
                               int precision, int max_nodes, kfbi_ctx** out) {
  kfbi_ctx* c = new kfbi_ctx();
  *out = c;
  c->N = N;
  c->logN = ilog2(N);
  c->xmin = xmin; c->xmax = xmax; c->ymin = ymin; c->ymax = ymax;
  c->h = (xmax - xmin) / N;
  c->kappa = kappa;
  c->boxbc = boxbc;
  c->precision = precision;
  c->max_nodes = max_nodes;
  const size_t NN = (size_t)N * N;
  const int M = SUBSAMPLES * max_nodes;
  const int nk = max_nodes / 2 + 1;
  KFBI_CHECK(dalloc(&c->sintab, 4 * (size_t)N));
  KFBI_CHECK(dalloc(&c->sintab_f, 4 * (size_t)N));
  KFBI_CHECK(dalloc(&c->lam, N));
  if ((size_t)N * N * sizeof(double) <= RINV_MAX_BYTES) KFBI_CHECK(dalloc(&c->rinv, (size_t)N * N));
  KFBI_CHECK(dalloc(&c->lam_f, N));
  KFBI_CHECK(dalloc(&c->twN, 2 * (size_t)N));
  KFBI_CHECK(dalloc(&c->twN_f, 2 * (size_t)N));
  KFBI_CHECK(dalloc(&c->xy, 2 * (size_t)max_nodes));
  KFBI_CHECK(dalloc(&c->twn, 2 * (size_t)max_nodes));
  KFBI_CHECK(dalloc(&c->twn_f, 2 * (size_t)max_nodes));
  KFBI_CHECK(dalloc(&c->npack, 4 * (size_t)max_nodes));
  KFBI_CHECK(dalloc(&c->npack_f, 4 * (size_t)max_nodes));
  if (boxbc == KFBI_BOX_FREESPACE_DL && (size_t)4 * N * box_ld(max_nodes) * 12 <= BOXK_MAX_BYTES) {
    KFBI_CHECK(dalloc(&c->boxK, (size_t)4 * N * box_ld(max_nodes)));
    KFBI_CHECK(dalloc(&c->boxK_f, (size_t)4 * N * box_ld(max_nodes)));
  }
  KFBI_CHECK(dalloc(&c->prow_list, N + 1));
  KFBI_CHECK(dalloc(&c->facespec, 2 * (size_t)N));
  KFBI_CHECK(dalloc(&c->icoef, 4 * (size_t)nk));
  KFBI_CHECK(dalloc(&c->fine, 2 * (size_t)M));
  KFBI_CHECK(dalloc(&c->twM, 2 * (size_t)M));
  KFBI_CHECK(dalloc(&c->seg_count, 2 * (size_t)M + 1));
  KFBI_CHECK(dalloc(&c->seg_off, 2 * (size_t)M + 1));
  KFBI_CHECK(dalloc(&c->hcount, NN));
  KFBI_CHECK(dalloc(&c->vcount, NN));
  KFBI_CHECK(dalloc(&c->hid, NN));
  KFBI_CHECK(dalloc(&c->vid, NN));
  KFBI_CHECK(dalloc(&c->side, NN));
  KFBI_CHECK(dalloc(&c->rowcnt, N + 1));
  KFBI_CHECK(dalloc(&c->row_ptr, N + 1));
  KFBI_CHECK(dalloc(&c->stencil, max_nodes));
  KFBI_CHECK(dalloc(&c->stencil_f, max_nodes));
  KFBI_CHECK(dalloc(&c->dens_f, max_nodes));
  KFBI_CHECK(dalloc(&c->stw, 2 * (size_t)N));
  KFBI_CHECK(dalloc(&c->stw_d, 2 * (size_t)N));
  KFBI_CHECK(dalloc(&c->probe_mark, NN));
  KFBI_CHECK(dalloc(&c->prow_cnt, N + 1));
  KFBI_CHECK(dalloc(&c->prow_ptr, N + 1));
  KFBI_CHECK(dalloc(&c->probe_i, 6 * (size_t)max_nodes));
  KFBI_CHECK(dalloc(&c->probe_j, 6 * (size_t)max_nodes));
  KFBI_CHECK(dalloc(&c->flags, 4));
  KFBI_CHECK(dalloc(&c->counts, 8));
  KFBI_TRY(cudaMallocHost((void**)&c->host_counts, 16 * sizeof(int)));
  KFBI_CHECK(dalloc(&c->dcoef, 2 * (size_t)nk));
  KFBI_CHECK(dalloc(&c->dint, 8));
  KFBI_CHECK(dalloc(&c->boxg, 4 * (size_t)N));
  KFBI_CHECK(dalloc(&c->spec, NN));
  // the solved grid of the float64 applies that refine with float32 solves (see apply_t)
  if (c->precision == KFBI_MIXED && c->boxbc != KFBI_BOX_FREESPACE_DL && N >= IR_APPLY_MIN_N)
    KFBI_CHECK(dalloc(&c->ir_grid, NN));
  KFBI_CHECK(dalloc(&c->rowinfo, 2 * (size_t)N));
  KFBI_CHECK(dalloc(&c->probe_val, 6 * (size_t)max_nodes));
  KFBI_CHECK(dalloc(&c->tmp_vals, max_nodes));
  KFBI_CHECK(dalloc(&c->gctl, 1));
  KFBI_TRY(cudaMallocHost((void**)&c->host_gctl, sizeof(GmresCtl)));
  KFBI_CHECK(dalloc(&c->gV, (size_t)(MAX_RESTART + 1) * max_nodes));
  if (precision == KFBI_MIXED) KFBI_CHECK(dalloc(&c->gVf, (size_t)(MAX_RESTART + 1) * max_nodes));
  KFBI_CHECK(dalloc(&c->gpart, ((size_t)max_nodes / 32 + MAX_RESTART + 2) * (MAX_RESTART + 1)));
  KFBI_CHECK(dalloc(&c->gw, max_nodes));
  KFBI_CHECK(dalloc(&c->gin, max_nodes));
  KFBI_CHECK(dalloc(&c->gin_f, max_nodes));
  KFBI_CHECK(dalloc(&c->gb, max_nodes));
  KFBI_CHECK(dalloc(&c->gx, max_nodes));
  KFBI_CHECK(dalloc(&c->gr, max_nodes));
  KFBI_CHECK(dalloc(&c->irctl, 1));
  KFBI_TRY(cudaMallocHost((void**)&c->host_irctl, sizeof(IrCtl)));
  KFBI_CHECK(dalloc(&c->ir_b, max_nodes));
  KFBI_CHECK(dalloc(&c->ir_x, max_nodes));
  KFBI_CHECK(dalloc(&c->ir_dn, max_nodes));
  KFBI_CHECK(dalloc(&c->zero_flag, 4));
  KFBI_TRY(cudaMemset(c->zero_flag, 0, 4 * sizeof(int)));
  KFBI_TRY(cudaMemset(c->hcount, 0, NN * sizeof(int)));
  KFBI_TRY(cudaMemset(c->vcount, 0, NN * sizeof(int)));
  KFBI_TRY(cudaMemset(c->probe_mark, 0, NN * sizeof(int)));
  KFBI_TRY(cudaMemset(c->gctl, 0, sizeof(GmresCtl)));
  KFBI_TRY(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
  KFBI_TRY(cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking));
  KFBI_TRY(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
  KFBI_TRY(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
  c->user = cudaStreamLegacy;
  c->user_default = true;
  c->stream = c->own;
  KFBI_TRY(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  KFBI_TRY(cudaEventCreateWithFlags(&c->ev_boxK, cudaEventDisableTiming));
  KFBI_TRY(cudaEventCreateWithFlags(&c->ev_boxK0, cudaEventDisableTiming));
  KFBI_TRY(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  KFBI_CHECK(ensure_cross_capacity(c, 4096));
  KFBI_CHECK(dalloc(&c->gev, max_nodes));
  KFBI_CHECK(apply_setup_attributes(c));
  KFBI_CHECK(geometry_setup_attributes());
  launched(c, 1);
  k_init_tables<<<cdiv(4L * N, 256), 256, 0, c->own>>>(N, c->h, boxbc == KFBI_BOX_NEUMANN0, c->sintab, c->sintab_f,
                                                     c->lam, c->lam_f, c->twN, c->twN_f);
  KFBI_TRY(cudaGetLastError());
  if (c->rinv != nullptr) {
    launched(c, 1);
    k_rinv<<<cdiv((long)N * N, 256), 256, 0, c->own>>>(N, c->lam, kappa, c->rinv);
  }
  // staged twiddles of the Stockham FFT: for each radix-4 stage with span Ns (first stage
  // radix 2 when log2 N is odd), w^{r jm N / (4 Ns)} at [off + (r-1) Ns + jm], r = 1..3
  {
    int off = 0;
    for (int Ns = (c->logN & 1) ? 2 : 1; Ns < N; Ns <<= 2) {
      k_stage_twiddles<<<cdiv(3L * Ns, 256), 256, 0, c->own>>>(N, Ns, off, c->twN, c->stw_d, c->stw);
      launched(c, 1);
      off += 3 * Ns;
    }
  }
  KFBI_TRY(cudaGetLastError());
  KFBI_TRY(cudaStreamSynchronize(c->own));
  return KFBI_OK;
}

static bool ctx_ok(const kfbi_ctx* c) { return c != nullptr; }

}  // namespace kfbi

using namespace kfbi;

extern "C" {

kfbi_status kfbi_create(int N, double xmin, double xmax, double ymin, double ymax, double kappa, int boxbc,
                        int precision, int max_nodes, kfbi_ctx** out) {
  if (out == nullptr) return KFBI_ERR_ARG;
  *out = nullptr;
  if (N < 16 || N > 4096 || (N & (N - 1)) != 0) return KFBI_ERR_ARG;
  if (!(xmax > xmin) || !(ymax > ymin)) return KFBI_ERR_ARG;
  double hx = (xmax - xmin) / N, hy = (ymax - ymin) / N;
  if (fabs(hx - hy) > 1e-12 * hx) return KFBI_ERR_ARG;
  if (!(kappa >= 0.0) || !std::isfinite(kappa)) return KFBI_ERR_ARG;
  if (boxbc < KFBI_BOX_DIRICHLET0 || boxbc > KFBI_BOX_FREESPACE_DL) return KFBI_ERR_ARG;
  if (precision != KFBI_FP64 && precision != KFBI_MIXED) return KFBI_ERR_ARG;
  if (max_nodes < 8 || max_nodes > (1 << 16)) return KFBI_ERR_ARG;
  if (boxbc == KFBI_BOX_NEUMANN0 && kappa == 0.0) return KFBI_ERR_SINGULAR;
  if (boxbc == KFBI_BOX_FREESPACE_DL && kappa != 0.0) return KFBI_ERR_ARG;
  kfbi_ctx* c = nullptr;
  kfbi_status st = create_impl(N, xmin, xmax, ymin, ymax, kappa, boxbc, precision, max_nodes, &c);
  if (st != KFBI_OK) {
    if (c) {
      free_all(c);
      delete c;
    }
    return st;
  }
  *out = c;
  return KFBI_OK;
}

void kfbi_destroy(kfbi_ctx* c) {
  if (c == nullptr) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->aux) cudaStreamSynchronize(c->aux);
  free_all(c);
  delete c;
}

kfbi_status kfbi_set_stream(kfbi_ctx* c, void* stream) {
  if (!ctx_ok(c)) return KFBI_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  c->user_default = st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread;
  c->user = st == nullptr ? cudaStreamLegacy : st;
  c->stream = c->user_default ? c->own : st;
  return KFBI_OK;
}

kfbi_status kfbi_set_interface(kfbi_ctx* c, int n, const double* xy) {
  if (!ctx_ok(c) || xy == nullptr) return KFBI_ERR_ARG;
  if (n < 8) return KFBI_ERR_ARG;
  if (n > c->max_nodes) return KFBI_ERR_CAPACITY;
  KFBI_TRY(stream_enter(c));
  kfbi_status st = set_interface_impl(c, n, xy);
  KFBI_TRY(stream_exit(c));
  return st;
}

kfbi_status kfbi_apply_layer_potential(kfbi_ctx* c, int layer, const double* density, double* values,
                                       double* dnormal, double* grid) {
  if (!ctx_ok(c)) return KFBI_ERR_ARG;
  if (!c->have_iface) return KFBI_ERR_STATE;
  if (density == nullptr || values == nullptr) return KFBI_ERR_ARG;
  if (layer != KFBI_SINGLE && layer != KFBI_DOUBLE) return KFBI_ERR_ARG;
  if (c->boxbc == KFBI_BOX_FREESPACE_DL && layer != KFBI_DOUBLE) return KFBI_ERR_ARG;
  KFBI_TRY(stream_enter(c));
  kfbi_status st = apply_enqueue(c, layer, c->precision == KFBI_MIXED, density, values, dnormal, grid, -1, nullptr,
                                 nullptr);
  KFBI_TRY(stream_exit(c));
  return st;
}

kfbi_status kfbi_bie_apply(kfbi_ctx* c, int kind, const double* eps_v, const double* x, double* y) {
  if (!ctx_ok(c) || x == nullptr || y == nullptr) return KFBI_ERR_ARG;
  if (kind < KFBI_BIE_INTERIOR_DL || kind > KFBI_BIE_STEFAN_SL) return KFBI_ERR_ARG;
  if (kind == KFBI_BIE_STEFAN_SL && eps_v == nullptr) return KFBI_ERR_ARG;
  if (kind == KFBI_BIE_STEFAN_SL && c->boxbc == KFBI_BOX_FREESPACE_DL) return KFBI_ERR_ARG;
  if (!c->have_iface) return KFBI_ERR_STATE;
  int layer = kind == KFBI_BIE_STEFAN_SL ? KFBI_SINGLE : KFBI_DOUBLE;
  KFBI_TRY(stream_enter(c));
  kfbi_status st = apply_enqueue(c, layer, c->precision == KFBI_MIXED, x, y, nullptr, nullptr, kind, eps_v, nullptr);
  KFBI_TRY(stream_exit(c));
  return st;
}

kfbi_status kfbi_solve_bie(kfbi_ctx* c, int kind, const double* eps_v, const double* rhs, double tol, int max_iter,
                           int restart, double* density, kfbi_solve_info* info) {
  if (!ctx_ok(c) || rhs == nullptr || density == nullptr) return KFBI_ERR_ARG;
  if (kind < KFBI_BIE_INTERIOR_DL || kind > KFBI_BIE_STEFAN_SL) return KFBI_ERR_ARG;
  if (kind == KFBI_BIE_STEFAN_SL && eps_v == nullptr) return KFBI_ERR_ARG;
  if (kind == KFBI_BIE_STEFAN_SL && c->boxbc == KFBI_BOX_FREESPACE_DL) return KFBI_ERR_ARG;
  if (!(tol > 0.0) || max_iter < 1 || restart < 1 || restart > MAX_RESTART) return KFBI_ERR_ARG;
  if (!c->have_iface) return KFBI_ERR_STATE;
  KFBI_TRY(stream_enter(c));
  kfbi_status st = solve_bie_impl(c, kind, eps_v, rhs, tol, max_iter, restart, density, info);
  KFBI_TRY(stream_exit(c));
  return st;
}

kfbi_status kfbi_grid_solve(kfbi_ctx* c, const double* rhs, double* u) {
  if (!ctx_ok(c) || rhs == nullptr || u == nullptr) return KFBI_ERR_ARG;
  KFBI_TRY(stream_enter(c));
  kfbi_status st = grid_solve_enqueue(c, rhs, u);
  KFBI_TRY(stream_exit(c));
  return st;
}

kfbi_status kfbi_grid_solve_mixed(kfbi_ctx* c, const double* rhs, double* u, int sweeps) {
  if (!ctx_ok(c) || rhs == nullptr || u == nullptr || rhs == u || sweeps < 0 || sweeps > 8) return KFBI_ERR_ARG;
  if (c->precision != KFBI_MIXED) return KFBI_ERR_ARG;
  KFBI_TRY(stream_enter(c));
  kfbi_status st = grid_solve_mixed_enqueue(c, rhs, u, sweeps);
  KFBI_TRY(stream_exit(c));
  return st;
}

kfbi_status kfbi_interp_grid(kfbi_ctx* c, const double* grid, double* values) {
  if (!ctx_ok(c) || grid == nullptr || values == nullptr) return KFBI_ERR_ARG;
  if (!c->have_iface) return KFBI_ERR_STATE;
  KFBI_TRY(stream_enter(c));
  kfbi_status st = interp_grid_enqueue(c, grid, values);
  KFBI_TRY(stream_exit(c));
  return st;
}

kfbi_status kfbi_interface_stats(kfbi_ctx* c, int* n_crossings, int* n_irregular, int* n_probes) {
  if (!ctx_ok(c)) return KFBI_ERR_ARG;
  if (!c->have_iface) return KFBI_ERR_STATE;
  if (n_crossings) *n_crossings = c->n_cross;
  if (n_irregular) *n_irregular = c->n_irr;
  if (n_probes) *n_probes = c->n_probe;
  return KFBI_OK;
}

kfbi_status kfbi_copy_sides(kfbi_ctx* c, uint8_t* sides) {
  if (!ctx_ok(c) || sides == nullptr) return KFBI_ERR_ARG;
  if (!c->have_iface) return KFBI_ERR_STATE;
  KFBI_TRY(stream_enter(c));
  KFBI_TRY(cudaMemcpyAsync(sides, c->side, (size_t)c->N * c->N, cudaMemcpyDeviceToDevice, c->stream));
  KFBI_TRY(stream_exit(c));
  return KFBI_OK;
}

__global__ void k_pack_crossings(int cnt, const int* kind, const int* line, const int* first, const double* alpha,
                                 const double* xi, int* klf, double* ax) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  klf[3 * t] = kind[t];
  klf[3 * t + 1] = line[t];
  klf[3 * t + 2] = first[t];
  ax[2 * t] = alpha[t];
  ax[2 * t + 1] = xi[t];
}

kfbi_status kfbi_copy_crossings(kfbi_ctx* c, int cap, int* kind_line_first, double* alpha_xi) {
  if (!ctx_ok(c) || kind_line_first == nullptr || alpha_xi == nullptr || cap < 0) return KFBI_ERR_ARG;
  if (!c->have_iface) return KFBI_ERR_STATE;
  int cnt = cap < c->n_cross ? cap : c->n_cross;
  KFBI_TRY(stream_enter(c));
  if (cnt > 0) launched(c, 1);
  if (cnt > 0)
    k_pack_crossings<<<cdiv(cnt, 256), 256, 0, c->stream>>>(cnt, c->cr_kind, c->cr_line, c->cr_first, c->cr_alpha,
                                                            c->cr_xi, kind_line_first, alpha_xi);
  KFBI_TRY(cudaGetLastError());
  KFBI_TRY(stream_exit(c));
  return KFBI_OK;
}

__global__ void k_pack_irregular(int cnt, const IrrNode* irr, int* ji) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  ji[2 * t] = irr[t].j;
  ji[2 * t + 1] = irr[t].i;
}

kfbi_status kfbi_copy_irregular(kfbi_ctx* c, int cap, int* ji) {
  if (!ctx_ok(c) || ji == nullptr || cap < 0) return KFBI_ERR_ARG;
  if (!c->have_iface) return KFBI_ERR_STATE;
  int cnt = cap < c->n_irr ? cap : c->n_irr;
  KFBI_TRY(stream_enter(c));
  if (cnt > 0) launched(c, 1);
  if (cnt > 0) k_pack_irregular<<<cdiv(cnt, 256), 256, 0, c->stream>>>(cnt, c->irr, ji);
  KFBI_TRY(cudaGetLastError());
  KFBI_TRY(stream_exit(c));
  return KFBI_OK;
}

const char* kfbi_status_string(kfbi_status s) {
  switch (s) {
    case KFBI_OK: return "ok";
    case KFBI_ERR_ARG: return "invalid argument";
    case KFBI_ERR_CUDA: return g_last_error[0] ? g_last_error : "CUDA error";
    case KFBI_ERR_OUTSIDE_BOX: return "interface too close to the box";
    case KFBI_ERR_UNDERRESOLVED: return "interface under-resolved by the grid";
    case KFBI_ERR_NOT_CONVERGED: return "GMRES did not converge";
    case KFBI_ERR_SINGULAR: return "singular operator (Neumann box with kappa = 0)";
    case KFBI_ERR_TIMEOUT: return "device-side wait gave up";
    case KFBI_ERR_STATE: return "call order violated";
    case KFBI_ERR_CAPACITY: return "capacity exceeded";
  }
  return "unknown status";
}

kfbi_status kfbi_set_option(kfbi_ctx* c, int option, int value) {
  if (!ctx_ok(c)) return KFBI_ERR_ARG;
  if (option == KFBI_OPT_CLUSTER_SIZE) {
    if (value != 0 && value != 8 && value != 16) return KFBI_ERR_ARG;
    c->force_cs = value;
    c->gmf = c->gmf32 = kfbi_ctx::GmfConfig{};
    c->cfg_version += 1;
    return KFBI_OK;
  }
  if (option == KFBI_OPT_COL_PAIRS) {
    if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8 && value != 16) return KFBI_ERR_ARG;
    c->col_P = value;
    c->cfg_version += 1;
    return KFBI_OK;
  }
  if (option == KFBI_OPT_GRID_IR) {
    if (value < 0 || value > 8) return KFBI_ERR_ARG;
    c->grid_ir = value;
    return KFBI_OK;
  }
  if (option == KFBI_OPT_COL_POINTS) {
    if (value != 0 && value != 8 && value != 16) return KFBI_ERR_ARG;
    c->col_pt = value;
    c->cfg_version += 1;
    return KFBI_OK;
  }
  if (option == KFBI_OPT_COL_RADIX4) {
    if (value < 0 || value > 3) return KFBI_ERR_ARG;
    c->col_radix4 = value;
    c->cfg_version += 1;
    return KFBI_OK;
  }
  if (option == KFBI_OPT_BODY_CAP || option == KFBI_OPT_SWEEP_CAP) {
    if (value < 0) return KFBI_ERR_ARG;
    if (option == KFBI_OPT_BODY_CAP) c->body_cap_set = value;
    else c->sweep_cap_set = value;
    c->cfg_version += 1;
    return KFBI_OK;
  }
  if (value != 0 && value != 1) return KFBI_ERR_ARG;
  if (option == KFBI_OPT_BOX_MATRIX) {
    if (value == 1 && c->boxK == nullptr) return KFBI_ERR_CAPACITY;
    c->use_boxK = value != 0;
  } else if (option == KFBI_OPT_FP32_ARNOLDI) {
    c->arn32 = value != 0;
  } else if (option == KFBI_OPT_FUSE_INTERP) {
    c->fuse_interp = value != 0;
  } else if (option == KFBI_OPT_FUSE_DFT) {
    c->fuse_dft = value != 0;
  } else if (option == KFBI_OPT_FUSE_ROWS) {
    c->fuse_rows = value != 0;
  } else if (option == KFBI_OPT_COL_REG) {
    c->col_reg = value != 0;
  } else if (option == KFBI_OPT_COL_TC) {
    if (value != 0) {
      if (c->N > COL_TC_MAX_N) return KFBI_ERR_CAPACITY;
      KFBI_CHECK(col_tc_setup(c));
    }
    c->col_tc = value != 0;
  } else if (option == KFBI_OPT_PUSH_REDUCE) {
    c->gmf_push = value != 0;
    c->gmf = c->gmf32 = kfbi_ctx::GmfConfig{};
  } else if (option == KFBI_OPT_CUDA_GRAPHS) {
    c->use_graphs = value != 0;
  } else if (option == KFBI_OPT_CLUSTER_GMRES) {
    c->gm_cluster = value != 0;
    c->gmf = c->gmf32 = kfbi_ctx::GmfConfig{};
  } else if (option == KFBI_OPT_PDL) {
    c->use_pdl = value != 0;
  } else {
    return KFBI_ERR_ARG;
  }
  c->cfg_version += 1;
  return KFBI_OK;
}

kfbi_status kfbi_get_option(kfbi_ctx* c, int option, int* value) {
  if (!ctx_ok(c) || value == nullptr) return KFBI_ERR_ARG;
  if (option == KFBI_OPT_CUDA_GRAPHS) *value = c->use_graphs ? 1 : 0;
  else if (option == KFBI_OPT_CLUSTER_GMRES) *value = c->gm_cluster ? 1 : 0;
  else if (option == KFBI_OPT_LAST_CLUSTER) *value = c->gmf_last_cs;
  else if (option == KFBI_OPT_PDL) *value = c->use_pdl ? 1 : 0;
  else if (option == KFBI_OPT_CLUSTER_SIZE) *value = c->force_cs;
  else if (option == KFBI_OPT_COL_PAIRS) *value = c->col_P;
  else if (option == KFBI_OPT_BOX_MATRIX) *value = (c->boxK != nullptr && c->use_boxK) ? 1 : 0;
  else if (option == KFBI_OPT_FP32_ARNOLDI) *value = c->arn32 ? 1 : 0;
  else if (option == KFBI_OPT_PUSH_REDUCE) *value = c->gmf_push ? 1 : 0;
  else if (option == KFBI_OPT_FUSE_INTERP) *value = c->fuse_interp ? 1 : 0;
  else if (option == KFBI_OPT_FUSE_DFT) *value = c->fuse_dft ? 1 : 0;
  else if (option == KFBI_OPT_COL_REG) *value = c->col_reg ? 1 : 0;
  else if (option == KFBI_OPT_COL_TC) *value = c->col_tc ? 1 : 0;
  else if (option == KFBI_OPT_COL_RADIX4) *value = c->col_radix4;
  else if (option == KFBI_OPT_COL_POINTS) *value = c->col_pt;
  else if (option == KFBI_OPT_GRID_IR) *value = c->grid_ir;
  else if (option == KFBI_OPT_FUSE_ROWS) *value = c->fuse_rows ? 1 : 0;
  else if (option == KFBI_OPT_BODY_CAP) *value = c->body_cap_set;
  else if (option == KFBI_OPT_SWEEP_CAP) *value = c->sweep_cap_set;
  else return KFBI_ERR_ARG;
  return KFBI_OK;
}

kfbi_status kfbi_timing_enable(kfbi_ctx* c, int enable) {
  if (!ctx_ok(c)) return KFBI_ERR_ARG;
  if (enable && c->tev == nullptr) {
    c->tev = new cudaEvent_t[2 * TIMING_CAP]();
    c->tprec = new uint8_t[TIMING_CAP]();
    for (int i = 0; i < 2 * TIMING_CAP; ++i) KFBI_TRY(cudaEventCreate(&c->tev[i]));
  }
  c->timing = enable != 0;
  c->timing_used = 0;
  return KFBI_OK;
}

kfbi_status kfbi_timing_read(kfbi_ctx* c, double* ms_fp64, int* launches_fp64, double* ms_fp32, int* launches_fp32) {
  if (!ctx_ok(c)) return KFBI_ERR_ARG;
  double ms[2] = {0.0, 0.0};
  int cnt[2] = {0, 0};
  if (c->timing_used > 0) {
    KFBI_TRY(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < c->timing_used; ++i) {
      float t = 0.f;
      KFBI_TRY(cudaEventElapsedTime(&t, c->tev[2 * i], c->tev[2 * i + 1]));
      ms[c->tprec[i]] += t;
      cnt[c->tprec[i]] += 1;
    }
  }
  if (ms_fp64) *ms_fp64 = ms[0];
  if (launches_fp64) *launches_fp64 = cnt[0];
  if (ms_fp32) *ms_fp32 = ms[1];
  if (launches_fp32) *launches_fp32 = cnt[1];
  return KFBI_OK;
}

}  // extern "C"

// ALU peak probe: every thread runs eight independent fused multiply-add chains
// x <- x a + b (a = 0.999, b = 0.001: bounded values); the sum is stored only when it equals a
// value it never takes, so the compiler keeps every operation and nothing is written.
template <typename T>
static __global__ void __launch_bounds__(256) k_fma_peak(T* out, T a, T b, int iters) {
  T x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = (T)(threadIdx.x + j) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == (T)-1234.5) out[blockIdx.x] = s;
}

template <typename T>
static kfbi_status alu_peak_t(double* tflops, cudaStream_t s, int iters) {
  int dev = 0, sms = 0;
  KFBI_TRY(cudaGetDevice(&dev));
  KFBI_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  cudaEvent_t e0, e1;
  KFBI_TRY(cudaEventCreate(&e0));
  KFBI_TRY(cudaEventCreate(&e1));
  double best = 0.0;
  for (int rep = 0; rep < 4; ++rep) {  // the first launch warms up
    KFBI_TRY(cudaEventRecord(e0, s));
    k_fma_peak<T><<<blocks, threads, 0, s>>>(nullptr, (T)0.999, (T)0.001, iters);
    KFBI_TRY(cudaEventRecord(e1, s));
    KFBI_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    KFBI_TRY(cudaEventElapsedTime(&ms, e0, e1));
    const double flops = 2.0 * 32.0 * iters * (double)blocks * threads;
    if (rep > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  KFBI_TRY(cudaGetLastError());
  *tflops = best;
  return KFBI_OK;
}

extern "C" {

kfbi_status kfbi_alu_peak(int kind, double* tflops, void* stream) {
  if (tflops == nullptr || (kind != 0 && kind != 1)) return KFBI_ERR_ARG;
  if (kind == 0) return alu_peak_t<float>(tflops, (cudaStream_t)stream, 8192);
  return alu_peak_t<double>(tflops, (cudaStream_t)stream, 256);
}

kfbi_status kfbi_launch_count(kfbi_ctx* c, long long* count) {
  if (!ctx_ok(c) || count == nullptr) return KFBI_ERR_ARG;
  *count = c->launches;
  return KFBI_OK;
}

}  // extern "C"
