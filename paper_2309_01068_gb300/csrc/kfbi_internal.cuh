// Internal declarations of libkfbi: the context layout and device helpers shared by the
// translation units. Nothing here is part of the C ABI (include/kfbi.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <vector>

#include "kfbi.h"

#define KFBI_TRY(call)                                        \
  do {                                                        \
    cudaError_t kfbi_e_ = (call);                             \
    if (kfbi_e_ != cudaSuccess) {                             \
      kfbi::note_cuda_error(kfbi_e_, #call, __FILE__, __LINE__); \
      return KFBI_ERR_CUDA;                                   \
    }                                                         \
  } while (0)

#define KFBI_CHECK(st)                    \
  do {                                    \
    kfbi_status kfbi_s_ = (st);           \
    if (kfbi_s_ != KFBI_OK) return kfbi_s_; \
  } while (0)

namespace kfbi {

void note_cuda_error(cudaError_t e, const char* what, const char* file, int line);

constexpr double PI = 3.14159265358979323846;
constexpr double TWO_PI = 6.28318530717958647692;
constexpr int SUBSAMPLES = 8;        // fine samples per node interval for the crossing search
constexpr int NEWTON_MAXIT = 60;
constexpr double NEWTON_TOL = 1e-15;
// a crossing closer than SNAP_TOL h to a grid node is placed on the node, and on the arm that
// leaves the node toward the outside of the curve: a node on the curve is in the closed interior
constexpr double SNAP_TOL = 1e-10;
constexpr double BOX_MARGIN = 3.0;   // interface must stay 3h inside the box
constexpr int MAX_RESTART = 200;
constexpr int TIMING_CAP = 8192;
constexpr int TSTART_STRIDE = 34;  // per target: 32 lane start twiddles, e^{i alpha}, e^{i n alpha / 2}

// device error flags (bitmask in Iface::flags)
enum : int { FLAG_OUTSIDE = 1, FLAG_UNDERRES = 2, FLAG_CAPACITY = 4 };

// per-target geometry: crossings first, then the interface nodes
struct TargetGeo {
  double alpha;
  double xa, ya, xaa, yaa, sa, saa;
  double A3i[9];  // inverse of the 3x3 second-jump matrix (App. A.1), row-major
};

// float32 copy of the per-target geometry for the float32 kernels
struct TargetGeoF {
  float alpha;
  float xa, ya, xaa, yaa, sa, saa;
  float A3i[9];
};

// one irregular node and its (up to) four crossed arms: W, E, S, N
struct IrrNode {
  int i, j;
  int target[4];   // crossing index per arm, -1 if the arm is not crossed
  double d[4];     // neighbour minus crossing along the arm
  double sign;     // -1 for an Omega+ node, +1 for Omega- (times 1/h^2 applied later)
  float df[4];     // float32 copies of d and sign
  float signf;
  int pad;
};

// one interface node's interpolation stencil (Sec. 4.3)
struct Stencil {
  int q[6];        // flat grid index j * N + i of each point
  int probe[6];    // index into the probe-value array
  int minus[6];    // 1 if the point is in Omega-
  double dx[6], dy[6];
  double r0[6], r1[6], r2[6];  // rows 0..2 of the inverse 6x6 matrix (value, d/dx, d/dy)
  double nx, ny;   // unit outward normal at the node
  double w;        // s_alpha * 2 pi / n (trapezoidal arclength weight)
};

// float32 copy of a stencil for the float32 interpolation
struct StencilF {
  int q[6];
  int probe[6];
  int minus[6];
  float dx[6], dy[6];
  float r0[6], r1[6], r2[6];
  float nx, ny;
  float w;
};

template <typename T>
struct StencilOf;
template <>
struct StencilOf<double> {
  using type = Stencil;
};
template <>
struct StencilOf<float> {
  using type = StencilF;
};

// Inputs of the interpolation and boundary-integral epilogue of an apply (the last step of
// k_interp), so that a consumer of the apply's values can form them itself; st = nullptr:
// not in use.
template <typename T>
struct InterpArgs {
  const typename StencilOf<T>::type* st = nullptr;
  const T* pval = nullptr;    // probe values
  const T* Jall = nullptr;    // jumps of the crossings, then of the nodes
  const int* ncr = nullptr;   // crossing count (device)
  const T* x_in = nullptr;    // density (identity term)
  const double* eps_v = nullptr;
  const T* dint = nullptr;    // density integral (Hele-Shaw operator)
  T ca = 0, cb = 1, cc = 0;
};

// The value k_interp writes for node p: b_m = u(q_m) + [q_m in Omega-] C(q_m), v+ = r0.b,
// value = v+ - [u]/2, out = a x + b value + c int(x) ds, in the same operation order. Computed
// by the 8 lanes of an aligned lane group (lanes m = 0..5 of the group take the stencil
// points; every lane of the warp takes part, active = false for a group without a node); the
// result is valid in the group's lane 0. interp_pre reads what the interface fixed (the
// stencil point, the node's jump row), so that it can run before the wait for the apply;
// interp_finish reads the apply's probe values and jumps and combines.
template <typename T>
struct InterpPre {
  int probe = 0, minus = 0;
  T dx = 0, dy = 0, r0 = 0;
  const T* J = nullptr;
};
template <typename T>
__device__ __forceinline__ InterpPre<T> interp_pre(const InterpArgs<T>& a, int p, int m, bool active) {
  InterpPre<T> q;
  if (!active) return q;
  const typename StencilOf<T>::type& S = a.st[p];
  q.J = a.Jall ? a.Jall + ((long)*a.ncr + p) * 6 : nullptr;
  if (m < 6) {
    q.probe = S.probe[m];
    q.minus = S.minus[m];
    q.dx = (T)S.dx[m];
    q.dy = (T)S.dy[m];
    q.r0 = (T)S.r0[m];
  }
  return q;
}
template <typename T>
__device__ __forceinline__ T interp_finish(const InterpArgs<T>& a, const InterpPre<T>& q, int p, int m, bool active) {
  T v = 0;
  const T* J = q.J;
  if (active && m < 6) {
    const T dx = q.dx, dy = q.dy;
    T u = a.pval[q.probe];
    if (J != nullptr && q.minus) {
      u += J[0] + dx * J[1] + dy * J[2] + (T)0.5 * dx * dx * J[3] + dx * dy * J[5] + (T)0.5 * dy * dy * J[4];
    }
    v = q.r0 * u;
  }
  for (int o = 4; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o, 8);
  if (!active) return 0;
  if (J != nullptr) v -= (T)0.5 * J[0];
  T out = a.cb * v;  // the same explicit fused multiply-adds as k_interp
  if (a.x_in != nullptr) out = fma(a.eps_v != nullptr ? (T)a.eps_v[p] : a.ca, a.x_in[p], out);
  if (a.dint != nullptr) out = fma(a.cc, *a.dint, out);
  return out;
}

// GMRES control block in device memory. The scalar header comes first so that the host
// can poll it without copying the arrays.
struct GmresCtl {
  int phase;        // PH_*
  int next_phase;
  int done;         // 1 once the solve has finished (read by every kernel of a body)
  int action;       // ACT_* decided for the elementwise follow-up kernel
  int j;            // current Arnoldi column
  int k_end;        // columns used at the end of a cycle
  int its;          // Arnoldi applies
  int cycles;       // completed cycles
  int max_iter, m;
  int status;       // kfbi_status when done
  int ticket;       // last-block ticket for reductions
  int breakdown;
  int trust;        // finish on the Givens estimate without a true-residual apply
  int bodies;       // bodies executed (bounded by the loop cap)
  double tol, bnorm, beta, hnorm, res_est;
  double g[MAX_RESTART + 1];
  double cs[MAX_RESTART], sn[MAX_RESTART];
  double y[MAX_RESTART];
  double rinv[MAX_RESTART];       // 1 / R[i][i] of the rotated Hessenberg matrix (cluster form)
  double hcol[MAX_RESTART + 1];   // Gram-Schmidt coefficients of the current pass
  double H[(MAX_RESTART + 1) * MAX_RESTART];  // column-major, leading dim m+1
};
enum : int { PH_RESID = 0, PH_ARNOLDI = 1, PH_DONE = 2 };

// Control block of the device-driven iterative refinement (mixed precision): one float64
// apply and residual per sweep, then an inner float32 GMRES run on the residual.
struct IrCtl {
  int done, status, sweeps, total_its, total_cycles, inner_bodies, run_inner, outer_bodies;
  int max_iter, max_sweeps, cap_outer, pad;
  double tol, rel;
};

}  // namespace kfbi

struct kfbi_ctx {
  // grid
  int N = 0, logN = 0;
  double xmin = 0, xmax = 0, ymin = 0, ymax = 0, h = 0;
  double kappa = 0;
  int boxbc = 0, precision = 0, max_nodes = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t aux = nullptr;   // side stream for work independent of the main chain
  cudaStream_t own = nullptr;   // the context's stream when the caller uses a default stream
  cudaStream_t user = nullptr;  // the stream set by the caller
  bool user_default = true;     // caller's stream is the legacy or per-thread default stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;

  // constant tables
  double* sintab = nullptr;   // [4N] sin(pi m / (2N))
  float* sintab_f = nullptr;
  double* lam = nullptr;      // [N] 1-D eigenvalues of the box operator
  // [N][N] 1 / (lam[l] + lam[k] - kappa) (row k = x-mode): the float64 column solve's
  // divisions as products (allocated when N^2 doubles fit RINV_MAX_BYTES)
  double* rinv = nullptr;
  float* lam_f = nullptr;
  double* twN = nullptr;      // [N] complex: e^{-2 pi i m / N}, m < N
  float* twN_f = nullptr;

  // interface
  int n = 0;
  bool have_iface = false;
  int n_cross = 0, n_irr = 0, n_probe = 0;
  int cap_cross = 0, cap_irr = 0;
  double* xy = nullptr;         // [max_nodes][2]
  double* twn = nullptr;        // [max_nodes] complex e^{2 pi i m / n}
  float* twn_f = nullptr;       // the same in float32
  double* tstart = nullptr;     // [cap_cross + max_nodes][TSTART_STRIDE] complex twiddle starts
  float* tstart_f = nullptr;
  double* npack = nullptr;      // [max_nodes] double4 (x, y, y_a, -x_a) for the box quadrature
  float* npack_f = nullptr;     // float4 copy
  // free-space box: the box quadrature's kernel for the current interface, [4N][n] row-major
  // (face point, node), scale folded in, so that the box data of an apply is one product with
  // the density; allocated when 4N max_nodes 12 B fits BOXK_MAX_BYTES
  double* boxK = nullptr;
  float* boxK_f = nullptr;
  bool boxK_ok = false;         // filled for the current interface
  // the table is built on the aux stream (overlapping the work that follows set_interface);
  // ev_boxK marks its completion, boxK_pending until the main stream has waited on it
  cudaEvent_t ev_boxK = nullptr, ev_boxK0 = nullptr;
  bool boxK_pending = false;
  bool use_boxK = true;         // KFBI_OPT_BOX_MATRIX
  int* prow_list = nullptr;     // [N] rows that hold interpolation probes
  int n_prow = 0;
  double* icoef = nullptr;      // [2][max_nodes/2+1] complex Fourier coefficients of x, y
  double* fine = nullptr;       // [SUBSAMPLES*max_nodes][2]
  double* twM = nullptr;        // [SUBSAMPLES*max_nodes] complex e^{2 pi i m / M}, M = SUBSAMPLES n
  int* seg_count = nullptr;     // [2*M + 1]
  int* seg_off = nullptr;       // [2*M + 1]
  int* cr_kind = nullptr;       // [cap_cross]
  int* cr_line = nullptr;
  int* cr_seg = nullptr;
  int* cr_first = nullptr;
  double* cr_alpha = nullptr;
  double* cr_xi = nullptr;
  kfbi::TargetGeo* tgeo = nullptr;  // [cap_cross + max_nodes]
  kfbi::TargetGeoF* tgeo_f = nullptr;
  int* hcount = nullptr;        // [N][N] crossings per horizontal arm (i-1,j)-(i,j)
  int* vcount = nullptr;        // [N][N] crossings per vertical arm (i,j-1)-(i,j)
  int* hid = nullptr;           // [N][N] crossing index on the arm (if exactly one)
  int* vid = nullptr;
  uint8_t* side = nullptr;      // [N][N]
  int* rowcnt = nullptr;        // [N + 1]
  int* row_ptr = nullptr;       // [N + 1]
  kfbi::IrrNode* irr = nullptr; // [cap_irr]
  // float32 applies with the row transform folded into the column kernel: per irregular node
  // 2 i + 1 (the sine argument's column factor) and its four arm corrections
  // sign / h^2 (J0 + d J1 + d^2 J2 / 2), written by the jump kernel (zero for arms without a
  // crossing); per crossing the (4 node + arm) codes of the two arms it cuts (-1 if none) and
  // their (d, sign / h^2)
  int* irr_ci = nullptr;        // [cap_irr]
  float* arm_slot = nullptr;    // [cap_irr][4]
  int* arm_rev = nullptr;       // [cap_cross][2]
  float* arm_coef = nullptr;    // [cap_cross][2][2]
  double* corr_val = nullptr;   // [cap_irr] correction at each irregular node (mixed grid output)
  int* corr_pos = nullptr;      // [cap_irr] its grid index j N + i
  double* ir_grid = nullptr;    // [N][N] solved grid of refined float64 applies (N >= IR_APPLY_MIN_N)
  bool fuse_rows = false;       // KFBI_OPT_FUSE_ROWS
  int grid_ir = 2;              // KFBI_OPT_GRID_IR: correction sweeps of mixed grid solves
  int apply_sweeps = 0;         // sweeps of refined float64 applies inside a mixed solve (0: grid_ir)
  kfbi::Stencil* stencil = nullptr;  // [max_nodes]
  kfbi::StencilF* stencil_f = nullptr;
  float* dens_f = nullptr;      // [max_nodes] float32 copy of the apply's density
  float* stw = nullptr;         // staged FFT twiddles per radix-4 stage, float32 [N]
  double* stw_d = nullptr;      // the same in float64
  int* probe_mark = nullptr;    // [N][N] probe index + 1 (0 = not a probe)
  int* prow_cnt = nullptr;      // [N + 1]
  int* prow_ptr = nullptr;      // [N + 1]
  int* probe_i = nullptr;       // [6*max_nodes] column of each probe (row from prow_ptr)
  int* probe_j = nullptr;       // [6*max_nodes] row of each probe
  int* flags = nullptr;         // device error flags
  int* counts = nullptr;        // device counters [8]
  int* host_counts = nullptr;   // pinned [8]

  // per-apply work buffers
  double* dcoef = nullptr;      // [max_nodes/2+1] complex density coefficients
  double* dint = nullptr;       // [1] integral of the density
  double* boxg = nullptr;       // [4N] free-space box data
  double* facespec = nullptr;   // [2N] transformed south / north face rows
  double* jumps = nullptr;      // [cap_cross + max_nodes][6] jumps at the targets (T)
  double* spec = nullptr;       // [N][N] row-transformed grid (T)
  double* rowinfo = nullptr;    // [N] (w, e) of rows the row transform left to the column kernel (T pairs)
  float* col_fwd = nullptr;     // [N][N] forward DST-II / DCT-II along y (tensor-core column solve)
  float* col_inv = nullptr;     // [N][N] its exact inverse (DST-III / DCT-III with weights, 2/N)
  float* col_tmp = nullptr;     // [N][N] eigen-divided transform between the two contractions
  int* col_tc_err = nullptr;    // [1] tensor-core completion flag
  double* probe_val = nullptr;  // [6*max_nodes] (T)
  double* tmp_vals = nullptr;   // [max_nodes]

  // GMRES
  kfbi::GmresCtl* gctl = nullptr;
  kfbi::GmresCtl* host_gctl = nullptr;  // pinned
  double* gV = nullptr;         // [(MAX_RESTART+1)][max_nodes]
  double* gpart = nullptr;      // [max_nodes/32 + MAX_RESTART + 2][MAX_RESTART+1] block partials
  int gm_m = 1;                 // restart length of the running GMRES
  double* gw = nullptr;         // apply output / Arnoldi vector w  [max_nodes]
  double* gin = nullptr;        // apply input [max_nodes]
  float* gin_f = nullptr;       // float32 copy of the apply input
  double* gb = nullptr;         // right-hand side copy [max_nodes]
  double* gx = nullptr;         // iterate [max_nodes]
  double* gr = nullptr;         // outer residual / correction (refinement) [max_nodes]
  int* zero_flag = nullptr;     // device int 0

  // solve graphs: one CUDA graph per (BIE kind, apply precision) holding a conditional
  // WHILE node whose body is one GMRES iteration; rebuilt when the interface changes
  struct SolveGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long version = -1;
    int m = 0;
    int cs = 0;             // cluster size of the Gram-Schmidt kernel (0: multi-kernel form)
    bool pdl = false;       // built with programmatic dependent launch
    int cfg = -1;           // cfg_version it was built with
    int body_launches = 0;  // kernels per replayed body
    int f32 = 0;            // built with the float32 Gram-Schmidt kernel
    int cap = 0;            // body cap baked into the loop test
  } sgraph[3][2];
  // cluster form of the GMRES body (k_gm_cluster) for the last (n, m); cs = 0: multi-kernel
  struct GmfConfig {
    int n = -1, m = -1;
    int cs = 0, R = 0, hsmem = 0;
    size_t smem = 0;
    int f32 = 0;                // float32 Gram-Schmidt (k_gm_cluster<float>, basis gVf)
    int push = 0;               // push reductions (bulk copies + mbarriers) between the CTAs
  } gmf, gmf32;                 // float64 and float32 forms
  float* gVf = nullptr;         // [(MAX_RESTART+1)][max_nodes] float32 basis (mixed precision)
  bool arn32 = true;            // KFBI_OPT_FP32_ARNOLDI
  bool gmf_push = true;         // KFBI_OPT_PUSH_REDUCE
  bool fuse_interp = true;      // KFBI_OPT_FUSE_INTERP
  bool fuse_dft = true;         // KFBI_OPT_FUSE_DFT
  // device-driven refinement: control block, rhs / iterate / normal-derivative copies, and
  // one graph per (BIE kind, with normal derivative) holding the nested refinement loop
  kfbi::IrCtl* irctl = nullptr;
  kfbi::IrCtl* host_irctl = nullptr;  // pinned
  double* ir_b = nullptr;       // [max_nodes]
  double* ir_x = nullptr;       // [max_nodes]
  double* ir_dn = nullptr;      // [max_nodes]
  struct IrGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long version = -1;
    int m = 0, cs = 0, cap = 0, cfg = -1;
    bool pdl = false;
    int inner_body_launches = 0;
    int f32 = 0;
    int asw = -1;  // sweeps of the refined float64 applies captured in it
  } irgraph[3][2];
  bool gm_cluster = true;       // allow the cluster form
  bool use_pdl = true;          // programmatic dependent launch between the kernels of a body
  int force_cs = 0;             // cluster size of the Gram-Schmidt kernel: 0 automatic, 8 or 16
  int col_P = 0;                // column pairs per block of the float32 column kernel (0 automatic)
  bool col_tc = false;          // float32 column solve as two tensor-core contractions (N <= 256), KFBI_OPT_COL_TC
  bool col_reg = false;         // float32 column solve with register FFTs (N <= 1024), KFBI_OPT_COL_REG
  int col_radix4 = 2;           // KFBI_OPT_COL_RADIX4: bit 0 (float32) / bit 1 (float64) select the radix-4 kernel
  int col_pt = 0;               // KFBI_OPT_COL_POINTS: points per thread of the float32 radix-16 kernel (0 auto, 8, 16)
  int body_cap_set = 0;         // GMRES loop body cap (0: derived from max_iter), KFBI_OPT_BODY_CAP
  int sweep_cap_set = 0;        // refinement loop body cap (0: sweeps + 2), KFBI_OPT_SWEEP_CAP
  int cfg_version = 0;          // bumped by every option that changes the launched kernels
  int gmf_last_cs = 0;          // cluster size used by the last GMRES run
  size_t gmf_smem_max[2] = {0, 0};  // per element type (double, float): 0 = not queried, 1 = unavailable
  long iface_version = 0;
  // bumped when an interface changes what a captured apply launches (node count, buffer
  // capacities); graphs keyed on it survive set_interface otherwise
  long layout_version = 0;
  int ncr_grid = 0;             // crossings the captured jump launches cover (with headroom)
  bool use_graphs = true;
  bool capturing = false;
  double* gev = nullptr;        // [max_nodes] eps_V copy for the Stefan operator

  // timing of the column kernel: event pairs recorded without synchronising
  bool timing = false;
  int timing_used = 0;
  cudaEvent_t* tev = nullptr;   // [2 * TIMING_CAP]
  uint8_t* tprec = nullptr;     // [TIMING_CAP] 1 = float32 launch
  long long launches = 0;       // kernels launched by this context
  int per_apply_launches[2] = {0, 0};  // kernels of one apply (float64, float32), for graph replays
};

namespace kfbi {

// --------------------------------------------------------------------------- helpers
// Grid coordinate lo + (l + 1/2) h with separate rounding of the product and the sum
// (no fused multiply-add), so that comparisons against it are reproducible.
__device__ __forceinline__ double grid_coord(double lo, double h, int l) {
  return __dadd_rn(lo, __dmul_rn(__dadd_rn((double)l, 0.5), h));
}

// number of grid coordinates lo + (l+1/2)h (l = 0..N-1) that are <= c
__device__ __forceinline__ int count_le(double lo, double h, int N, double c) {
  double t = (c - lo) / h - 0.5;
  int l = (int)floor(t) + 1;  // candidate count
  if (l < 0) l = 0;
  if (l > N) l = N;
  while (l < N && grid_coord(lo, h, l) <= c) ++l;
  while (l > 0 && !(grid_coord(lo, h, l - 1) <= c)) --l;
  return l;
}

template <typename T>
struct Cplx {
  T re, im;
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

inline int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}
// log2 v for a power of two v >= 1, else -1
inline int ilog2_exact(int v) { return v >= 1 && (v & (v - 1)) == 0 ? ilog2(v) : -1; }

inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

inline void launched(kfbi_ctx* c, int k) { c->launches += k; }

// Programmatic dependent launch: a kernel launched with launch_k(pdl = true) may start while
// the previous kernel in its stream is finishing (its blocks are scheduled as the previous
// kernel's blocks exit; no kernel signals its successor earlier, which measured slower: the
// early blocks took SM slots from the running kernel). It first reads only data that was
// complete before that kernel started (tables, geometry, the control block), then waits with
// pdl_wait() for the previous kernel to finish and its writes to be visible. Every kernel calls
// pdl_wait() before it reads or writes anything its predecessor touches and before it
// returns, so a finished kernel implies that all kernels before it have finished. Without the
// attribute pdl_wait() is a no-op.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Work runs on c->stream. When the caller's stream is a default stream (which cannot be
// captured into a graph), c->stream is the context's own stream, ordered after the caller's
// prior work on entry and before the caller's later work on exit.
inline cudaError_t stream_enter(kfbi_ctx* c) {
  if (!c->user_default) return cudaSuccess;
  cudaError_t e = cudaEventRecord(c->ev_in, c->user);
  if (e != cudaSuccess) return e;
  return cudaStreamWaitEvent(c->own, c->ev_in, 0);
}
inline cudaError_t stream_exit(kfbi_ctx* c) {
  if (!c->user_default) return cudaSuccess;
  cudaError_t e = cudaEventRecord(c->ev_out, c->own);
  if (e != cudaSuccess) return e;
  return cudaStreamWaitEvent(c->user, c->ev_out, 0);
}
kfbi_status apply_setup_attributes(kfbi_ctx* c);

// tensor-core contraction C = alpha A B^T (kfbi_gemm.cu): A(m, k) = transA ? A[k lda + m] :
// A[m lda + k], B(n, k) likewise, float32 in and out, split-bfloat16 products (terms 3), A in
// three bfloat16 terms against a B exact in bfloat16 (terms 4), both in three terms (terms 6,
// float32 accuracy) or the plain bfloat16 product (terms 1); epilogue: store, add, or divide by
// dm[m] + dn[n] + shift
enum { TC_STORE = 0, TC_ADD = 1, TC_EIGEN = 2 };
struct TcGemmArgs {
  const float* A = nullptr;
  long lda = 0;
  int transA = 0;
  const float* B = nullptr;
  long ldb = 0;
  int transB = 0;
  float* C = nullptr;
  long ldc = 0;
  int M = 0, N = 0, K = 0;
  float alpha = 1.0f;
  int mode = TC_STORE;
  const float* dm = nullptr;
  const float* dn = nullptr;
  float shift = 0.0f;
  int terms = 3;
  int* error = nullptr;  // device flag, set to 1 when a completion wait gave up
  int bn = 0;            // column tile (32, 64, 128, 256; 0: the widest that covers N, at most 256)
};
kfbi_status tc_gemm(const TcGemmArgs& g, cudaStream_t s);
// the tensor-core column solve's matrices and buffers (kfbi_apply.cu), for N <= COL_TC_MAX_N
constexpr int COL_TC_MAX_N = 256;
kfbi_status col_tc_setup(kfbi_ctx* c);

// the column solve with register-resident radix-16 FFTs (kfbi_colfft.cu), 32 <= N <= 4096
// (float64 up to 2048: larger tables do not fit one block's shared memory):
// float32 (fp32) or float64 spectral grid `spec`, rows the row transform left out in `rowinfo`
// (or nullptr), launched on c->stream with programmatic dependent launch when pdl is set
bool col_fft_supported(int logN, bool fp32);
// the row transform's inputs, for the float32 column kernel that forms its rows itself
// (rows = nullptr in col_fft_launch: the kernel reads the row transform's output)
struct RowSrc {
  const int* row_ptr = nullptr;   // [N + 1] irregular nodes by row
  const int* ci = nullptr;        // [n_irr] 2 i + 1
  const float4* slot = nullptr;   // [n_irr] the four arm corrections
  const float* boxg = nullptr;    // [2N] w_j at j, e_j at N + j (free-space box), or nullptr
  const float* face = nullptr;    // [2N] transforms of rows 0 and N - 1, or nullptr
  int cap = 0;                    // node capacity of the shared-memory arrays (set by the launch)
  int tab = 0;                    // nodes whose sines are tabulated in shared memory (set by the launch)
};
// whether the context's layout (grid size, node capacity) fits that kernel's shared memory
bool col_fft_rows_fit(const kfbi_ctx* c);
kfbi_status col_fft_launch(kfbi_ctx* c, bool fp32, void* spec, const void* rowinfo, const int* skip, bool pdl,
                           const RowSrc* rows = nullptr);
kfbi_status col_fft_setup_attributes();

// host-side helpers implemented in the .cu files
kfbi_status ensure_cross_capacity(kfbi_ctx* c, int n_cross);
kfbi_status apply_enqueue(kfbi_ctx* c, int layer, bool fp32, const double* density, double* values,
                          double* dnormal, double* grid, int bie_kind, const double* eps_v,
                          const int* skip_flag, const float* density_f = nullptr, bool skip_interp = false);
// the interpolation inputs of a float32 apply of the density density_f (what its k_interp
// would read), for a consumer that forms the values itself (skip_interp = true)
InterpArgs<float> interp_args_f32(kfbi_ctx* c, int bie_kind, const double* eps_v, const float* density_f);
kfbi_status grid_solve_enqueue(kfbi_ctx* c, const double* rhs, double* u);
kfbi_status grid_solve_mixed_enqueue(kfbi_ctx* c, const double* rhs, double* u, int sweeps);
kfbi_status apply_grid_mixed_enqueue(kfbi_ctx* c, int layer, const double* density, double* grid, int sweeps);
// grids from this size on: the float64 applies of mixed contexts (no box data) solve their grid
// by float32 solves with float64 residual sweeps (the float64 column solve is slower there)
constexpr int IR_APPLY_MIN_N = 4096;
// a mixed solve to this tolerance or looser refines its float64 applies' grid solve with one
// correction sweep (about 5e-11 of the values at 4096^2, below 1/100 of the tolerance)
constexpr double IR_ONE_SWEEP_TOL = 1e-8;
// free-space box: fills boxK / boxK_f for the current interface (after the node data)
constexpr size_t BOXK_MAX_BYTES = (size_t)1 << 30;
constexpr size_t RINV_MAX_BYTES = (size_t)1 << 27;
// row stride of the table: node count rounded up to a multiple of 4 (16-byte rows), padded
// with zeros
__host__ __device__ inline int box_ld(int n) { return (n + 3) & ~3; }
kfbi_status box_matrix_enqueue(kfbi_ctx* c, int n);
// makes stream s wait for a box table still being built (before a graph launch or an
// interface change); no-op otherwise
kfbi_status box_table_join(kfbi_ctx* c, cudaStream_t s);
// largest dynamic shared memory of the FFT-based fine sampling (node counts up to 4096)
constexpr size_t FINE_FFT_SMEM = 3 * 16 * (size_t)4096;
kfbi_status geometry_setup_attributes();

// graph building blocks shared by the single solve and the batch (kfbi_gmres.cu)
kfbi_status cap_begin(kfbi_ctx* c, cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd);
kfbi_status cap_end(kfbi_ctx* c, std::vector<cudaGraphNode_t>* sinks);
kfbi_ctx::GmfConfig gmf_select(kfbi_ctx* c, int n, int m, bool inner = false);
int body_cap(int max_iter, int m);
int restart_length(int restart, int n);
kfbi_status add_gmres_nodes(kfbi_ctx* c, cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd, int kind, bool fp32,
                            const double* eps_v, const double* b, double* x, int cap, const kfbi_ctx::GmfConfig& gf,
                            cudaGraphNode_t* node, int* body_launches);
kfbi_status add_ir_nodes(kfbi_ctx* c, cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd, int kind, bool want_dn,
                         int m, const kfbi_ctx::GmfConfig& gf, int cap_inner, cudaGraphNode_t* node,
                         int* inner_body_launches);
// enqueue on c->stream: the start of a float64 GMRES run on (gb, gx) with gx the initial guess,
// or the start of a refinement run on (ir_b, ir_x)
kfbi_status gmres_start_enqueue(kfbi_ctx* c, double tol, int max_iter, int m);
kfbi_status ir_start_enqueue(kfbi_ctx* c, double tol, int max_iter);
constexpr int IR_MAX_SWEEPS = 12;
kfbi_status interp_grid_enqueue(kfbi_ctx* c, const double* grid, double* values);

}  // namespace kfbi
