/*
 * kfbi.h -- C ABI of libkfbi, a GB300 (sm_103a) implementation of the kernel-free
 * boundary integral (KFBI) layer-potential apply and the solvers built on it, after
 * Zhou, Li & Ying, "A Cartesian grid-based boundary integral method for moving
 * interface problems".
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Memory:     every array argument is a DEVICE pointer owned by the caller (for example
 *             a torch tensor's data_ptr()); the library never frees or retains it past
 *             the call. All device workspace is owned by the context.
 * Ordering:   work is enqueued on the context's stream (kfbi_set_stream; default the
 *             legacy default stream). kfbi_apply_layer_potential, kfbi_bie_apply,
 *             kfbi_grid_solve and kfbi_interp_grid are asynchronous. kfbi_set_interface,
 *             kfbi_solve_bie and kfbi_step synchronise the stream to read counts and
 *             status flags back.
 * Grid:       cell-centred N x N cells on a square-celled box [xmin,xmax] x [ymin,ymax];
 *             cell (i, j) has centre (xmin + (i + 1/2) h, ymin + (j + 1/2) h) and grid
 *             arrays are row-major [j][i] (y index outer), float64.
 * Interface:  n nodes X_j = X(alpha_j), alpha_j = 2 pi j / n, counter-clockwise, as
 *             [n][2] float64 (x, y interleaved). Omega+ is the bounded interior.
 *             Interface functions (densities) are [n] float64 nodal values; their
 *             derivatives come from the global trigonometric interpolant.
 * Errors:     every call returns a kfbi_status; nothing else crosses the ABI. After an
 *             error other than KFBI_ERR_NOT_CONVERGED or (from kfbi_solve_bie)
 *             KFBI_ERR_TIMEOUT the outputs are unspecified.
 * Precision:  KFBI_FP64 runs every step in float64. KFBI_MIXED runs the grid part of the
 *             inner applies (jumps, corrections, transforms, interpolation) in float32
 *             and keeps float64 for GMRES (Arnoldi, Givens, least squares), the outer
 *             residual and the iterative-refinement update.
 */
#ifndef KFBI_H
#define KFBI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KFBI_OK = 0,
  KFBI_ERR_ARG = 1,           /* invalid argument (null pointer, bad size or mode) */
  KFBI_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  KFBI_ERR_OUTSIDE_BOX = 3,   /* interface closer than 3h to the box, or stencil off-grid */
  KFBI_ERR_UNDERRESOLVED = 4, /* three crossings on one grid arm, or arms inconsistent */
  KFBI_ERR_NOT_CONVERGED = 5, /* GMRES reached max_iter; the best iterate is returned */
  KFBI_ERR_SINGULAR = 6,      /* Neumann box with kappa = 0 (constant null space) */
  KFBI_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up */
  KFBI_ERR_STATE = 8,         /* call order violated (e.g. apply before set_interface) */
  KFBI_ERR_CAPACITY = 9       /* more nodes or crossings than the context was created for */
} kfbi_status;

/* Box boundary condition of the grid problem (Sec. 4.1). */
enum {
  KFBI_BOX_DIRICHLET0 = 0,   /* u = 0 on the box: DST-II solve (interior problems) */
  KFBI_BOX_NEUMANN0 = 1,     /* du/dn = 0 on the box: DCT-II solve (Stefan, Sec. 3.2) */
  KFBI_BOX_FREESPACE_DL = 2  /* Dirichlet data = free-space double layer by the trapezoidal
                                rule on the box faces (Hele-Shaw, Sec. 4.1); kappa = 0 only */
};
enum { KFBI_FP64 = 0, KFBI_MIXED = 1 };
/* Layer potentials and their jumps (Table 2). */
enum { KFBI_SINGLE = 0, KFBI_DOUBLE = 1 };
/* Boundary integral equations (Sec. 3). */
enum {
  KFBI_BIE_INTERIOR_DL = 0,     /* (1/2) phi + D phi = g, interior Dirichlet problem */
  KFBI_BIE_HS_EXTERIOR_MDL = 1, /* -(1/2) phi + D phi + int phi ds = g (Sec. 3.1) */
  KFBI_BIE_STEFAN_SL = 2        /* eps_V psi - S psi = g (Sec. 3.2) */
};

typedef struct kfbi_ctx kfbi_ctx;

typedef struct {
  int iterations;      /* GMRES operator applies (all refinement sweeps) */
  int restarts;        /* GMRES restarts */
  int refinements;     /* float64 residual evaluations of iterative refinement (MIXED) */
  int status;          /* kfbi_status of the solve */
  double rel_residual; /* ||b - A x||_2 / ||b||_2 of the returned density, float64 operator */
} kfbi_solve_info;

/*
 * kfbi_create -- a context for one grid, box and operator (Delta - kappa) (Sec. 4.2).
 *   N          cells per side, a power of two in [16, 4096]
 *   xmin..ymax box; (xmax - xmin) / N must equal (ymax - ymin) / N (square cells)
 *   kappa      c^2 >= 0 of the modified Helmholtz operator Delta - c^2 (Sec. 3.2;
 *              kappa = 0 is the Laplacian). Not a curvature.
 *   boxbc      KFBI_BOX_*; NEUMANN0 needs kappa > 0, FREESPACE_DL needs kappa = 0
 *   precision  KFBI_FP64 or KFBI_MIXED
 *   max_nodes  largest interface node count this context will see (>= 8)
 *   out        receives the context; release it with kfbi_destroy
 * Errors: ARG, SINGULAR, CUDA (allocation).
 */
kfbi_status kfbi_create(int N, double xmin, double xmax, double ymin, double ymax, double kappa,
                        int boxbc, int precision, int max_nodes, kfbi_ctx** out);

/* Releases the context and all device workspace it owns. NULL is ignored. */
void kfbi_destroy(kfbi_ctx* ctx);

/* Sets the cudaStream_t (passed as void*) that later calls enqueue on. */
kfbi_status kfbi_set_stream(kfbi_ctx* ctx, void* stream);

/*
 * kfbi_set_interface -- geometry of the interface (Sec. 4.2 irregular nodes, Sec. 4.3
 * interpolation stencils).
 *   n   node count, 8 <= n <= max_nodes
 *   xy  device [n][2] float64 node coordinates (read only)
 * Finds every crossing of the curve with the grid lines (Newton on the trigonometric
 * interpolant), classifies grid nodes into Omega+/Omega-, lists irregular nodes and
 * their crossed arms, and builds the 6-point interpolation stencils.
 * Synchronises the stream. Errors: ARG, OUTSIDE_BOX, UNDERRESOLVED, CAPACITY, CUDA.
 */
kfbi_status kfbi_set_interface(kfbi_ctx* ctx, int n, const double* xy);

/*
 * kfbi_apply_layer_potential -- the KFBI apply (Sec. 4): solves the equivalent interface
 * problem (Delta - kappa) v = 0 with [v] = Phi, [dv/dn] = Psi from Table 2 by the corrected
 * five-point scheme and a fast DST/DCT solve, then extracts the boundary operator
 * (average of the one-sided limits, Sec. 4.3).
 *   layer    KFBI_SINGLE (S psi: Phi = 0, Psi = -psi) or KFBI_DOUBLE (D phi: Phi = phi)
 *   density  device [n] float64
 *   values   device [n] float64 output: (S psi) or (D phi) on the curve
 *   dnormal  device [n] float64 output or NULL: n . (grad v+ + grad v-)/2
 *   grid     device [N][N] float64 output or NULL: the grid solution v_h
 * Asynchronous. FREESPACE_DL contexts accept KFBI_DOUBLE only.
 * Errors: ARG, STATE, CUDA.
 */
kfbi_status kfbi_apply_layer_potential(kfbi_ctx* ctx, int layer, const double* density, double* values,
                                       double* dnormal, double* grid);

/*
 * kfbi_bie_apply -- y = A x for the boundary integral operator of `kind` (Sec. 3):
 *   INTERIOR_DL:       y = x/2 + D x
 *   HS_EXTERIOR_MDL:   y = -x/2 + D x + int x ds           (Sec. 3.1)
 *   STEFAN_SL:         y = eps_v .* x - S x                 (Sec. 3.2)
 *   eps_v  device [n] float64, STEFAN_SL only (else ignored, may be NULL)
 *   x, y   device [n] float64
 * Uses the context's precision for the grid part. Asynchronous. Errors: ARG, STATE, CUDA.
 */
kfbi_status kfbi_bie_apply(kfbi_ctx* ctx, int kind, const double* eps_v, const double* x, double* y);

/*
 * kfbi_solve_bie -- matrix-free restarted GMRES for A x = rhs (Sec. 4), one operator
 * apply per iteration, Arnoldi (two-pass classical Gram-Schmidt), Givens rotations and
 * the least-squares update all on the device. MIXED contexts run float32 grid applies
 * inside GMRES and iterative refinement with a float64 residual until
 * ||rhs - A x|| <= tol ||rhs||.
 *   kind      KFBI_BIE_*;  eps_v as in kfbi_bie_apply
 *   rhs       device [n] float64
 *   tol       relative residual target (> 0)
 *   max_iter  cap on GMRES applies (>= 1);  restart  Krylov dimension (1..200)
 *   density   device [n] float64: initial guess in, solution out
 *   info      host pointer, filled on return (may be NULL)
 * Synchronises the stream. Errors: ARG, STATE, NOT_CONVERGED (best iterate returned),
 * TIMEOUT (a device-side loop bound was reached, KFBI_OPT_BODY_CAP / KFBI_OPT_SWEEP_CAP;
 * the iterate described there is returned and `info` is filled), CUDA.
 */
kfbi_status kfbi_solve_bie(kfbi_ctx* ctx, int kind, const double* eps_v, const double* rhs, double tol,
                           int max_iter, int restart, double* density, kfbi_solve_info* info);

/*
 * kfbi_grid_solve -- (Delta_h - kappa) u = rhs on the whole grid with the context's box
 * condition, no interface corrections (the smooth part T1 of Sec. 3.2).
 *   rhs, u  device [N][N] float64 (may alias). Asynchronous. Errors: ARG, CUDA.
 */
kfbi_status kfbi_grid_solve(kfbi_ctx* ctx, const double* rhs, double* u);

/*
 * kfbi_grid_solve_mixed -- the same box solve as kfbi_grid_solve for KFBI_MIXED contexts,
 * by mixed-precision iterative refinement (not in the paper; Sec. 4.2's solve is its inner
 * step): u = the float32 solve of rhs (row transforms, column solve and eigenvalue division on
 * the float32 spectral grid with the float32 tables), then `sweeps` corrections
 *   r = rhs - (Delta_h - kappa) u   (float64, five-point Laplacian with the box condition's
 *                                    ghost values: u_{-1} = -u_0 for DST-II, u_0 for DCT-II),
 *   u += the float32 solve of r     (r rounded to float32).
 * Each sweep reduces the error of u by about the float32 solve's relative accuracy; two
 * sweeps reach the float64 solve's accuracy on the Stefan workloads (tests).
 *   rhs, u  device [N][N] float64, must not alias; sweeps 0..8. Asynchronous; uses the
 *           context's spectral buffer. Errors: ARG (NULL, aliasing, sweeps out of range,
 *           a KFBI_FP64 context), CUDA.
 */
kfbi_status kfbi_grid_solve_mixed(kfbi_ctx* ctx, const double* rhs, double* u, int sweeps);

/*
 * kfbi_interp_grid -- values at the interface nodes of a smooth grid function by the
 * 6-point interpolation of Sec. 4.3 with zero jumps.
 *   grid    device [N][N] float64;  values  device [n] float64
 * Asynchronous. Errors: ARG, STATE, CUDA.
 */
kfbi_status kfbi_interp_grid(kfbi_ctx* ctx, const double* grid, double* values);

/*
 * Introspection of the last kfbi_set_interface, for tests:
 *   kfbi_interface_stats  host ints: crossings, irregular nodes, interpolation probes
 *   kfbi_copy_sides       device [N][N] uint8: 1 = Omega+, 0 = Omega-
 *   kfbi_copy_crossings   device outputs for the first `cap` crossings in the order
 *                         (horizontal lines first, then vertical; by sub-segment, then
 *                         line): ints [cap][3] = (kind, line, first), doubles [cap][2] =
 *                         (alpha, coordinate along the line)
 *   kfbi_copy_irregular   device ints [cap][2] = (j, i), row-major order
 */
kfbi_status kfbi_interface_stats(kfbi_ctx* ctx, int* n_crossings, int* n_irregular, int* n_probes);
kfbi_status kfbi_copy_sides(kfbi_ctx* ctx, uint8_t* sides);
kfbi_status kfbi_copy_crossings(kfbi_ctx* ctx, int cap, int* kind_line_first, double* alpha_xi);
kfbi_status kfbi_copy_irregular(kfbi_ctx* ctx, int cap, int* ji);

/*
 * theta-L interface evolution (Sec. 5): one semi-implicit time step.
 * The state lives in device memory allocated by kfbi_thetal_create:
 *   eta[n]     theta - alpha at the nodes (Sec. 5.3 remark)
 *   scalars    L, Xbar (2), t, and the Adams-Bashforth history M, Q (2), L, N-hat (2n)
 *   density[n] last BIE density (warm start of the next solve)
 *   xy[n][2]   nodes of the curve the last step solved on
 *   T, T_prev  [N][N] grid temperatures (Stefan only)
 */
enum { KFBI_STEP_HELE_SHAW = 0, KFBI_STEP_STEFAN = 1 };

typedef struct kfbi_thetal kfbi_thetal;

typedef struct {
  int kind;          /* KFBI_STEP_* */
  /* Hele-Shaw (Sec. 2.1, 3.1): surface tension sigma, injection rate J */
  double sigma, J;
  /* Stefan (Sec. 2.2, 3.2): undercooling St, eps_C = eps_c (1 - eps_aniso cos(fold
     (theta - pi/2))), constant eps_V >= 0. eps_V > 0: second-kind equation, small-scale
     decomposition case I (stiff part lambda_1 (2 pi/L)^2 theta_aa, lambda_1 = max |eps_C/eps_V|);
     eps_V = 0: first-kind equation -S psi = -eps_C kappa - T1, case II (stiff part
     lambda_2 (2 pi/L)^3 H[theta_aaa], lambda_2 = max |2 eps_C|), Sec. 5.2.2 and 5.3 */
  double St, eps_c, eps_aniso, eps_v;
  int fold;
  /* GMRES controls of the per-step BIE solve */
  double tol;
  int max_iter, restart;
  /* KFBI_SCHEME_SEMI_IMPLICIT (0): the stiff part by its propagator, the rest by
     Adams-Bashforth (Sec. 5.3); KFBI_SCHEME_EXPLICIT (1): Adams-Bashforth on the whole
     right-hand side, no stiff part split off (the comparison scheme of Sec. 6.2.2) */
  int scheme;
  /* marker doubling (Sec. 6.1.4): before a step, while L / n > refine_ratio h, the node count
     doubles (eta, the density and the Adams-Bashforth history carried over as the same
     trigonometric interpolants); 0 = off. The state's arrays are then sized for the context's
     max_nodes, the ceiling of the doubling. */
  double refine_ratio;
  /* Hele-Shaw only, 1 = the step works in the rescaled frame of the long-time computation
     (Sec. 6.1.4; the rescaling is cited there, not printed, and read as follows): x = R xb with
     R = e^{tb}, dt / dtb = (A0 / pi) R^2, A0 the area at the first step; the scaled problem has
     surface tension sigma / R and normal velocity (A0 / pi) U - xb.n, which keeps the scaled
     area at A0 for J = 1. The state's t is then the scaled time tb; physical time
     t = (A0 / pi)(e^{2 tb} - 1) / 2 and the physical curve R X (A0 in scalars slot 16). */
  int rescale;
} kfbi_thetal_params;
enum { KFBI_SCHEME_SEMI_IMPLICIT = 0, KFBI_SCHEME_EXPLICIT = 1 };

/*
 * kfbi_thetal_create -- device state for the context's grid from equal-arclength nodes.
 *   n         node count;  eta  device [n] float64 (theta - alpha_j);  L  curve length
 *   xbar      host [2] mean node position
 * Errors: ARG, CUDA.
 */
kfbi_status kfbi_thetal_create(kfbi_ctx* ctx, int n, const double* eta, double L, const double* xbar,
                               const kfbi_thetal_params* params, kfbi_thetal** out);
void kfbi_thetal_destroy(kfbi_thetal* st);

/*
 * kfbi_step -- one time step of size dt (Sec. 5.3): reconstruct the curve from
 * (eta, L, Xbar), set the interface, solve the BIE (Hele-Shaw: Sec. 3.1; Stefan: Sec. 3.2
 * with T1 from kfbi_grid_solve), form the normal velocity U and advance (eta, L, Xbar)
 * with the integrating-factor / Adams-Bashforth scheme. Synchronises the stream.
 *   info  host pointer or NULL: the step's BIE solve
 * Errors: those of kfbi_set_interface and kfbi_solve_bie.
 */
kfbi_status kfbi_step(kfbi_ctx* ctx, kfbi_thetal* st, double dt, kfbi_solve_info* info);

/*
 * Checkpoint and resume of the theta-L state. Device buffers, NULL skips an item:
 *   eta [n], xy [n][2] nodes of the last solved curve (read only), density [n],
 *   nhat [(n/2+1)][2] the Adams-Bashforth history of N-hat (complex), T and T_prev
 *   [N][N] (Stefan only). `scalars` is a HOST array of KFBI_THETAL_SCALARS doubles:
 *   (L, Xbar_x, Xbar_y, t, steps, M_prev, Q_prev_x, Q_prev_y, L_prev, then work slots; slots
 *   14 and 15 are the learned warm start's counters, see kfbi_thetal_set_warmstart; slot 16 is
 *   the rescaled frame's A0).
 * Writing back what was read restores the state exactly. kfbi_thetal_read synchronises
 * the stream when `scalars` is given. Errors: ARG, CUDA.
 */
#define KFBI_THETAL_SCALARS 20
kfbi_status kfbi_thetal_read(kfbi_thetal* st, double* eta, double* xy, double* density, double* nhat, double* T,
                             double* T_prev, double* scalars);
kfbi_status kfbi_thetal_write(kfbi_thetal* st, const double* eta, const double* density, const double* nhat,
                              const double* T, const double* T_prev, const double* scalars);

/* Human-readable name of a status code (static storage). */
const char* kfbi_status_string(kfbi_status s);

/*
 * kfbi_grid_solve_noalloc -- the same box solve as kfbi_grid_solve, (Delta_h - kappa) u = rhs
 * with a Dirichlet-0 (DST-II) or Neumann-0 (DCT-II) box, for callers that cannot allocate
 * device memory: an application that hands all device memory to its own pool at start-up,
 * or a loop with a fixed latency budget that must not call cudaMalloc (which can
 * synchronise the device and take unbounded time). No context is needed; this entry point
 * makes no allocation of any kind (no cudaMalloc, cudaFree or allocating library routine).
 * The paper has no counterpart: it is an interface convenience of this library.
 *   N      cells per side, a power of two in [16, 512] (larger N: KFBI_ERR_CAPACITY)
 *   h      cell width (> 0);  kappa  c^2 >= 0;  boxbc  KFBI_BOX_* (FREESPACE_DL solves as
 *          DIRICHLET0: the plain solve has no interface data)
 *   rhs, u device [N][N] float64 (may alias);  stream  cudaStream_t as void*
 * Scratch: one static device array of about 2.1 MB in libkfbi, which every GPU that loads
 * the library holds until the process exits. The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture. The address is kept for the life of the process: a
 * device reset (cudaDeviceReset) between calls is not supported. All calls share the array
 * and each call rewrites it
 * completely, so calls that overlap on the GPU (different streams or host threads) race:
 * serialise them. Asynchronous. Errors: ARG, CAPACITY, SINGULAR, CUDA.
 */
kfbi_status kfbi_grid_solve_noalloc(int N, double h, double kappa, int boxbc, const double* rhs, double* u,
                                    void* stream);

/*
 * Per-kernel device timing for roofline reports. When enabled, the library records a pair
 * of CUDA events on the context's stream around every launch of the column kernel of the
 * fast solve (the dominant grid kernel), without synchronising. kfbi_timing_read
 * synchronises the stream and returns the summed milliseconds and launch counts since
 * enable, separately for the float64 and float32 instantiations (host outputs; NULL skips).
 * At most 8192 launches are recorded per enable.
 */
kfbi_status kfbi_timing_enable(kfbi_ctx* ctx, int enable);
kfbi_status kfbi_timing_read(kfbi_ctx* ctx, double* ms_fp64, int* launches_fp64, double* ms_fp32,
                             int* launches_fp32);

/*
 * Execution options of a context (none changes a result beyond rounding order):
 *   KFBI_OPT_CUDA_GRAPHS      1 (default): a GMRES run is one CUDA graph launch whose
 *                             conditional WHILE node replays one iteration until the device
 *                             decides the run is over; 0: the host enqueues iterations in
 *                             chunks and polls the device between chunks.
 *   KFBI_OPT_CLUSTER_GMRES    1 (default): the Gram-Schmidt step of an iteration is one
 *                             launch of a thread-block cluster (16 or 8 CTAs, selected by
 *                             node count, restart length and shared-memory capacity) when the
 *                             device can schedule it; 0: the five-kernel form.
 *   KFBI_OPT_LAST_CLUSTER     read only: cluster size used by the last GMRES run (0 = the
 *                             five-kernel form).
 *   KFBI_OPT_CLUSTER_SIZE     0 (default): the cluster form takes 16 CTAs, else 8; 8 or 16:
 *                             only that size (the five-kernel form when it does not fit).
 *   KFBI_OPT_COL_PAIRS        0 (default): column pairs per block of the column transform;
 *                             values 0, 1, 2, 4, 8, 16. Radix-4 kernel: 2 by default (float64: 1),
 *                             else the value bounded by 4 and by its shared memory. Radix-16
 *                             kernel: instantiated for PMIN = max(1, 512 / N) (one warp per block
 *                             at least), 2 PMIN and, while a block stays within 256 threads,
 *                             4 PMIN; it runs the largest of these not above the value (PMIN if
 *                             none), the largest of all by default.
 *   KFBI_OPT_PDL              1 (default): consecutive kernels of an apply and of a GMRES
 *                             iteration use programmatic dependent launch (a kernel is
 *                             scheduled as its predecessor's blocks exit, reads its static
 *                             inputs, and waits on the device before it reads the
 *                             predecessor's output); 0: plain stream order. Batch graphs are
 *                             always built without it.
 *   KFBI_OPT_BOX_MATRIX       1 (default): with KFBI_BOX_FREESPACE_DL, kfbi_set_interface
 *                             tabulates the box quadrature's kernel between the interface
 *                             nodes and the 4 N face points (4 N max_nodes values in float64
 *                             and float32, allocated by kfbi_create when they take at most
 *                             1 GiB), and every apply forms the box data as one product of
 *                             that table with the density; 0: every apply evaluates the
 *                             quadrature directly. Setting 1 on a context without the table
 *                             returns CAPACITY; reading gives 1 only when the table is in use.
 *   KFBI_OPT_FP32_ARNOLDI     1 (default): in KFBI_MIXED, the inner GMRES of the refinement
 *                             (whose operator is the float32 apply) stores its basis and does
 *                             its Gram-Schmidt passes, rotations and update in float32 when
 *                             the cluster form runs; 0: in float64. The float64 refinement
 *                             decides convergence either way.
 *   KFBI_OPT_PUSH_REDUCE      1 (default): the cluster form combines its CTAs' partial sums by
 *                             pushing them (bulk shared-memory copies to every CTA of the
 *                             cluster, completed on each receiver's mbarrier) when the
 *                             receive rows fit in shared memory; 0: a cluster barrier, then
 *                             every CTA loads the partial sums from the others.
 *   KFBI_OPT_FUSE_INTERP      1 (default): with the float32 Gram-Schmidt kernel, each CTA
 *                             forms its slice of A v from the apply's probe values and jumps
 *                             (the apply's interpolation step, same arithmetic) instead of a
 *                             separate interpolation kernel; 0: the separate kernel.
 *   KFBI_OPT_FUSE_DFT         1 (default): float32 applies with a power-of-two node count
 *                             (16..4096) form the density's Fourier coefficients inside the
 *                             jump kernel (a shared-memory FFT in every block) instead of a
 *                             separate DFT kernel; 0: the separate kernel.
 *   KFBI_OPT_COL_RADIX4       2 (default): float32 applies (grids with N >= 32) run the
 *                             register-resident column kernel (radix-16 stages with 16 points per
 *                             thread, radix-8 with 8: KFBI_OPT_COL_POINTS), float64 applies the
 *                             shared-memory radix-4 Stockham kernel. In the register kernel each
 *                             column pair is owned by N/16 threads holding 16 points through the
 *                             forward FFT, the eigenvalue division and the inverse (Stockham
 *                             stages of radix 16, the last of radix 2, 4 or 8, through one
 *                             shared-memory buffer). Bit 0 set (1, 3): float32 applies run the
 *                             radix-4 kernel; bit 1 clear (0, 1): float64 applies run the
 *                             radix-16 kernel. Values 0..3.
 *   KFBI_OPT_COL_POINTS       0 (default), 8 or 16: points per thread of the float32
 *                             register-resident column kernel. 8: N/8 threads per column pair
 *                             (twice the warps), Stockham stages of radix 8 (the last of radix
 *                             2 or 4; N = 1024 is 8, 8, 8, 2), available for N <= 1024 (16 is
 *                             used above). 0: 8 for N <= 1024, 16 above (the faster form at each
 *                             size).
 *   KFBI_OPT_FUSE_ROWS        0 (default): the row transform is its own kernel. 1: float32
 *                             applies whose jumps come from the fused jump kernel
 *                             (KFBI_OPT_FUSE_DFT) and whose column solve is the radix-16 kernel
 *                             form the row transform inside the column kernel: the jump kernel
 *                             writes each crossed arm's correction, and the column kernel sums,
 *                             for each of its rows, the corrections of the row's irregular nodes
 *                             times the DST/DCT basis functions of its columns (tabulated in
 *                             shared memory before the wait for the jump kernel), plus the box
 *                             data; the row-transform kernel is not launched. Applies when the
 *                             node capacity fits the column kernel's shared memory. Measured
 *                             slower on the Hele-Shaw 1024^2 workload (37.2 against 32.7 us per
 *                             float32 apply), hence off by default.
 *   KFBI_OPT_COL_REG          0 (default); 1 (grids with N <= 1024): the float32 column solve
 *                             holds every FFT in registers by one group of B lanes (an A-point
 *                             DFT per lane, one transpose through shared memory, B-point DFTs;
 *                             N = A B). Takes precedence over KFBI_OPT_COL_RADIX4.
 *   KFBI_OPT_COL_TC           0 (default); 1 (grids with N <= 256, else KFBI_ERR_CAPACITY):
 *                             the float32 column solve as two dense contractions on the tensor
 *                             cores (kfbi_tc_gemm, split bfloat16 products): the transform along
 *                             y as an N x N matrix, the eigenvalue division in the first one's
 *                             epilogue, then the inverse transform matrix. The row transform then
 *                             writes every row. Setting it allocates the two N x N matrices.
 *                             Takes precedence over KFBI_OPT_COL_REG and KFBI_OPT_COL_RADIX4.
 *   KFBI_OPT_GRID_IR          2 (default), 0..8: in KFBI_MIXED contexts the Stefan step's two
 *                             dense grid solves run by mixed-precision refinement with this many
 *                             float64 correction sweeps: T1 as kfbi_grid_solve_mixed, and the
 *                             single layer's grid values (T2) as the same solve with the
 *                             corrected right-hand side of the float64 jumps at the irregular
 *                             nodes (the apply's column solve and interface values are not
 *                             formed). On grids with N >= 4096 and no box data, the float64
 *                             applies of the refinement (KFBI_MIXED solves) solve their grid the
 *                             same way and gather the probe values from it, with one sweep when
 *                             the solve's tolerance is 1e-8 or looser (their error, about 5e-11 of
 *                             the values, is then far below it; a test checks the returned
 *                             density's residual under the float64 context's operator). 0:
 *                             float64 solves (kfbi_grid_solve and the float64 apply's column
 *                             solve).
 *   KFBI_OPT_BODY_CAP         0 (default): the device-side GMRES loop (the body count of the
 *                             graph's WHILE node, or of the host-driven loop) stops after
 *                             2 max_iter + 2 max_iter / restart + 8 bodies; a value > 0 sets
 *                             that bound instead. A solve that reaches it returns
 *                             KFBI_ERR_TIMEOUT with the iterate of its last completed restart
 *                             cycle in `density` (the initial guess if none completed); the
 *                             context stays usable.
 *   KFBI_OPT_SWEEP_CAP        0 (default): the refinement loop of KFBI_MIXED stops after 14
 *                             sweeps (two more than the 12 it may take); a value > 0 sets that
 *                             bound instead. A solve that reaches it returns KFBI_ERR_TIMEOUT
 *                             with the refined iterate of its last sweep in `density`.
 * kfbi_set_option: value 0 or 1 unless stated. kfbi_get_option writes the value to *value (host).
 * Errors: ARG (unknown option, bad value, NULL, read-only option).
 */
enum {
  KFBI_OPT_CUDA_GRAPHS = 1,
  KFBI_OPT_CLUSTER_GMRES = 2,
  KFBI_OPT_LAST_CLUSTER = 3,
  KFBI_OPT_PDL = 4,
  KFBI_OPT_CLUSTER_SIZE = 5,
  KFBI_OPT_COL_PAIRS = 6,
  KFBI_OPT_BOX_MATRIX = 7,
  KFBI_OPT_FP32_ARNOLDI = 8,
  KFBI_OPT_PUSH_REDUCE = 9,
  KFBI_OPT_FUSE_INTERP = 10,
  KFBI_OPT_FUSE_DFT = 11,
  KFBI_OPT_BODY_CAP = 12,
  KFBI_OPT_SWEEP_CAP = 13,
  KFBI_OPT_COL_REG = 14,
  KFBI_OPT_COL_TC = 15,
  KFBI_OPT_COL_RADIX4 = 16,
  KFBI_OPT_FUSE_ROWS = 17,
  KFBI_OPT_COL_POINTS = 18,
  KFBI_OPT_GRID_IR = 19
};
kfbi_status kfbi_set_option(kfbi_ctx* ctx, int option, int value);
kfbi_status kfbi_get_option(kfbi_ctx* ctx, int option, int* value);

/* ------------------------------------------------------------------------------------
 * Learned warm start of GMRES. The paper has no learned component: it solves each
 * boundary integral equation by GMRES from a given initial density (Sec. 4). Here a small
 * network predicts that initial density from per-node interface features; GMRES still
 * iterates to the caller's tolerance, so the solution does not depend on the prediction.
 *
 * Features of node j (KFBI_MLP_FEATURES = 47, float32), l = L / (2 pi), L the curve length:
 *   0..31  Re, Im of khat_k e^{i k alpha_j} l, k = 0..15, khat_k = (1/n) sum_m kappa_m e^{-i k alpha_m}
 *   32     kappa_j l                33, 34  outward unit normal
 *   35     s_j / L (trapezoidal arclength from node 0)
 *   36     g_j / rms(g)             37, 38  (x_j - mean x) / l, (y_j - mean y) / l
 *   39..46 Re, Im of ghat_k e^{i k alpha_j} / rms(g), k = 0..3 (low modes of the data g)
 * Network: 47 -> H -> H -> 1, ReLU, weights rounded to bfloat16 (nearest even), float32
 * biases, activations and accumulation; its output y_j predicts phi_j / rms(g).
 * Parameters (float32, host arrays of kfbi_mlp_param_count entries), in this order:
 *   W1 [H][47], b1 [H], W2 [H][H], b2 [H], w3 [H], b3.
 * Training: mean squared error over the rows, gradients through the rounded weights applied
 * to the float32 weights, Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).
 * ------------------------------------------------------------------------------------ */
enum { KFBI_MLP_FEATURES = 47, KFBI_MLP_MODES = 16, KFBI_MLP_DATA_MODES = 4 };
typedef struct kfbi_mlp kfbi_mlp;

/* hidden: multiple of 32 in [32, 256]; max_rows: largest batch (and node count) served.
 * Parameters start at zero: load them with kfbi_mlp_set_params. Errors: ARG, CUDA. */
kfbi_status kfbi_mlp_create(int hidden, int max_rows, kfbi_mlp** out);
void kfbi_mlp_destroy(kfbi_mlp* mlp);
/* Stream of the kfbi_mlp_* calls (default: the legacy default stream). */
kfbi_status kfbi_mlp_set_stream(kfbi_mlp* mlp, void* stream);
kfbi_status kfbi_mlp_param_count(kfbi_mlp* mlp, int* count);
/* The H x H layer (forward, input gradient and weight gradient) on the tensor cores through
 * kfbi_tc_gemm (enable = 1, the default) or on the CUDA cores (0, one fused kernel per 16 rows).
 * kfbi_mlp_tc_error reads the tensor-core completion flag (0: every wait completed); both
 * synchronise the network's stream. */
kfbi_status kfbi_mlp_set_tensor_cores(kfbi_mlp* mlp, int enable);
kfbi_status kfbi_mlp_tc_error(kfbi_mlp* mlp, int* flag);
/* Host float32 parameters in and out; set_params also resets Adam's moments and step
 * count. Both synchronise the stream. */
kfbi_status kfbi_mlp_set_params(kfbi_mlp* mlp, const float* params);
kfbi_status kfbi_mlp_get_params(kfbi_mlp* mlp, float* params);
/* y[r] for rows r < rows of feat (device [rows][47] float32); y device [rows]. Async. */
kfbi_status kfbi_mlp_forward(kfbi_mlp* mlp, const float* feat, int rows, float* y);
/* Gradient of the mean squared error of rows idx[0..rows) (device int32; NULL: rows
 * 0..rows-1) of feat against target (device float32): grad device [param_count] (NULL keeps
 * it internal); loss: host float (NULL: not read, no synchronisation). */
kfbi_status kfbi_mlp_gradients(kfbi_mlp* mlp, const float* feat, const float* target, const int* idx, int rows,
                               float* grad, float* loss);
/* One Adam step on the rows idx[0..rows) with learning rate lr (> 0); loss as above. */
kfbi_status kfbi_mlp_train_step(kfbi_mlp* mlp, const float* feat, const float* target, const int* idx, int rows,
                                float lr, float* loss);
/* Features of the context's interface nodes for the right-hand side rhs (device [n]
 * float64): feat device [n][47] float32, scale device [1] float64 = rms(rhs). n <= 8192
 * (else CAPACITY). Errors: ARG, STATE (no interface), CAPACITY, CUDA. Async. */
kfbi_status kfbi_warmstart_features(kfbi_ctx* ctx, const double* rhs, float* feat, double* scale);
/* density[j] = rms(rhs) y_j: the network's initial density for kfbi_solve_bie (device
 * [n] float64), on the context's stream. n <= max_rows of the network. Async. */
kfbi_status kfbi_warmstart_predict(kfbi_ctx* ctx, kfbi_mlp* mlp, const double* rhs, double* density);

/*
 * Learned warm start inside kfbi_step (not in the paper). With a network attached, every step
 * forms the network's initial density for its BIE (kfbi_warmstart_predict on the step's
 * right-hand side) and the residual norms ||b - A g|| of that guess and ||b - A x|| of the
 * previous step's density under the float64 operator (two applies), and starts GMRES from the
 * one with the smaller residual. GMRES still iterates to the step's tolerance, so the solution
 * is the method's either way. Scalars slot 14 counts the steps that took the network's start,
 * slot 15 holds the last ratio ||b - A g|| / ||b - A x||. mlp = NULL detaches; the network is
 * not owned (keep it alive while attached) and needs max_rows >= n.
 */
kfbi_status kfbi_thetal_set_warmstart(kfbi_thetal* st, kfbi_mlp* mlp);
/* kfbi_thetal_count -- the state's current node count (host int; marker doubling changes it). */
kfbi_status kfbi_thetal_count(kfbi_thetal* st, int* n);
/*
 * kfbi_thetal_training_pair -- the warm-start training sample of the system the last kfbi_step
 * solved: features [n][KFBI_MLP_FEATURES] float32 of its curve and right-hand side, and the
 * target density / rms(rhs) [n] float32 (device arrays). Asynchronous. Errors: ARG, STATE,
 * CAPACITY, CUDA.
 */
kfbi_status kfbi_thetal_training_pair(kfbi_thetal* st, float* feat, float* target);

/* ------------------------------------------------------------------------------------
 * Batched solves: many independent interface problems (each its own grid, box, kappa,
 * interface and right-hand side) solved by one CUDA graph launch. Each instance runs exactly
 * the method of kfbi_solve_bie (the paper solves one problem at a time, Sec. 4); the batch
 * only puts all instances' solves into one graph as independent branches and gathers their
 * results, so the host synchronises once per batch.
 * ------------------------------------------------------------------------------------ */
typedef struct {
  int N;                          /* cells per side (as kfbi_create) */
  double xmin, xmax, ymin, ymax;  /* square cells */
  double kappa;                   /* c^2 >= 0 */
  int boxbc;                      /* KFBI_BOX_* */
  int max_nodes;                  /* interface node capacity */
} kfbi_instance_desc;
typedef struct kfbi_batch kfbi_batch;

/* Creates count contexts (one per descriptor) in one precision (KFBI_FP64 or KFBI_MIXED).
 * Errors: ARG, CAPACITY, CUDA (as kfbi_create). */
kfbi_status kfbi_batch_create(int count, const kfbi_instance_desc* descs, int precision, kfbi_batch** out);
/* Destroys the batch and its contexts. NULL is ignored. */
void kfbi_batch_destroy(kfbi_batch* batch);
/* Context of instance i (owned by the batch): set its interface with kfbi_set_interface, use
 * any single-instance call on it. Errors: ARG. */
kfbi_status kfbi_batch_context(kfbi_batch* batch, int i, kfbi_ctx** ctx);
/* Stream the batch solve is ordered after (default: the legacy default stream). */
kfbi_status kfbi_batch_set_stream(kfbi_batch* batch, void* stream);
/* Solves every instance: rhs[i], density[i] device float64 [n_i] (host arrays of count
 * pointers); density[i] holds the initial guess and receives the solution. kind:
 * KFBI_BIE_INTERIOR_DL or KFBI_BIE_HS_EXTERIOR_MDL. tol, max_iter, restart as kfbi_solve_bie,
 * the same for all instances. infos: host [count] (NULL skips). The graph is rebuilt when an
 * interface, an option, a buffer pointer or tol / max_iter changed since the last call.
 * Synchronises once. Returns OK when every instance converged, else the first failing
 * status (NOT_CONVERGED before others); per-instance statuses are in infos.
 * Errors: ARG, STATE (an instance without interface), CUDA. */
kfbi_status kfbi_batch_solve(kfbi_batch* batch, int kind, const double* const* rhs, double* const* density,
                             double tol, int max_iter, int restart, kfbi_solve_info* infos);
/* Autotuner: for each grid size N of the batch, chooses the Gram-Schmidt form (16-CTA
 * cluster, 8-CTA cluster, five kernels), the column pairs per block of the column transform
 * (KFBI_OPT_COL_PAIRS 0, 1, 2, 4) and, in mixed batches, the float32 transform's form (radix-16
 * register-resident kernel, four-step register FFTs for N <= 1024, tensor-core contractions for
 * N <= 256, radix-4 shared-memory kernel: KFBI_OPT_COL_RADIX4 2 or 3) by timing whole batch
 * solves of rhs from zero (coordinate search, the second of two launches timed) and leaves the
 * fastest set on every context (read them back with kfbi_get_option). best_ms (host, NULL skips): batch solve time of the final choice.
 * Errors: ARG, STATE, CUDA. */
kfbi_status kfbi_batch_autotune(kfbi_batch* batch, int kind, const double* const* rhs, double tol, int max_iter,
                                int restart, double* best_ms);

/* Number of kernels this context has launched since creation (host output). */
kfbi_status kfbi_launch_count(kfbi_ctx* ctx, long long* count);

/*
 * kfbi_time_column -- mean duration of the column solve of the fast box solver (Sec. 4.2: DST/DCT
 * along y, division by the eigenvalues, inverse) in the form the context's options select, for
 * the roofline of the benchmark (not in the paper). fp32 = 1: the float32 kernel of the inner
 * applies, 0: the float64 kernel. One warm-up launch, then `reps` (1..100000) launches back to
 * back on the context's stream (programmatic dependent launch as in an apply) between two CUDA
 * events; writes the elapsed time / reps in microseconds to *us_per_launch (host). The
 * launches solve the context's spectral-grid scratch buffer in place: its contents are
 * meaningless afterwards, and the next apply rewrites it. Synchronises the stream.
 * Errors: ARG (NULL, reps out of range, fp32 not 0/1), STATE (during graph capture), CUDA.
 */
kfbi_status kfbi_time_column(kfbi_ctx* ctx, int fp32, int reps, double* us_per_launch);

/*
 * kfbi_alu_peak -- measured fused multiply-add throughput of this GPU, the denominator of the
 * ALU roofline fractions the benchmark reports (not in the paper). kind 0: float32 FMA,
 * 1: float64 FMA. Launches a probe kernel (eight independent FMA chains per thread, eight
 * 256-thread blocks per SM) four times on `stream` (cudaStream_t as void*; the first launch
 * warms up), times each with CUDA events and writes the best rate in TFLOP/s (2 flops per
 * FMA) to *tflops (host). Synchronises the stream; allocates nothing on the device.
 * Errors: ARG, CUDA.
 */
kfbi_status kfbi_alu_peak(int kind, double* tflops, void* stream);

/*
 * kfbi_tc_gemm -- C = A B^T on the fifth-generation tensor cores (tcgen05), the contraction
 * behind the warm-start network's 256-wide layers and the small-grid column transforms (not in
 * the paper). Float32 device matrices: A(m, k) = A[m lda + k] (transA = 0) or A[k lda + m]
 * (transA = 1), m < M, k < K; B(n, k) = B[n ldb + k] or B[k ldb + n], n < N; C[m ldc + n].
 * terms = 3 splits every input into two bfloat16 values (hi + lo) and accumulates
 * hi hi + hi lo + lo hi in float32 (about 2^-16 relative per product); terms = 4 is for B
 * exact in bfloat16: A is split into three bfloat16 terms (its full float32 value) and each
 * is multiplied by B; terms = 6 splits both into three terms and accumulates the six products
 * above 2^-24 relative (a float32-accurate contraction); terms = 1 takes the bfloat16 product
 * alone. error: device int, set to 1 if a completion wait gave up (the result
 * is then unspecified). Asynchronous on `stream` (cudaStream_t as void*); allocates nothing.
 * Errors: ARG, CUDA.
 */
kfbi_status kfbi_tc_gemm(int M, int N, int K, const float* A, long lda, int transA, const float* B, long ldb,
                         int transB, float* C, long ldc, int terms, int* error, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* KFBI_H */
