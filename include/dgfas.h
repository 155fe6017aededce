/*
 * dgfas.h - C ABI of the B300 FAS multigrid hot path for SIP DG-SEM elliptic
 * problems (Stiller, "Adaptive multigrid for high-order discontinuous Galerkin
 * methods based on the full approximation scheme").
 *
 * Problem (Sec. 2.1, Eq. (1)):  kappa u - div(nu grad u) = f in Omega, u = u_D
 * on Dirichlet faces, nu du/dn = q_N on Neumann faces; constant kappa >= 0 and
 * nu > 0.  Discretization (Sec. 2.2, Eq. (2)): symmetric interior penalty DG on
 * hexahedra with a GLL nodal basis of degree p per element and GLL collocation
 * quadrature; the algebraic system is A u = f (Eq. (3)).
 *
 * Conventions shared by every call
 * - Vectors are FP64, element-major: u[e][k][j][i] with i fastest, (p+1)^3
 *   nodes per element, e the element index of the level.
 * - Vector pointers passed to the calls below are DEVICE pointers owned by the
 *   caller unless stated otherwise; mesh arrays in dgfas_level are HOST
 *   pointers, copied during setup (the caller may free them afterwards).
 * - Every call is ordered on the CUDA stream given at setup and is
 *   asynchronous, except where a host output (rnorm_out, info) forces a
 *   synchronization.
 * - Return codes: DGFAS_OK (0) or a negative DGFAS_ERR_* code; nothing throws
 *   across the ABI.  dgfas_strerror() gives a static message for a code, and
 *   dgfas_last_error() the detail of the last failure in this thread.
 */
#ifndef DGFAS_H
#define DGFAS_H

#ifdef __cplusplus
extern "C" {
#endif

#define DGFAS_OK 0
#define DGFAS_ERR_INVALID -1        /* bad argument or inconsistent mesh arrays */
#define DGFAS_ERR_OOM -2            /* device allocation failed */
#define DGFAS_ERR_CUDA -3           /* a CUDA runtime call failed */
#define DGFAS_ERR_MESH -4           /* non-positive Jacobian at a GLL node, or faces
                                       not shared with aligned local axes */
#define DGFAS_ERR_NOT_CONVERGED -5  /* max_cycles reached before rtol */
#define DGFAS_ERR_DIVERGED -6       /* NaN/Inf or residual growth > 1e3 x r_0 */
#define DGFAS_ERR_UNSUPPORTED -7    /* p > 10, subdomain width > 16, ... */

/* element classes of Sec. 3.1 */
#define DGFAS_LEAF 0
#define DGFAS_TWIG 1
#define DGFAS_FROZEN 2

/* smoother-internal precision (the V-cycle residual, tau, restriction and
   root solve are always FP64) */
#define DGFAS_FP64 0
#define DGFAS_FP32 1
#define DGFAS_BF16 2   /* FP32 smoother residual and combine; FD mode products on
                          the tensor cores (BF16 operands, FP32 accumulation, FP32
                          scaling by the inverse eigenvalue sums) */

/* smoother (Sec. 4.3): weighted additive Schwarz (Alg. 5) or Schwarz-
   preconditioned inexact CG (Alg. 6).  SCG takes the preconditioned residual
   as its first search direction (p = z), as in the inexact PCG of Golub and
   Ye that Sec. 4.3.2 adopts; all its scalar products stay on the device, so an
   SCG smoother issues no host synchronization. */
#define DGFAS_WAS 0
#define DGFAS_SCG 1

/* root (coarsest-level) solver (Sec. 4.3.2: SCG also serves as the solver of
   the coarse problem): the exact dense inverse (root <= 8192 DoF), or FP64 SCG
   from the projected solution, root_steps steps or until
   |r| <= root_rtol |r_start| */
#define DGFAS_COARSE_DENSE 0
#define DGFAS_COARSE_SCG 1

/* FAS solution projection P (Sec. 3.2): embedded interpolation (the fine
   polynomial at the coarse nodes, averaged at nodes shared by h-children for
   even p), or L2 projection in reference coordinates with the fine GLL
   quadrature, P = (I^T W I)^-1 I^T W per direction (each h-child contributes
   its half of the parent's width; no averaging) */
#define DGFAS_P_INTERP 0
#define DGFAS_P_L2 1

/* One level of the multilevel mesh (Sec. 3.1): a conforming hexahedral mesh
   with one polynomial degree.  All arrays are host arrays of n_elem rows. */
typedef struct {
  int p;                     /* polynomial degree, 1 <= p <= 10 */
  int n_elem;
  const double* corners;     /* [n_elem][8][3] trilinear map corners,
                                corner c = cx + 2 cy + 4 cz */
  const int* nbr;            /* [n_elem][6] face (-x,+x,-y,+y,-z,+z): neighbour
                                element, -1 Dirichlet, -2 Neumann; neighbours
                                share aligned local axes */
  const int* nbr27;          /* [n_elem][27] element at offset (ox,oy,oz) in
                                {-1,0,1}^3, slot (ox+1)+3(oy+1)+9(oz+1), -1 none
                                (overlap layers of the Schwarz subdomains) */
  const int* parent;         /* [n_elem] element of level l-1; ignored on root */
  const int* octant;         /* [n_elem] h-child octant cx+2cy+4cz, or -1 when
                                the parent is the same element (p-refinement) */
  const signed char* cls;    /* [n_elem] DGFAS_LEAF / TWIG / FROZEN */
} dgfas_level;

typedef struct {
  int n_levels;              /* >= 1, root first */
  const dgfas_level* levels;
  double nu;                 /* diffusivity (constant) */
  double kappa;              /* reaction coefficient (constant, >= 0) */
} dgfas_mesh;

typedef struct {
  double mu_star;            /* penalty scaling mu_* > 1 (Sec. 2.2) */
  double delta;              /* Schwarz overlap 0 < delta < 0.5 (Sec. 4.3.1) */
  int s1, s2, sc;            /* pre-, post-, crossover smoothing steps */
  int precision;             /* DGFAS_FP64, DGFAS_FP32 or DGFAS_BF16 smoother */
  int smoother;              /* DGFAS_WAS or DGFAS_SCG */
  int max_cycles;            /* default cap for dgfas_solve when <= 0 is passed */
  int coarse;                /* DGFAS_COARSE_DENSE or DGFAS_COARSE_SCG */
  double root_rtol;          /* SCG root: relative exit tolerance (<= 0: 1e-3) */
  int root_steps;            /* SCG root: step cap per visit (<= 0: 64); the
                                steps past the exit test leave u unchanged, so
                                a visit is a fixed launch sequence (graphs) */
  int projection;            /* DGFAS_P_INTERP or DGFAS_P_L2 */
} dgfas_params;

typedef struct {
  int cycles;                /* V-cycles run */
  double r0;                 /* initial residual r_2^0 */
  double r_final;            /* final residual r_2 */
  double seconds;            /* wall time of the cycles (host clock) */
  double history[128];       /* r_2 after each cycle (first 128) */
} dgfas_info;

/* Builds all device state of the hierarchy: geometry factors, penalties, the
   nine 1D fast-diagonalization variants per level (Sec. 4.3.1), the geometric
   surrogate widths per element, transfer matrices (Sec. 3.2) and the factorized
   root operator.  `cuda_stream` is a cudaStream_t (NULL = legacy default).
   Errors: INVALID (arrays inconsistent), UNSUPPORTED, MESH, OOM, CUDA. */
int dgfas_setup_levels(const dgfas_mesh* mesh, const dgfas_params* prm,
                       void* cuda_stream, void** out_ctx);

/* Host-only validation of a hierarchy's input arrays, also run first by
   dgfas_setup_levels (no device work, callable without a GPU): arrays present,
   1 <= p <= 10, neighbour indices in range, the 27-neighbourhood's centre slot
   the element and its face slots the face neighbours (-1 on boundary faces)
   (INVALID / UNSUPPORTED), and the
   face-neighbour relation reciprocal through the opposite face with the two
   faces' corners coinciding corner by corner up to one translation (aligned
   local axes; periodic identification by translation), else DGFAS_ERR_MESH
   with the element and face in dgfas_last_error(). */
int dgfas_check_mesh(const dgfas_mesh* mesh);

void dgfas_destroy(void* ctx);

/* DoF count (n_elem (p+1)^3) of level `level` (0 = root), or a negative code. */
long long dgfas_level_ndof(void* ctx, int level);

/* Physical coordinates of the GLL nodes of `level` into xyz [ndof][3] (device).
   Used to sample manufactured data f(x), u_D(x). */
int dgfas_node_coords(void* ctx, int level, double* xyz);

/* Right-hand side of Eq. (2) on the top level: b = int v f + Dirichlet terms
   (2 mu nu v u_D - nu dv/dn u_D), from nodal f and u_D (both [ndof], device;
   uD may be NULL for u_D = 0). */
int dgfas_assemble_rhs(void* ctx, const double* f_nodal, const double* uD_nodal,
                       double* b);

/* Right-hand side of Eq. (2) on any level (as dgfas_assemble_rhs); with local
   refinement the leaves of every level need their own RHS. */
int dgfas_assemble_rhs_level(void* ctx, int level, const double* f_nodal,
                             const double* uD_nodal, double* b);

/* Sets the RHS f_l [ndof of level] (device) kept on the leaf elements of a
   level below the top (Eq. (4c): leaves replicate the original RHS).  Levels
   without leaves ignore it. */
int dgfas_set_level_rhs(void* ctx, int level, const double* f);

/* r_2 of Sec. 6.1: the Euclidean norm of the residual over the leaf elements
   of all levels (the top level's from u_top, f_top; the others from the
   context's level solutions and their leaf RHS).  Synchronizes. */
int dgfas_composite_residual(void* ctx, double* u_top, const double* f_top, double* out);

/* Copies the context's current solution of a level below the top into u. */
int dgfas_get_level_solution(void* ctx, int level, double* u);

/* Operator application of Eq. (2) on `level`: out = A u, or out = g - A u when
   g != NULL (the residual; rows of frozen elements are 0, Eq. (4d)).  u, g, out
   [ndof] device; out must not alias u. */
int dgfas_apply_op(void* ctx, int level, const double* u, const double* g, double* out);

/* The smoother-precision operator of the same equation: out = g - A u (g != NULL)
   or A u (g == NULL) with u, out and the arithmetic in FP32 and g FP64; the
   form every FP32 / BF16 smoother applies to its corrections (on curvilinear
   levels the metric is recomputed in FP32 from the trilinear map).  u, out
   [ndof] FP32, g [ndof] FP64, all device; out must not alias u. */
int dgfas_apply_op32(void* ctx, int level, const float* u, const double* g, float* out);

/* n sweeps of the level smoother (Alg. 5 WAS, or Alg. 6 SCG if selected) on
   A u = g: each WAS sweep computes r = g - A u and adds the weighted Schwarz
   correction sum_e R_s^T W^e (A~_s^e)^-1 R_s r of Eq. (11); frozen entries of u
   are unchanged.  u updated in place. */
int dgfas_schwarz_smooth(void* ctx, int level, double* u, const double* g, int nsweeps);

/* One FAS V-cycle (Alg. 2) on the hierarchy: s1 pre-smoothing sweeps on the
   top level, residual, projection, parent RHS (tau), ..., root solve,
   correction prolongation, s2 post-smoothing.  u_top [ndof_top] updated in
   place, f_top the top RHS.  If rnorm_out != NULL the Euclidean norm of the
   top residual after pre-smoothing is written there (synchronizes). */
int dgfas_fas_vcycle(void* ctx, double* u_top, const double* f_top, double* rnorm_out);

/* V-cycles with crossover smoothing (Sec. 6.1) until r_2 <= rtol * r_2^0 or
   max_cycles: s1 top sweeps, then per cycle the stopping test on the top
   residual, the FAS down/up legs and sc top sweeps.  Synchronizes every cycle
   for the stopping test.  Returns OK, NOT_CONVERGED or DIVERGED. */
int dgfas_solve(void* ctx, double* u_top, const double* f_top, double rtol, int max_cycles,
                dgfas_info* info);

/* Euclidean norm of v [ndof of level] (deterministic two-pass reduction). */
int dgfas_norm(void* ctx, int level, const double* v, double* out_host);

/* Replaces the per-element surrogate coefficients g0..g3 of Eq. (10) on
   `level` (default: the geometric surrogate of Sec. 4.3.1) by g [n_elem][4]
   (device, FP64), e.g. the output of the learned surrogate. */
int dgfas_set_surrogate(void* ctx, int level, const double* g);

/* Copies the current surrogate coefficients of `level` to g [n_elem][4] (device). */
int dgfas_get_surrogate(void* ctx, int level, double* g);

/* Enables (1) or disables (0) CUDA-graph replay of the V-cycle body in
   dgfas_fas_vcycle / dgfas_solve (captured on first use per (u, f) pair; the
   graphs of the four most recently used pairs are kept, so a caller may
   alternate buffers, e.g. to overlap its own copies with the solve). */
int dgfas_use_graph(void* ctx, int enable);

/* Per-kernel timing of `reps` smoother sweeps on `level` (level >= 1) with CUDA
   events on the context's stream.  ms_out [4] (host) receives the average
   duration in ms of: the smoother-precision residual, the FD kernel (gather,
   fast diagonalization, weighting), the combine kernel, and the FP64 residual
   apply of the V-cycle.  u is updated by the sweeps. */
int dgfas_profile_sweep(void* ctx, int level, double* u, const double* g, int reps,
                        double* ms_out);

/* Per-kernel timing of one SCG step (Alg. 6) on `level` (>= 1) in the
   context's smoother precision, CUDA events on the context's stream, averaged
   over `reps` steps from the residual g - A u.  ms_out [6] (host): the FD
   kernel of the Schwarz sweep, its combine, the scalar product z.r with the
   direction update, the operator A p, the scalar product p.q with the fused
   residual / iterate update, and the FP64 residual apply.  u is not modified;
   the level's work vectors are scratch afterwards.  INVALID unless the
   context was set up with SCG (smoother or root). */
int dgfas_profile_scg(void* ctx, int level, double* u, const double* g, int reps, double* ms_out);

/* Outcome of the last SCG block run on the context's stream (the root solve of
   the last V-cycle when the root solver is DGFAS_COARSE_SCG): out_host[0] =
   |r|^2 when its exit test last ran, out_host[1] = the steps taken before the
   test |r| <= root_rtol |r_start| held (the step cap if it never did),
   out_host[2] = 1 if it held, 0 if the visit ended at its step cap.
   Synchronizes the stream. */
int dgfas_scg_info(void* ctx, double* out_host);

/* Full multigrid startup (FAS-FMG, Alg. 4): the root is solved exactly for
   its own right-hand side f_levels[0]; then for l = 1 .. L-1 the root's (or
   previous level's) solution is interpolated to level l, u_l = I u_{l-1},
   and cycles_per_level FAS V-cycles (Alg. 2) with level l as the top and its
   own right-hand side f_levels[l] improve it; finally u_top = I u_{L-1}.
   u_top (device, top-level layout) is the start value for dgfas_solve /
   dgfas_fas_vcycle on the full hierarchy.  f_levels: host array of
   n_levels device pointers, f_levels[l] the assembled right-hand side of
   level l (dgfas_assemble_rhs_level), f_levels[n_levels-1] the top's (read
   only for validation).  Paper: one V-cycle per level.  On a locally refined
   hierarchy level l's active rows all use f_levels[l] while it is the top,
   the leaves below it the right-hand sides set by dgfas_set_level_rhs, and
   the level solutions it leaves below the top (lv u) are the start of the
   following composite solve.  DGFAS_ERR_UNSUPPORTED for a single level.
   Stream-ordered, not captured. */
int dgfas_fmg(void* ctx, const double* const* f_levels, int cycles_per_level, double* u_top);

/* Cascadic startup (FAS-CMG, Alg. 3): the root is solved for its own
   right-hand side f_levels[0] (as by the root solver of the context); then
   for l = 1 .. L-1 the previous level's solution is interpolated to level l
   (the whole level, frozen elements included), u_l = I u_{l-1}, and improved
   by n_sc steps of the level smoother (WAS or SCG, in the context's
   precision) on A_l u_l = f_levels[l]; finally u_top = I u_{L-1}.  Same
   arguments, level solutions and stream ordering as dgfas_fmg; n_sc >= 0
   (0: interpolation only).  DGFAS_ERR_UNSUPPORTED for a single level. */
int dgfas_cmg(void* ctx, const double* const* f_levels, int n_sc, double* u_top);

/* Element error indicators of the adaptive loop (Sec. 6.4): the level-l
   operator applied to the complete error vector eps [ndof(level)] (device),
   restricted to each element and weighted with that element's error
   coefficients: out[e] = eps_e . (A_l eps)_e, out [n_elem] (device).  Rows of
   frozen elements are 0 (the operator's frozen rows).  Summed over the leaf
   elements of every level it gives the square of the composite energy norm
   of the error (Sec. 6.1).  Stream-ordered; uses the context's smoother
   scratch, so not concurrently with a solve. */
int dgfas_element_energy(void* ctx, int level, const double* eps, double* out);

/* Launch-shape autotuner (the batching / tile-tuning step of the hot path):
   for every level it times, with CUDA events on the context's stream, the
   candidate launch shapes of the tunable kernels and keeps the fastest:
     kernel 0  FP64 operator (residual, tau):        elements per CTA
     kernel 1  smoother-precision operator:          elements per CTA
     kernel 2  FD for subdomains narrower than 9:    elements per CTA
     kernel 3  tensor-core FD (BF16, width >= 12):   CTAs per SM
   Every candidate computes bit-identical results (the shapes only change how
   elements are mapped to CTAs).  reps launches are timed per candidate
   (the built-in default, value 0, included).  report [max_entries][5] (host,
   nullable when max_entries = 0) receives (level, kernel, chosen value,
   best ms, default ms) per tuned pair; *n_entries their number.  Synchronous.
   The level work vectors and the patch buffer are used as scratch, so call it
   between solves, never while a stream capture is active; a captured V-cycle
   graph is dropped and captured again on next use. */
int dgfas_autotune(void* ctx, int reps, double* report, int max_entries, int* n_entries);

/* Forces the launch shape of `kernel` (0..3, as above) on `level`: value 0
   restores the default, any other value must be one of the candidates that
   dgfas_get_tuning lists (else DGFAS_ERR_INVALID). */
int dgfas_set_tuning(void* ctx, int level, int kernel, int value);

/* Current launch shape (*value, 0 = default) of `kernel` on `level` and,
   if n_candidates is not null, its candidate values (candidates
   [max_candidates], host) and their number. */
int dgfas_get_tuning(void* ctx, int level, int kernel, int* value, int* candidates,
                     int max_candidates, int* n_candidates);

/* Measured FMA throughput of the current device in TFLOP/s (FP64 and FP32):
   the denominators of the roofline of ALU-bound kernels. */
int dgfas_fma_peak(double* tflops_fp64, double* tflops_fp32);

/* Host-only (no device work): the fast-diagonalization data of one side variant
   (variant = 4*left + right with side types 0 = interior, 1 = Dirichlet,
   2 = Neumann, 3 = interior face whose neighbour is frozen, which contributes
   no overlap layers) for
   degree p, overlap delta and penalty mu_star (Sec. 4.3.1): subdomain width n,
   S [n][n] (row = node, column = mode; S^T M S = I, S^T L S = diag(lambda)),
   lambda [n] and the weights W [n].  Buffers of at least 16*16 / 16 doubles. */
int dgfas_host_fd_variant(int p, double delta, double mu_star, int variant, double* S,
                          double* lam, double* W, int* n_out);

/* ---- learned surrogate (the paper has no learned part; this is the
   network that predicts the surrogate coefficients of Eq. (10) from an
   element's corners).  MLP 24 -> 64 -> 64 -> 6, tanh hidden layers, linear
   output, FP32; parameters in one flat device array of
   dgfas_mlp_param_count() floats: W1[64][24] b1[64] W2[64][64] b2[64]
   W3[6][64] b3[6].  Inputs X [n][24]: corner coordinates minus the centroid,
   divided by V^(1/3); outputs [n][6]: log(dx_i / V^(1/3)), log(s_i). */
int dgfas_mlp_param_count(void);

/* The network's inputs X [n][24] (device FP32) of n elements given by their
   corners [n][8][3] (device FP64): corner coordinates minus the centroid,
   divided by the cube root of the element volume (2-point Gauss of det J).
   Synchronizes `stream`. */
int dgfas_mlp_inputs(const double* corners, int n, float* X, void* stream);

/* out [n][6] = MLP(params, X) (device pointers; synchronizes `stream`). */
int dgfas_mlp_forward(const float* params, const float* X, int n, float* out, void* stream);

/* grad [param_count] = d/dparams of the mean squared error of MLP(X) - Y over
   all n samples and 6 outputs (device pointers; synchronizes). */
int dgfas_mlp_grad(const float* params, const float* X, const float* Y, int n, float* grad,
                   void* stream);

/* Adam training (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with
   minibatches of `batch` samples drawn by a per-epoch permutation from `seed`.
   params, m, v [param_count] device, updated in place (m = v = 0 and t0 = 0 at
   the start); X [n][24], Y [n][6] device.  loss_out (host, may be NULL)
   receives the full-data loss after every epoch.  Synchronizes. */
int dgfas_mlp_train(float* params, float* m, float* v, const float* X, const float* Y, int n,
                    int epochs, int batch, float lr, unsigned long long seed, int t0,
                    float* loss_out, void* stream);

/* Sets the surrogate coefficients of `level` from the network's prediction:
   g_i = s_i nu dx_j dx_k / (2 dx_i), g_0 = kappa dx_1 dx_2 dx_3 / 8.  Elements
   whose predicted |log s_i| exceeds max_log_scaling (or is not finite) keep
   their geometric coefficients; their count goes to *n_fallback (host). */
int dgfas_learned_surrogate(void* ctx, int level, const float* params, double max_log_scaling,
                            int* n_fallback);

/* 1 if a completion wait of the tensor-core FD kernel ran out since setup
   (its bounded waits never hang; a timed-out sweep leaves an invalid patch),
   0 otherwise, or a negative code. */
int dgfas_tc_error(void* ctx);

/* Self-test of the tensor-core path (tcgen05.mma kind::f16, BF16 operands,
   FP32 accumulation in TMEM): one CTA computes D[128][16] = A B^T with
   A[r][k] = (r + 2k) % 7 - 3 and B[n][k] = (3n + k) % 5 - 2 (exact in BF16 and
   FP32) into out_host [128*16]; *timeout_host = 1 if the completion wait ran
   out (the kernel never waits unboundedly). */
int dgfas_tc_selftest(float* out_host, int* timeout_host);

/* Self-test of an MN-major A operand (no swizzle) for tcgen05.mma: out_host
   [2][128][16] holds D for the two assignments of the core-matrix strides to
   the descriptor's leading / stride byte offsets ([1] is the layout the FD
   kernel uses: leading = stride along K, stride = stride along M). */
int dgfas_tc_selftest_mn(float* out_host, int* timeout_host);

/* Number of kernels the library has launched in this process (including the
   kernel nodes of replayed CUDA graphs). */
long long dgfas_kernel_launches(void);

/* Allocation-free Schwarz correction (the paper has no counterpart; it exists
   for callers that cannot allocate device memory when they smooth, e.g. code
   running inside its own stream capture or under an allocator that owns all
   device memory).  Adds to u [ndof] the FP64 weighted Schwarz correction
   u += sum_e R_s^T W^e (A~_s^e)^-1 R_s r of the residual r [ndof] on `level`
   (>= 1): the subdomain patches of r, the fast-diagonalization solves with the
   level's surrogate, the overlap weights, and the sum back into u.  Both are
   device pointers; u is updated in place, r is read only.
   Scratch: a fixed 16 MiB device array inside the library (2^21 FP64 patch
   entries) replaces the context's patch buffer; levels needing more, i.e.
   n_elem (p+1+2m)^3 > 2^21, are rejected with DGFAS_ERR_UNSUPPORTED.  The call
   makes no device allocation of any kind.  Its first call on a device looks up
   the array's device address (cudaGetSymbolAddress), so make that first call
   before any stream capture.  The address is kept for the life of the process:
   do not reset the device (cudaDeviceReset) between calls.  Devices numbered
   64 or higher are refused (DGFAS_ERR_UNSUPPORTED).  All calls share the one array: calls whose work
   overlaps on the GPU (different streams, or several contexts) race on it. */
int dgfas_schwarz_correct_static(void* ctx, int level, const double* r, double* u);

const char* dgfas_strerror(int code);
const char* dgfas_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DGFAS_H */
