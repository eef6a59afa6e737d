/*
 * mch.h - C ABI of the GB300 (sm_103a) hierarchical multicontinuum cell-problem solver.
 *
 * What it computes (arXiv 2503.01276):
 *   For every macropoint x_p of every level n of a nested macrogrid (Sec. 3.1, Eq. defi_Sn),
 *   the R = N (1 + d) constrained cell functions Phi_p (Sec. 2, Eqs. phi_avar and phi_grad,
 *   in the energy form of Sec. 3, Eq. phi_abstract): minimise 1/2 int kappa |grad v|^2 over
 *   Q1 finite-element functions on the RVE Y+ = [-l/2, l/2]^d that vanish on its boundary,
 *   subject to int_{R_q} psi_j v = delta_ij int_{R_q} psi_j          (constant functions)
 *   and        int_{R_q} psi_j v = delta_ij int_{R_q} (x_m - c_mj) psi_j (linear functions)
 *   for every continuum j and every sub-block R_q (the P^d periods of the RVE).
 *   At level n > 1 the function is the interpolation of the parents' functions plus a
 *   correction solved on the level's coarser grid (Sec. 3.3, Eqs. PhiXiI, phiXiI_all,
 *   phi_avar_corrector, phi_grad_corrector). The effective coefficients are the energy Gram
 *   of the cell functions (Sec. 2, Eq. Bs_defi), reported as
 *       E[p][r][s] = (1/|R_p|) int_{R_p} kappa grad Phi_r . grad Phi_s,
 *   with R_p = Y+ (no oversampling); the caller multiplies by |K_p|. Cell function r is
 *   phi_i for r = i < N and phi_i^m for r = N + i d + m.
 *
 * Conventions:
 *   - Macro indices run over [0, macro_n)^d; level n contains the indices that are multiples
 *     of level_stride[n-1] along every axis and not in an earlier level. Points of a level
 *     are ordered lexicographically with x fastest.
 *   - Level n uses an RVE grid of n_fine / eta^(n-1) elements per side. Element fields are
 *     stored per point as [n^d] with x fastest; kappa is FP64, labels are uint8 continuum
 *     indices in [0, n_cont).
 *   - Every pointer argument may be host memory or device memory of the current device; the
 *     library detects which and stages host buffers through its own device buffers (the
 *     copies are counted by mch_level_stats). All work is enqueued on the stream given to
 *     mch_create and each call synchronises that stream once before returning its status.
 *   - The library owns its workspaces and the cell functions of every level; the caller owns
 *     every buffer it passes in.
 *   - Level n may only be solved after levels 1..n-1 (MCH_ERR_ORDER otherwise).
 */
#ifndef MCH_H
#define MCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mch_handle mch_handle;

typedef enum {
  MCH_OK = 0,
  MCH_ERR_ARG = 1,            /* invalid argument or descriptor                      */
  MCH_ERR_CUDA = 2,           /* a CUDA call failed (see mch_last_error)              */
  MCH_ERR_OOM = 3,            /* device allocation failed                             */
  MCH_ERR_ORDER = 4,          /* a level was solved before its parent levels          */
  MCH_ERR_NOT_CONVERGED = 5,  /* iteration or refinement cap reached above rtol       */
  MCH_ERR_BREAKDOWN = 6,      /* non-positive curvature or non-finite value in PCG    */
  MCH_ERR_DEGENERATE = 7,     /* singular constraint Gram, kappa <= 0, empty continuum */
  MCH_ERR_UNSUPPORTED = 8     /* a size this build has no kernel for                  */
} mch_status;

enum { MCH_FP64 = 0, MCH_MIXED = 1 };

typedef struct {
  int dim;                  /* d: 2 or 3                                                    */
  int n_cont;               /* N: continua, 1..4                                            */
  int n_levels;             /* L                                                            */
  int eta;                  /* FE coarsening factor between levels (Sec. 3.2)               */
  int macro_n;              /* macro indices per axis on T_L                                */
  const int *level_stride;  /* [n_levels] stride of T_n in macro-index units, last = 1      */
  int n_fine;               /* elements per RVE side at level 1                             */
  int periods;              /* P: sub-blocks R_q per side; n_level / P must be >= 2         */
  int overs;                /* oversampling layers o: E is integrated over R_p, the central
                               (P - 2o)^d periods, with centroids c_mj over R_p (Sec. 2, Eqs.
                               phi_grad, Bs_defi); constraints stay on every period. 2D only
                               (3D: MCH_ERR_UNSUPPORTED); P - 2o >= 1. E over R_p is not
                               stationary in the cell functions, so mch_backward treats the
                               level's own term as an adjoint source                         */
  double rve_len;           /* l: RVE side length                                           */
  int precision;            /* MCH_MIXED (FP32 PCG inside FP64 refinement) or MCH_FP64      */
  double rtol;              /* stop when sqrt(r'M^-1 r / rho_ref) < rtol for the FP64
                               projected residual r (0 -> 1e-8), with rho_ref the larger of
                               the first step's r'M^-1 r and b'M^-1 b, b the right-hand side
                               of a correction problem (n > 1), so the test bounds the error
                               of the cell function I + P Xi relative to its own scale. A
                               child's coefficients inherit the error of its parents'
                               functions to first order (about rtol); a level's own
                               coefficients are quadratic in its error */
  double inner_tol;         /* per-sweep PCG reduction of the same norm (0 -> 1e-5 in 2D,
                               1e-4 in 3D)                                                  */
  int max_iter;             /* PCG iterations per sweep (0 -> 4 n_level + 50)               */
  int max_refine;           /* refinement sweeps (0 -> 6)                                   */
  int keep_parents;         /* 1: keep every level's cell functions on the level-1 grid
                               after the forward pass (checkpoint for mch_backward);
                               0: free them once the last level is solved and after
                               mch_backward, and recompute them from the stored level-grid
                               solutions (interpolation + prolongation, no new solve) when
                               mch_backward, mch_cell_functions or a later mch_solve_level
                               needs them                                                   */
  int interp;               /* parents of a point of level n > 1 (Sec. 3.3): 0 = vertices of
                               the enclosing T_{n-1} cell with multilinear weights; 1 = the
                               nearest point of S_1 with weight one (the paper's experiments:
                               I_p = Phi_t, x_t in S_1; ties to the lower index)            */
  int point_batch;          /* points per constrained-solve launch: 0 = the whole level in
                               one persistent launch; k > 0 = at most k points per launch
                               (1 = one macropoint per launch, the unbatched comparator).
                               Results do not depend on it                                   */
} mch_desc;

typedef struct {
  int n_points;             /* points of the level                                  */
  int n_elem;               /* elements per RVE side on this level                  */
  int sweeps;               /* refinement sweeps used (max over the level)          */
  int max_iters;            /* largest PCG iteration count of one (point, function) */
  long long total_iters;    /* sum of PCG iterations over (point, function, sweep)  */
  double max_relres;        /* largest final FP64 projected residual ratio          */
  int n_dropped_rows;       /* constraint rows of empty (continuum, sub-block) pairs */
  int gpu_launches;         /* kernels launched by the last mch_solve_level         */
  long long h2d_bytes;      /* bytes staged host->device by the last call           */
  long long d2h_bytes;      /* bytes staged device->host by the last call           */
  /* Filled only while timing is enabled (mch_set_timing): CUDA-event times on the handle's
   * stream of each phase of the last mch_solve_level, in milliseconds.                    */
  double setup_ms;          /* constraint data                                      */
  double interp_ms;         /* interpolation and correction right-hand sides        */
  double pcg_ms;            /* all PCG sweep launches                               */
  double prep_ms;           /* all FP64 refinement steps                            */
  double final_ms;          /* effective coefficients and cell-function assembly    */
  int pcg_launches;         /* PCG sweep launches                                   */
  long long pcg_node_iters; /* sum over units of PCG iterations x interior nodes    */
  long long pcg_node_applies; /* sum over units of inner stencil applications x interior
                               nodes (PCG iterations times the preconditioner's Chebyshev
                               steps, plus its first application per sweep)            */
} mch_level_stats;

/* Validates the descriptor, builds the level plan (Eq. defi_Sn; parents and multilinear
 * weights of Sec. 3.3) on the host and allocates the per-level workspaces on the current
 * device. `cuda_stream` is a cudaStream_t (NULL = legacy default stream). On failure *out
 * is NULL and the status says why. */
mch_status mch_create(const mch_desc *desc, void *cuda_stream, mch_handle **out);

/* Host-only (no GPU work, no allocation on the device): the level plan of a descriptor.
 * Writes the number of points of level `level` to *n_points and, for each non-NULL array,
 * the macro indices [n_points][dim], parent levels (1-based, 0 = unused slot), parent
 * positions and weights [n_points][2^dim]. Call with NULL arrays first to size them. */
mch_status mch_plan_level(const mch_desc *desc, int level, int *n_points, int32_t *idx_out,
                          int32_t *parent_level, int32_t *parent_pos, double *weight);

/* Number of points of level `level` (1-based), or -1 for a bad handle/level. */
int mch_level_num_points(const mch_handle *h, int level);

/* Elements per RVE side of level `level`, or -1. */
int mch_level_n_elem(const mch_handle *h, int level);

/* Writes the macro indices of the level's points, [n_points][dim] int32, host memory. */
mch_status mch_level_points(const mch_handle *h, int level, int32_t *idx_out);

/* Writes the parents of the level's points: for point i, entries [i][0..2^dim) of
 * parent_level (1-based, 0 = unused), parent_pos and weight (Sec. 3.3: sum of weights 1).
 * Host memory, each array [n_points][2^dim]. */
mch_status mch_level_parents(const mch_handle *h, int level, int32_t *parent_level,
                             int32_t *parent_pos, double *weight);

/* Solves all cell problems of level `level` (Algorithm 1, lines 4-6): builds the constraint
 * data (Eqs. phi_avar, phi_grad), the interpolation of the parents and the correction
 * right-hand sides (Eqs. phi_avar_corrector, phi_grad_corrector), runs the batched
 * constrained solves, assembles Phi = I + Xi on the level-1 grid and reduces the effective
 * coefficients (Eq. Bs_defi). kappa [n_points][n^d] FP64 > 0 and labels [n_points][n^d]
 * uint8 (host or device). Status MCH_ERR_NOT_CONVERGED still leaves usable results whose
 * residuals are reported by mch_level_stats. */
mch_status mch_solve_level(mch_handle *h, int level, const double *kappa, const uint8_t *labels);

/* One level of a hierarchy shared by several handles (one per GPU): the macropoints of a
 * level are independent (Algorithm 1, lines 4-6), so each handle solves a contiguous range
 * [p0, p1) of them and the children of every level read their parents' cell functions,
 * which the other handles computed (Eq. phiXiI_all). This call solves points p0..p1-1 of
 * `level` exactly as mch_solve_level would; kappa and labels hold those p1 - p0 points only
 * ([p1 - p0][n^d], host or device). Every parent of the range must have cell functions on
 * this handle: solved here, or imported with mch_set_cell_functions. An empty range
 * (p0 == p1) only marks the level as complete on this handle (after its cell functions
 * were imported). Coefficients, iteration counts and cell functions of points outside the
 * ranges solved here are not computed (mch_effective_coeffs and mch_cell_functions still
 * copy whole levels). mch_backward refuses a handle that solved any level by ranges
 * (MCH_ERR_ORDER). MCH_ERR_ARG for a range outside [0, n_points]. */
mch_status mch_solve_level_range(mch_handle *h, int level, int p0, int p1, const double *kappa,
                                 const uint8_t *labels);

/* Imports the cell functions of points p0..p1-1 of `level`, computed by another handle (the
 * exchange step of a hierarchy split over several GPUs): phi [p1 - p0][R][(n_fine+1)^d] FP64
 * on the level-1 lattice (the layout of mch_cell_functions), host or device; copied (and in
 * mixed precision stored as float-float) into the library's storage, where the children of
 * later levels read them. Synchronises the handle's stream. */
mch_status mch_set_cell_functions(mch_handle *h, int level, int p0, int p1, const double *phi);

/* Copies the level's effective coefficients E [n_points][R][R] FP64 to `E` (host or device).
 * Optional outputs (NULL to skip): iters [n_points][R] int32 total PCG iterations, relres
 * [n_points][R] FP64 final projected residual ratio. */
mch_status mch_effective_coeffs(mch_handle *h, int level, double *E, int32_t *iters,
                                double *relres);

/* Copies the level's cell functions on the level-1 grid, [n_points][R][(n_fine+1)^d] FP64
 * (node lattice including the zero boundary, x fastest), to `phi` (host or device). With
 * keep_parents = 0 the cell functions are recomputed first if they were freed. */
mch_status mch_cell_functions(mch_handle *h, int level, double *phi);

/* Enables (1) or disables (0) CUDA-event timing of the phases of mch_solve_level (adds
 * event records on the handle's stream; no extra synchronisation). */
mch_status mch_set_timing(mch_handle *h, int enable);

/* Statistics of the last mch_solve_level call on `level` (host struct). */
mch_status mch_level_stats_get(const mch_handle *h, int level, mch_level_stats *out);

/* Optional, ahead of mch_solve_level: stages the level's kappa and labels and computes its
 * constraint data (setup) on a side stream of the handle, ordered after the work already
 * enqueued on the handle's stream. A later mch_solve_level on the same level with the same
 * kappa and labels pointers waits for that work instead of redoing it, so the setup of later
 * levels can run while an earlier level is being solved. The buffers must not change in
 * between. Not thread-safe with other calls on the same handle. */
mch_status mch_prepare_level(mch_handle *h, int level, const double *kappa,
                             const uint8_t *labels);

/* Launch shape of the 2D mixed-precision level solve (no counterpart in the paper; a GPU
 * tuning parameter). Shape 0 is the default; `count` shapes exist for the level's grid, and
 * a shape is valid when its rows per thread divide the sub-block size n / P. Results do not
 * depend on the shape beyond rounding. MCH_ERR_UNSUPPORTED for an invalid shape (and for
 * any shape other than 0 in 3D or in FP64 mode). */
mch_status mch_set_level_variant(mch_handle *h, int level, int variant);
mch_status mch_get_level_variant(const mch_handle *h, int level, int *variant, int *count);

/* Autotuner: solves `level` (as mch_solve_level, same arguments and ordering rules) once
 * with every valid launch shape, keeps the one whose level solve was fastest (CUDA events on
 * the handle's stream) and solves once more with it, so the level's results are those of a
 * plain mch_solve_level. If the environment variable MCH_TUNE_CACHE names a file, a shape
 * recorded there for the same (d, grid, P, N, precision, points) is used without timing, and
 * a newly timed choice is appended to it. `best` and `best_ms` (optional) receive the chosen
 * shape and its level-solve time (0 when taken from the cache). */
mch_status mch_autotune_level(mch_handle *h, int level, const double *kappa,
                              const uint8_t *labels, int *best, double *best_ms);

/* Gradient of a scalar loss of the effective coefficients with respect to kappa of every
 * element of every point of every level (adjoint of the constrained solves and of the
 * interpolation, derived from the energy form of Eq. phi_abstract). dL_dE[n-1] points to
 * [n_points][R][R] FP64, dL_dkappa[n-1] to [n_points][n^d] FP64 (host or device), for
 * n = 1..L. Requires every level solved; with keep_parents = 0 the cell functions are
 * recomputed from the level-grid solutions first. */
mch_status mch_backward(mch_handle *h, const double *const *dL_dE, double *const *dL_dkappa);

/* Source densities of the macroscopic problem (Sec. 2, Eq. Bs_defi, b_j / |K_p|, with the
 * source of the numerical examples of Sec. 5) for every point of `level`:
 *   fbar[p][j] = (1/|R_p|) int_{R_p} f phi_j,  j < N (the constant cell functions),
 *   f(x) = weights[j] exp(-alpha |x - center|^2) in continuum j,
 * f sampled at the centroids of the level-1-grid elements of the point's RVE at global
 * positions x = x_p + y, x_p = origin + (macro index) * spacing (the element's continuum is
 * that of the level-n element containing it); the integral is exact for this piecewise-
 * constant f and the Q1 phi_j. weights [N], center [d], origin [d]: host memory. fbar
 * [n_points][N] FP64, host or device. Requires the level solved; with keep_parents = 0 the
 * cell functions are recomputed first. R_p follows mch_desc.overs. */
mch_status mch_macro_source(mch_handle *h, int level, const double *weights,
                            const double *center, double alpha, const double *origin,
                            double spacing, double *fbar);

/* Macroscopic multicontinuum solve (Sec. 2, Eq. macro_eq): the coarse blocks
 * K_p = x_p + [-H/2, H/2]^d (H = spacing) of all macropoints form the macro mesh; U_j is Q1 on
 * their (macro_n + 1)^d vertices (x fastest) with zero Dirichlet data on the outer boundary and
 *   sum_p int_{K_p} w(V)^T E_p w(U) = sum_p int_{K_p} sum_j fbar_j(p) V_j,
 * w(U) = (U_i, d_m U_i) in the order of the cell functions (r = i, r = N + i d + m), with E_p
 * and fbar_p constant on K_p and integrated exactly (2 Gauss points per axis). E[n-1] points to
 * [n_points][R][R] and fbar[n-1] to [n_points][N] of level n = 1..L (host or device; the
 * outputs of mch_effective_coeffs and mch_macro_source). U: [N][(macro_n + 1)^d] FP64, host
 * or device, boundary entries 0. FP64 Jacobi-PCG to ||r|| <= tol ||b|| (tol 0 -> 1e-12) in at
 * most max_iter iterations (0 -> 20000); iters and relres (optional, host) receive the count
 * and the final ||r|| / ||b||. MCH_ERR_NOT_CONVERGED if the tolerance is not met, and
 * MCH_ERR_BREAKDOWN if the system is not positive definite (p'Ap <= 0). */
mch_status mch_macro_solve(mch_handle *h, const double *const *E, const double *const *fbar,
                           double spacing, double tol, int max_iter, double *U, int *iters,
                           double *relres);

/* Size of the fixed device buffer used by mch_direct_noalloc (32 MiB per GPU that loads the
 * library, held until the process exits). */
#define MCH_NOALLOC_SCRATCH_BYTES (32u << 20)

/* Effective coefficients of one level without a hierarchy (every point solved directly on
 * its n_elem^2 grid, as at level 1) for n_points macropoints, computed WITHOUT ALLOCATING any
 * device memory. For callers that cannot allocate when they need the result: device memory
 * already reserved by another framework's caching allocator, a fixed memory budget fixed at
 * start-up, or a latency-sensitive path where cudaMalloc/cudaFree would synchronise the
 * device. All intermediate data lives in one library-owned buffer of
 * MCH_NOALLOC_SCRATCH_BYTES; a batch that does not fit returns MCH_ERR_OOM (about 140 KB per
 * point at n_elem = 32 and 470 KB at n_elem = 64 with two continua).
 *   kappa [n_points][n_elem^2] FP64, labels [n_points][n_elem^2] uint8: device memory.
 *   E [n_points][R][R] FP64, R = n_cont * 3: device memory, overwritten.
 *   precision MCH_MIXED or MCH_FP64; rtol as in mch_desc (0 -> 1e-8). 2D only.
 * Work is enqueued on cuda_stream (a cudaStream_t, NULL = legacy default stream), which is
 * synchronised once before returning; a stream that is being captured is refused with
 * MCH_ERR_ARG, so never call this inside a stream capture.
 * Set-up: with CUDA's lazy module loading (the default) the driver creates the buffer, and
 * loads each kernel's code, at first use on a device, so the first call on a device, and the
 * first call with another n_elem, n_cont or precision, may allocate. Make one call with the
 * sizes and precision that later calls use, while that device is current and before its
 * memory is handed to a caching allocator; every later call with them allocates nothing.
 * The buffer's device address is looked up on every call (no address is cached), so calls
 * after a cudaDeviceReset are safe.
 * Calls share the buffer: calls that overlap on the GPU (other streams, other host threads)
 * race on it.
 * The paper has no counterpart to this entry point. */
mch_status mch_direct_noalloc(int n_cont, int n_elem, int periods, double rve_len, int precision,
                              double rtol, int n_points, const double *kappa,
                              const uint8_t *labels, double *E, void *cuda_stream);

/* Releases every library-owned buffer. Safe on NULL. */
void mch_destroy(mch_handle *h);

/* Text of the last error on this handle ("" if none). */
const char *mch_last_error(const mch_handle *h);

/* Status name, e.g. "MCH_ERR_ORDER". */
const char *mch_status_name(mch_status s);

#ifdef __cplusplus
}
#endif

#endif /* MCH_H */
