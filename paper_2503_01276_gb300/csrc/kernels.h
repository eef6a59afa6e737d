// Kernel launch interfaces (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mch {

struct SetupArgs {
  int npts, n, P, N, R, nc;
  double h, len;
  const double *kappa;    // [pt][n*n]
  const uint8_t *labels;  // [pt][n*n]
  double *G;              // [pt][nc][R] scaled targets
  double *Sinv64;         // [pt][nc][nc]
  float *Sinv32;          // [pt][nc][nc] or null
  int *status;            // [pt] bit0 kappa, bit1 label, bit2 singular S, bit3 absent continuum
  int *dropped;           // [pt]
  double *minv;           // [pt][nv] 1 / diag(A) at interior nodes (0 elsewhere)
  int nv;
  double *Sacc;           // [pt][nc][nc] scratch accumulator of S
  double *bacc;           // [pt][nc][d+1] scratch: element count, centroid sums per row
  float *kap32;           // 3D only: [pt][n^3] FP32 copy of kappa, or null
  float *minv32;          // 3D only: [pt][nv] FP32 copy of M^-1, or null
  int overs;              // 2D: centroids over the central (P - 2 overs)^2 periods
};
cudaError_t launch_setup2d(const SetupArgs &a, cudaStream_t st);
cudaError_t launch_setup3d(const SetupArgs &a, cudaStream_t st);

// Persistent level solve (k_level.cuh): for every (point, function) unit, FP64 refinement
// steps around inner projected-PCG sweeps, all on chip; writes the FP64 solution x.
template <typename T>
struct LevelArgs {
  int npts, R, n, P, N, nc, nv, lgm, lgP;
  const double *kappa;    // [pt][n*n]
  const uint8_t *labels;  // [pt][n*n]
  const T *Sinv;          // [pt][nc][nc] inner precision
  const double *Sinv64;   // [pt][nc][nc]
  const double *minv64;   // [pt][nv]
  const double *g;        // [pt][nc][R] scaled targets of this level's problem
  const double *b;        // [pt][R][nv] right-hand side (null = 0)
  double *x;              // [pt][R][nv] solution
  int *iters, *sweeps;    // [pt*R]
  double *ratio;          // [pt*R] final sqrt(rho / rho_first) of the FP64 projected residual
  int *status;            // [pt*R] 1 = breakdown
  float tol;              // inner sweep tolerance
  int max_iter;           // inner iterations per sweep
  double rtol;            // refinement tolerance
  int max_refine;         // inner sweeps
  double *lam;            // [pt*R][nc] final multipliers (b - A x = Ct^T lam), or null
  const double *bnorm;    // [pt*R] b'M^-1 b (reference floor of the stopping test), or null
  int variant;            // launch shape (0 = default; see level2d_variant_ok)
  double *r64;            // [pt*R][nv] scratch for the FP64 residual of shapes that cannot
                          // keep it in shared memory (else it is formed twice per step), or
                          // null
};
template <typename T>
cudaError_t launch_level2d(const LevelArgs<T> &a, cudaStream_t st);
bool level2d_supported(int n, int P, bool fp64);
// Alternative launch shapes of the FP32-inner 2D level kernel (k_level_f32_alt.cu): number
// of shapes for grid n (including the default, index 0), whether shape v is valid for
// (n, P), and the launcher for v >= 1.
int level2d_variant_count(int n, bool fp64);
bool level2d_variant_ok(int n, int P, bool fp64, int v);
cudaError_t launch_level2d_alt(const LevelArgs<float> &a, cudaStream_t st);
// Chebyshev steps of the preconditioner of launch shape v (1 = Jacobi): every PCG iteration
// applies the stencil this many times (k_level.cuh).
int level2d_cheb_steps(int n, bool fp64, int v);

// y = A(kappa) x + cb * b on an n-grid whose kappa lives on the (n/rho)-grid (piecewise
// constant), for a batch of vectors; FP64.
struct ApplyArgs {
  int npts, R, n, rho, nv;
  const double *kappa;    // [pt][(n/rho)^2]
  const double *x;        // [pt][R][nv]
  const double *b;        // [pt][R][nv] or null
  double cb;
  double *y;              // [pt][R][nv]
};
cudaError_t launch_apply2d(const ApplyArgs &a, cudaStream_t st);

// out[pt][e] = kappa[pt][e] on elements of the central (P - 2 overs)^d periods, else 0.
cudaError_t launch_mask_region(int dim, int npts, int n, int P, int overs, const double *kappa,
                               double *out, cudaStream_t st);

// out[unit] = sum_k b[unit][k]^2 minv[pt][k] over nv entries (units = npts * R), FP64.
cudaError_t launch_bnorm(int npts, int R, int nv, const double *b, const double *minv,
                         double *out, cudaStream_t st);

// Level-1-grid vectors are FP64, or float-float planes (ff.cuh) when `ffs` is set.

// out_coarse = scale * P^T y_fine (restriction by the transpose of the nested bilinear
// prolongation), coarse grid n_c = n_f / rho, rho in {2, 4, 8}; out is FP64.
cudaError_t launch_restrict2d(int npts, int R, int nf, int rho, const double *yf, int nvf,
                              double scale, double *outc, int nvc, cudaStream_t st,
                              bool ffs = false);

// phi_fine += P x_coarse (x FP64), rho in {2, 4, 8}.
cudaError_t launch_prolong_add2d(int npts, int R, int nf, int rho, const double *xc, int nvc,
                                 double *phif, int nvf, cudaStream_t st, bool ffs = false);

// `count` vectors: FP64 (stride nvs) -> float-float planes (stride nvd; entries >= len are 0),
// and float-float planes (stride nvs) -> FP64 (stride nvd, first len entries).
cudaError_t launch_to_ff(int count, const double *src, int nvs, double *dst, int nvd, int len,
                         cudaStream_t st);
cudaError_t launch_from_ff(int count, const double *src, int nvs, double *dst, int nvd, int len,
                           cudaStream_t st);

// Fine-grid work of a child level (k_child.cu): I = sum_t w_t Phi_t into phi, y = A_1 I, and
// g -= s * C_1 I (g holds the targets on entry).
struct ChildArgs {
  int npts, R, nf, lgr, nvf, slots, lgmf, P, N, nc;   // P sub-blocks per side, mf = 2^lgmf
  const double *const *par_ptr;   // [pt][slots] parent cell functions (R vectors each)
  const double *par_w;            // [pt][slots]
  const double *kappa_c;          // [pt][(nf >> lgr)^2]
  const uint8_t *labels_c;        // [pt][(nf >> lgr)^2]
  double *phi;                    // [pt][R][nvf]
  double *y;                      // [pt][R][nvf]
  double *g;                      // [pt][nc][R]
  double s;                       // rho^-2
  double *yR;                     // 2D oversampling: A_1 I with kappa zero outside R_p, or null
  int overs;
  const double *kappa_ff;         // float-float planes of kappa_c (float-float storage), or null
};
cudaError_t launch_child_fine2d(const ChildArgs &a, bool ffs, cudaStream_t st);

// E[pt][r][s] += alpha * 1/2 sum_k (X_r Y_s + Y_r X_s), R in {3, 4, 6, 8, 9, 12}; with sym
// (Y = A X for a symmetric A, so the two terms agree) as alpha * sum_k X_r Y_s.
cudaError_t launch_gram(int npts, int R, int nv, const double *X, const double *Y,
                        double alpha, double *E, cudaStream_t st, bool ffs = false,
                        bool sym = false);

// ---------------------------------------------------------------------------------------
// Macroscopic problem (k_macro.cu)

constexpr int MCH_MACRO_MAXN = 4;

struct MacroSourceArgs {
  int npts, dim, N, R, nf, lgr, nvf, P, overs;
  const double *phi;       // [pts][R][nvf] cell functions on the level-1 lattice
  const uint8_t *labels;   // [pts][(nf >> lgr)^d] level-n labels
  const double *xp;        // [pts][dim] macropoint positions
  double rve_len, alpha;
  double w[MCH_MACRO_MAXN];  // source weight per continuum
  double c[3];             // centre of the Gaussian
  double *fbar;            // [pts][N]
};
cudaError_t launch_macro_source(const MacroSourceArgs &a, bool ffs, cudaStream_t st);
// Eg[elem[p]] = E[p], fg[elem[p]] = fbar[p]
cudaError_t launch_macro_gather(int npts, int R, int N, const int *elem, const double *E,
                                const double *fbar, double *Eg, double *fg, cudaStream_t st);

struct MacroSolveArgs {
  int dim, M, N, R, max_iter;
  double H, tol;
  const double *E;   // [M^d][R][R] coefficient densities of the blocks (macro order)
  const double *f;   // [M^d][N] source densities
  double *U, *r, *p, *q, *diag;   // [N][(M+1)^d] solution and work vectors
  int *iters;
  double *relres;
};
cudaError_t launch_macro_cg(const MacroSolveArgs &a, cudaStream_t st);

// ---------------------------------------------------------------------------------------
// 3D (k3d.cuh conventions: (n+1)^3 lattice, nv = nv3_of(n))

// Persistent cooperative level solve (k_level3d.cu). Vectors stream through global memory;
// x and d must be zero and p must have zero boundary entries on entry.
template <typename T>
struct Level3Args {
  int npts, R, n, P, N, nc, nv, m;
  const double *kappa;    // [pt][n^3]
  const T *kapT;          // [pt][n^3] inner-precision kappa
  const uint8_t *labels;  // [pt][n^3]
  const T *SinvT;         // [pt][nc][nc]
  const double *Sinv64;   // [pt][nc][nc]
  const double *minv64;   // [pt][nv]
  const T *minvT;         // [pt][nv]
  const double *g;        // [pt][nc][R]
  const double *b;        // [unit][nv] or null
  double *x;              // [unit][nv]
  double *r64;            // [unit][nv] scratch
  T *p, *r, *d, *q;       // [unit][nv] scratch
  double *acc;            // [3][unit][8 + 2 nc] scratch, zero on entry
  int *cnt;               // [3] scratch, zero on entry
  int *iters, *sweeps;    // [unit]
  double *ratio;          // [unit]
  int *status;            // [unit]
  float tol;
  int max_iter;
  double rtol;
  int max_refine;
  double *lam;            // [unit][nc] or null
  double h;
  long long cols_per_cta; // set by the launcher
  int kmax;               // set by the launcher
  const double *bnorm;    // [unit] b'M^-1 b (reference floor of the stopping test), or null
};
template <typename T>
cudaError_t launch_level3d(const Level3Args<T> &a, cudaStream_t st);

// y = A(kappa_c prolonged) x + cb * b on an n-grid, kappa on the (n / rho)-grid.
cudaError_t launch_apply3d(const ApplyArgs &a, double h, cudaStream_t st);
// Level-1-grid vectors in FP64 or, with ffs, float-float planes (ff.cuh).
// phi[pt][r] = sum_t w_t Phi_t[r] on the level-1 lattice.
cudaError_t launch_interp3d(const ChildArgs &a, cudaStream_t st, bool ffs);
// y = A_1 phi (child kappa prolonged to the level-1 grid) and g -= s * C_1 phi.
cudaError_t launch_fine_apply3d(const ChildArgs &a, double hf, cudaStream_t st, bool ffs);
cudaError_t launch_restrict3d(int npts, int R, int nf, int rho, const double *yf, int nvf,
                              double scale, double *outc, int nvc, cudaStream_t st, bool ffs);
cudaError_t launch_prolong_add3d(int npts, int R, int nf, int rho, const double *xc, int nvc,
                                 double *phif, int nvf, cudaStream_t st, bool ffs);

// Backward pass kernels (k_adjoint.cu).
struct AdjArgs {
  int npts, R, nf, lgr, nvf, nvc, nc, lgmf, P, slots;  // P sub-blocks per side
  double inv_vol, inv_rho2;
  const double *W;          // [pt][R][R] dL/dE
  const double *phi;        // [pt][R][nvf] cell functions (level-1 grid)
  const double *mu;         // [pt][R][nvc] adjoint solution, or null
  const double *lam;        // [pt][R][nc] forward multipliers
  const double *lamadj;     // [pt][R][nc] adjoint multipliers, or null
  const double *kappa_c;    // [pt][ncg^2]
  const uint8_t *labels_c;  // [pt][ncg^2]
  const double *V;          // [pt][R][nvf] seeds of this level, or null
  double *psi1, *psi2;      // [pt][R][nvf] scratch
  double *dkappa;           // [pt][ncg^2]
  double *const *par_V;     // [pt][slots] parents' seed blocks
  const double *par_w;      // [pt][slots]
  int ffs;                  // phi stored as float-float planes
  int overs;                // > 0: E over R_p (central (P - 2 overs)^2 periods); the own term
                            // is an adjoint source (k_adj_own2d), no envelope terms
};
cudaError_t launch_adj_combine2d(const AdjArgs &a, cudaStream_t st);
cudaError_t launch_adj_grad2d(const AdjArgs &a, cudaStream_t st);
cudaError_t launch_adj_seed2d(const AdjArgs &a, cudaStream_t st);
// V[pt][r] += sum_s What_rs A_{1,R} Phi_s on the level-1 grid (oversampling only).
cudaError_t launch_adj_own2d(const AdjArgs &a, cudaStream_t st);
cudaError_t launch_adj_combine3d(const AdjArgs &a, cudaStream_t st);
cudaError_t launch_adj_grad3d(const AdjArgs &a, double hf, cudaStream_t st);
cudaError_t launch_adj_seed3d(const AdjArgs &a, double hf, cudaStream_t st);
// V[pt][r] += sum_s What_rs A_{1,R} Phi_s on the level-1 grid (3D oversampling only).
cudaError_t launch_adj_own3d(const AdjArgs &a, double hf, cudaStream_t st);

}  // namespace mch
