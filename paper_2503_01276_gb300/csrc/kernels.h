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
};
cudaError_t launch_setup2d(const SetupArgs &a, cudaStream_t st);

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
};
template <typename T>
cudaError_t launch_level2d(const LevelArgs<T> &a, cudaStream_t st);
bool level2d_supported(int n, int P, bool fp64);

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

// out_coarse = scale * P^T y_fine (restriction by the transpose of the nested bilinear
// prolongation), coarse grid n_c = n_f / rho.
cudaError_t launch_restrict2d(int npts, int R, int nf, int rho, const double *yf, int nvf,
                              double scale, double *outc, int nvc, cudaStream_t st);

// phi_fine += P x_coarse.
cudaError_t launch_prolong_add2d(int npts, int R, int nf, int rho, const double *xc, int nvc,
                                 double *phif, int nvf, cudaStream_t st);

// I[pt][r] = sum_t w[pt][t] Phi_{parent t}[r] on the fine lattice.
cudaError_t launch_interp(int npts, int R, int nvf, int slots, const double *const *par_ptr,
                          const double *par_w, double *I, cudaStream_t st);

// g[pt][b][r] = G[pt][b][r] - s * (Ct_fine v)[b] with the fine-grid constraint rows of the
// labels prolonged from the coarse grid (n_c = n_f / rho).
cudaError_t launch_ctapply2d(int npts, int R, int nf, int rho, int P, int N, int nc,
                             const uint8_t *labels_c, const double *v, int nvf,
                             const double *G, double s, double *g, cudaStream_t st);

// E[pt][r][s] = beta * E + alpha * 1/2 sum_k (X_r Y_s + Y_r X_s).
cudaError_t launch_gram(int npts, int R, int nv, const double *X, const double *Y,
                        double alpha, double beta, double *E, cudaStream_t st);

}  // namespace mch
