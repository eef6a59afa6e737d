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

// Projected PCG sweep on the level grid: solves min 1/2 d'A d - r'd subject to Ct d = 0 for
// every (point, function) unit whose flag is 0, starting from d = 0 with the projected
// residual r stored in `vec`, and overwrites `vec` with d. T = float (mixed) or double.
template <typename T>
struct PcgArgs {
  int npts, R, n, P, N, nc, nv;
  const double *kappa;    // [pt][n*n]
  const uint8_t *labels;  // [pt][n*n]
  const T *Sinv;          // [pt][nc][nc]
  T *vec;                 // [pt][R][nv]
  const int *done;        // [pt*R] unit already converged (skip)
  int *iters;             // [pt*R] accumulated iterations
  int *status;            // [pt*R] |= 1 on breakdown
  float tol;              // stop when sqrt(rho / rho0) < tol
  int max_iter;
  int lgm, lgP;           // log2(n / P), log2(P)
};
template <typename T>
cudaError_t launch_pcg2d(const PcgArgs<T> &a, cudaStream_t st, int *launches);
bool pcg2d_supported(int n, int P, bool fp64);

// FP64 refinement step for every (point, function) unit not yet converged: folds the last
// PCG correction into x, restores the constraints exactly (x += M^-1 Ct^T S^-1 (g - Ct x)),
// forms the residual b - A x, projects it (r - Ct^T S^-1 Ct M^-1 r), measures
// rho = r'M^-1 r against the unit's first value and writes the projected residual for the
// next PCG sweep (as T_inner) unless converged.
struct PrepArgs {
  int npts, R, n, P, N, nc, nv;
  const double *kappa, *Sinv64, *minv;
  const uint8_t *labels;
  const double *g;        // [pt][nc][R] scaled targets of this level's problem
  const double *b;        // [pt][R][nv] right-hand side (null = 0)
  double *x;              // [pt][R][nv]
  double *r64;            // [pt][R][nv] scratch
  void *vec;              // [pt][R][nv] inner vector (float or double): in delta, out residual
  int inner_fp64;
  int have_delta;
  int lgm, lgP;           // log2(n / P), log2(P)
  double *rho0;           // [pt*R]
  double *ratio;          // [pt*R]
  int *done;              // [pt*R]
  double rtol;
};
cudaError_t launch_prep2d(const PrepArgs &a, cudaStream_t st);

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
