// FP64 Q1 stencil apply on a batch of vectors (used for A_n Xi - 2 b before the Gram of the
// effective coefficients, Eq. Bs_defi).
#include "common.cuh"
#include "kernels.h"

namespace mch {

namespace {

__global__ void k_apply2d(ApplyArgs a) {
  const int unit = blockIdx.y;
  const int pt = unit / a.R;
  const int n = a.n, W = n + 1;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= W * W) return;
  const int kx = k % W, ky = k / W;
  double *y = a.y + (size_t)unit * a.nv;
  if (kx == 0 || ky == 0 || kx == n || ky == n) {
    y[k] = 0.0;
    return;
  }
  const int nc_ = n / a.rho;
  const double *kap = a.kappa + (size_t)pt * nc_ * nc_;
  auto K = [&](int ex, int ey) { return kap[(ex / a.rho) + nc_ * (ey / a.rho)]; };
  const double *x = a.x + (size_t)unit * a.nv;
  const double *xr = x + k;
  double v = q1_apply(K(kx - 1, ky - 1), K(kx, ky - 1), K(kx - 1, ky), K(kx, ky), xr[-W - 1],
                      xr[-W], xr[-W + 1], xr[-1], xr[0], xr[1], xr[W - 1], xr[W], xr[W + 1]);
  if (a.b) v += a.cb * a.b[(size_t)unit * a.nv + k];
  y[k] = v;
}

}  // namespace

cudaError_t launch_apply2d(const ApplyArgs &a, cudaStream_t st) {
  const int W = a.n + 1;
  dim3 grid((W * W + 255) / 256, a.npts * a.R);
  k_apply2d<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

namespace {

__global__ void __launch_bounds__(256) k_bnorm(int R, int nv, const double *b, const double *minv,
                                               double *out) {
  const int unit = blockIdx.x, pt = unit / R;
  const double *bb = b + (size_t)unit * nv;
  const double *mm = minv + (size_t)pt * nv;
  double s = 0.0;
  for (int k = threadIdx.x; k < nv; k += 256) s += bb[k] * bb[k] * mm[k];
  s = warp_sum(s);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    out[unit] = t;
  }
}

}  // namespace

namespace {

__global__ void k_mask_region(int dim, int n, int P, int overs, const double *kappa,
                              double *out) {
  const int pt = blockIdx.y;
  const long long ne = dim == 3 ? (long long)n * n * n : (long long)n * n;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int m = n / P;
  const int px = (int)(e % n) / m, py = (int)((e / n) % n) / m;
  const int pz = dim == 3 ? (int)(e / ((long long)n * n)) / m : overs;
  const bool in = px >= overs && px < P - overs && py >= overs && py < P - overs &&
                  pz >= overs && pz < P - overs;
  out[(size_t)pt * ne + e] = in ? kappa[(size_t)pt * ne + e] : 0.0;
}

}  // namespace

cudaError_t launch_mask_region(int dim, int npts, int n, int P, int overs, const double *kappa,
                               double *out, cudaStream_t st) {
  const long long ne = dim == 3 ? (long long)n * n * n : (long long)n * n;
  dim3 grid((unsigned)((ne + 255) / 256), npts);
  k_mask_region<<<grid, 256, 0, st>>>(dim, n, P, overs, kappa, out);
  return cudaGetLastError();
}

cudaError_t launch_bnorm(int npts, int R, int nv, const double *b, const double *minv,
                         double *out, cudaStream_t st) {
  k_bnorm<<<npts * R, 256, 0, st>>>(R, nv, b, minv, out);
  return cudaGetLastError();
}

}  // namespace mch
