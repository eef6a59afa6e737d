// FP64 kernels of the level solve: the Q1 stencil apply on batches of vectors, the nested
// prolongation/restriction, the interpolation of parent cell functions, the fine-grid
// constraint functional and the Gram reduction of the effective coefficients. They run in
// FP64 because they either set the accuracy of the final answer (constraints, Gram sums)
// or feed it directly.
#include "common.cuh"
#include "kernels.h"

namespace mch {

namespace {

constexpr int PREP_THREADS = 512;

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

__global__ void k_restrict2d(int R, int nf, int rho, const double *yf, int nvf, double scale,
                             double *outc, int nvc) {
  const int unit = blockIdx.y;
  const int ncg = nf / rho, Wc = ncg + 1, Wf = nf + 1;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Wc * Wc) return;
  const int Kx = k % Wc, Ky = k / Wc;
  double *o = outc + (size_t)unit * nvc;
  if (Kx == 0 || Ky == 0 || Kx == ncg || Ky == ncg) {
    o[k] = 0.0;
    return;
  }
  const double *y = yf + (size_t)unit * nvf;
  const double ir = 1.0 / rho;  // exact: rho is a power of two
  double s = 0.0;
  for (int dy = -(rho - 1); dy <= rho - 1; ++dy) {
    const double wy = 1.0 - abs(dy) * ir;
    const int fy = Ky * rho + dy;
    double sx = 0.0;
    for (int dx = -(rho - 1); dx <= rho - 1; ++dx)
      sx += (1.0 - abs(dx) * ir) * y[(Kx * rho + dx) + Wf * fy];
    s += wy * sx;
  }
  o[k] = scale * s;
}

__global__ void k_prolong_add2d(int nf, int rho, const double *xc, int nvc, double *phif, int nvf) {
  const int unit = blockIdx.y;
  const int ncg = nf / rho, Wc = ncg + 1, Wf = nf + 1;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Wf * Wf) return;
  const int fx = k % Wf, fy = k / Wf;
  const int bx = min(fx / rho, ncg - 1), by = min(fy / rho, ncg - 1);
  const double ir = 1.0 / rho;  // exact: rho is a power of two
  const double tx = (fx - bx * rho) * ir, ty = (fy - by * rho) * ir;
  const double *x = xc + (size_t)unit * nvc;
  const double v = (1 - tx) * (1 - ty) * x[bx + Wc * by] + tx * (1 - ty) * x[bx + 1 + Wc * by] +
                   (1 - tx) * ty * x[bx + Wc * (by + 1)] + tx * ty * x[bx + 1 + Wc * (by + 1)];
  phif[(size_t)unit * nvf + k] += v;
}

__global__ void k_interp(int R, int nvf, int slots, const double *const *par_ptr,
                         const double *par_w, double *I) {
  const int unit = blockIdx.y;
  const int pt = unit / R, r = unit % R;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nvf) return;
  double s = 0.0;
  for (int t = 0; t < slots; ++t) {
    const double w = par_w[pt * slots + t];
    if (w != 0.0) s += w * par_ptr[pt * slots + t][(size_t)r * nvf + k];
  }
  I[(size_t)unit * nvf + k] = s;
}

// Fine-grid constraint functional with labels prolonged from the coarse grid.
__global__ void __launch_bounds__(PREP_THREADS)
    k_ctapply2d(int R, int nf, int rho, int lgmf, int lgP, int N, int nc,
                const uint8_t *labels_c, const double *v, int nvf, const double *G, double s,
                double *g) {
  const int unit = blockIdx.x;
  const int pt = unit / R, r = unit % R;
  const int ncg = nf / rho;
  const uint8_t *lc = labels_c + (size_t)pt * ncg * ncg;
  const double *vv = v + (size_t)unit * nvf;
  __shared__ double bins[MCH_MAX_NC];
  for (int t = threadIdx.x; t < nc; t += PREP_THREADS) bins[t] = 0.0;
  __syncthreads();
  // fine labels as a lookup into the coarse array
  struct FineLab {
    const uint8_t *lc;
    int ncg, rho, nf;
    __device__ uint8_t operator[](int e) const {
      const int ex = e % nf, ey = e / nf;
      return lc[(ex / rho) + ncg * (ey / rho)];
    }
  } fl{lc, ncg, rho, nf};
  // ct_accumulate wants a pointer-like label source; expand it here
  {
    const int n = nf;
    const int tid = threadIdx.x;
    const int c = tid % n, gg = tid / n;
    const int RG = PREP_THREADS / n;
    const int rpt = (n - 1 + RG - 1) / RG;
    const bool col_active = c < n - 1;
    const int kx = c + 1, cE = c + 1 <= n - 1 ? c + 1 : n - 1;
    double acc[MCH_MAX_CONT] = {0, 0, 0, 0};
    Strip st;
    st.init(n, lgmf, lgP, c, gg * rpt, 1);
    for (int i = 0; i < rpt; ++i) {
      const int ky = 1 + gg * rpt + i;
      if (col_active && ky <= n - 1)
        scatter_node(st, ky, fl[c + n * (ky - 1)], fl[cE + n * (ky - 1)], fl[c + n * ky],
                     fl[cE + n * ky], vv[kx + (n + 1) * ky], acc, bins);
      const int kyn = ky + 1;
      if (i == rpt - 1 || ((kyn - 1) >> lgmf) != ((ky - 1) >> lgmf)) {
        flush_acc(st, acc, N, bins, true);
#pragma unroll
        for (int j = 0; j < MCH_MAX_CONT; ++j) acc[j] = 0.0;
        st.init(n, lgmf, lgP, c, kyn - 1, 1);
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nc; t += PREP_THREADS)
    g[((size_t)pt * nc + t) * R + r] = G[((size_t)pt * nc + t) * R + r] - s * bins[t];
}

constexpr int GRAM_THREADS = 256;
constexpr int GRAM_CHUNK = 16;

__global__ void __launch_bounds__(GRAM_THREADS)
    k_gram(int R, int nv, const double *X, const double *Y, double alpha, double beta, double *E) {
  const int pt = blockIdx.x;
  const int chunk = blockIdx.y;
  const int npairs = R * (R + 1) / 2;
  const int p0 = chunk * GRAM_CHUNK;
  int pr[GRAM_CHUNK], ps_[GRAM_CHUNK];
  int cnt = 0;
  {
    int idx = 0;
    for (int r = 0; r < R; ++r)
      for (int s = r; s < R; ++s, ++idx)
        if (idx >= p0 && idx < p0 + GRAM_CHUNK) {
          pr[idx - p0] = r;
          ps_[idx - p0] = s;
        }
    cnt = min(GRAM_CHUNK, npairs - p0);
  }
  double acc[GRAM_CHUNK];
#pragma unroll
  for (int i = 0; i < GRAM_CHUNK; ++i) acc[i] = 0.0;
  const double *Xp = X + (size_t)pt * R * nv;
  const double *Yp = Y + (size_t)pt * R * nv;
  for (int k = threadIdx.x; k < nv; k += GRAM_THREADS) {
#pragma unroll
    for (int i = 0; i < GRAM_CHUNK; ++i) {
      if (i < cnt) {
        const int r = pr[i], s = ps_[i];
        acc[i] += Xp[(size_t)r * nv + k] * Yp[(size_t)s * nv + k] +
                  Yp[(size_t)r * nv + k] * Xp[(size_t)s * nv + k];
      }
    }
  }
  __shared__ double red[GRAM_THREADS / 32][GRAM_CHUNK];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < GRAM_CHUNK; ++i) {
    const double v = warp_sum(acc[i]);
    if (lane == 0) red[w][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double s = 0.0;
    for (int ww = 0; ww < GRAM_THREADS / 32; ++ww) s += red[ww][threadIdx.x];
    const int r = pr[threadIdx.x], c = ps_[threadIdx.x];
    double *Ep = E + (size_t)pt * R * R;
    const double v = 0.5 * alpha * s;
    Ep[r * R + c] = beta * Ep[r * R + c] + v;
    if (c != r) Ep[c * R + r] = beta * Ep[c * R + r] + v;
  }
}

}  // namespace

cudaError_t launch_apply2d(const ApplyArgs &a, cudaStream_t st) {
  const int W = a.n + 1;
  dim3 grid((W * W + 255) / 256, a.npts * a.R);
  k_apply2d<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_restrict2d(int npts, int R, int nf, int rho, const double *yf, int nvf,
                              double scale, double *outc, int nvc, cudaStream_t st) {
  const int Wc = nf / rho + 1;
  dim3 grid((Wc * Wc + 255) / 256, npts * R);
  k_restrict2d<<<grid, 256, 0, st>>>(R, nf, rho, yf, nvf, scale, outc, nvc);
  return cudaGetLastError();
}

cudaError_t launch_prolong_add2d(int npts, int R, int nf, int rho, const double *xc, int nvc,
                                 double *phif, int nvf, cudaStream_t st) {
  const int Wf = nf + 1;
  dim3 grid((Wf * Wf + 255) / 256, npts * R);
  k_prolong_add2d<<<grid, 256, 0, st>>>(nf, rho, xc, nvc, phif, nvf);
  return cudaGetLastError();
}

cudaError_t launch_interp(int npts, int R, int nvf, int slots, const double *const *par_ptr,
                          const double *par_w, double *I, cudaStream_t st) {
  dim3 grid((nvf + 255) / 256, npts * R);
  k_interp<<<grid, 256, 0, st>>>(R, nvf, slots, par_ptr, par_w, I);
  return cudaGetLastError();
}

cudaError_t launch_ctapply2d(int npts, int R, int nf, int rho, int P, int N, int nc,
                             const uint8_t *labels_c, const double *v, int nvf,
                             const double *G, double s, double *g, cudaStream_t st) {
  int lgP = 0, lgmf = 0;
  while ((1 << (lgP + 1)) <= P) ++lgP;
  while ((1 << (lgmf + 1)) <= nf / P) ++lgmf;
  k_ctapply2d<<<npts * R, PREP_THREADS, 0, st>>>(R, nf, rho, lgmf, lgP, N, nc, labels_c, v, nvf,
                                                  G, s, g);
  return cudaGetLastError();
}

cudaError_t launch_gram(int npts, int R, int nv, const double *X, const double *Y,
                        double alpha, double beta, double *E, cudaStream_t st) {
  const int npairs = R * (R + 1) / 2;
  dim3 grid(npts, (npairs + GRAM_CHUNK - 1) / GRAM_CHUNK);
  k_gram<<<grid, GRAM_THREADS, 0, st>>>(R, nv, X, Y, alpha, beta, E);
  return cudaGetLastError();
}

}  // namespace mch
