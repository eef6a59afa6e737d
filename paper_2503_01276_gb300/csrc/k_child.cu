// Level-1-grid (fine) work of a child level and the Gram reductions, FP64.
//
// Sec. 3.3, Eqs. (PhiXiI), (phiXiI_all): a point of level n > 1 starts from the
// interpolation I = sum_t c_t Phi_t of its parents' cell functions on the level-1 grid.
// Eqs. (phi_avar_corrector), (phi_grad_corrector): its correction problem needs
//   b = -P^T A_1 I           (A_1 = level-1 stiffness of the child's medium, prolonged
//                             piecewise constantly from its level-n grid)
//   g = G - C_1 I            (constraint targets minus the constraint functionals of I)
// and its effective coefficients (Eq. Bs_defi) start from K_I = I^T A_1 I.
//
// k_child_fine2d does, per (cell function, band of fine rows): I from the parents into a
// shared-memory tile, I written as the child's cell function, y = A_1 I, and the
// band's part of C_1 I added atomically into g (which holds G on entry).
// k_gram2d reduces 1/2 sum_k (X_r Y_s + Y_r X_s) for every pair r <= s of a point with
// the pair sums in registers, adding into E.
// k_restrict2d forms b = scale * P^T y; k_prolong_add2d adds P x to the fine functions.
#include "common.cuh"
#include "kernels.h"

namespace mch {

namespace {

constexpr int CF_THREADS = 256;
constexpr int CF_BR = 16;   // fine rows per band

template <int NC>
__global__ void __launch_bounds__(CF_THREADS) k_child_fine2d(ChildArgs a) {
  const int unit = blockIdx.y;
  const int pt = unit / a.R, r = unit % a.R;
  const int nf = a.nf, W = nf + 1, lgr = a.lgr, ncg = nf >> lgr;
  const int band = blockIdx.x;
  const int row_lo = band * CF_BR;                 // first own lattice row
  const int row_hi = min(row_lo + CF_BR, nf + 1);  // one past the last own row
  __shared__ double tile[(CF_BR + 2) * 257];
  __shared__ double bins[MCH_MAX_NC];
  __shared__ const double *pp[4];
  __shared__ double pw[4];
  const int tid = threadIdx.x;
  if (tid < a.slots) {
    pw[tid] = a.par_w[pt * a.slots + tid];
    pp[tid] = a.par_ptr[pt * a.slots + tid];
  }
  for (int t = tid; t < a.nc; t += CF_THREADS) bins[t] = 0.0;
  __syncthreads();

  // I on rows row_lo-1 .. row_lo+CF_BR (rows outside the lattice are zero)
  const size_t off = (size_t)r * a.nvf;
  for (int t = tid; t < (CF_BR + 2) * W; t += CF_THREADS) {
    const int row = row_lo - 1 + t / W, col = t % W;
    double v = 0.0;
    if (row >= 0 && row <= nf) {
      const int k = col + W * row;
      for (int s = 0; s < a.slots; ++s)
        if (pw[s] != 0.0) v += pw[s] * pp[s][off + k];
    }
    tile[t] = v;
  }
  __syncthreads();

  const double *kc = a.kappa_c + (size_t)pt * ncg * ncg;
  double *phi = a.phi + (size_t)unit * a.nvf;
  double *y = a.y + (size_t)unit * a.nvf;
  for (int t = tid; t < (row_hi - row_lo) * W; t += CF_THREADS) {
    const int row = row_lo + t / W, col = t % W;
    const int k = col + W * row;
    const double *tr = tile + (row - row_lo + 1) * W + col;
    phi[k] = tr[0];
    double v = 0.0;
    if (row > 0 && row < nf && col > 0 && col < nf) {
      const int e0x = (col - 1) >> lgr, e1x = col >> lgr;
      const int e0y = (row - 1) >> lgr, e1y = row >> lgr;
      v = q1_apply(kc[e0x + ncg * e0y], kc[e1x + ncg * e0y], kc[e0x + ncg * e1y],
                   kc[e1x + ncg * e1y], tr[-W - 1], tr[-W], tr[-W + 1], tr[-1], tr[0], tr[1],
                   tr[W - 1], tr[W], tr[W + 1]);
    }
    y[k] = v;
  }

  // C_1 I on the band's element rows: element corner sums per (label, sub-block). Warp w
  // takes column chunk w % nch (32 element columns, one sub-block column or aligned
  // halves of one) and every (8 / nch)-th row.
  {
    const int warp = tid >> 5, lane = tid & 31;
    const int nch = nf >> 5;                       // nf >= 32
    const int chunk = warp % nch, rstep = (CF_THREADS / 32) / nch;
    const int ex = chunk * 32 + lane;
    const int lgm = a.lgmf, m = 1 << lgm;
    const int seg = m < 32 ? m : 32;
    const uint8_t *lc = a.labels_c + (size_t)pt * ncg * ncg;
    double acc[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[j] = 0.0;
    const int erow_hi = min(row_lo + CF_BR, nf);
    const int bx = ex >> lgm;
    auto flush = [&](int by) {
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        const double sj = seg_sum(acc[j], seg);
        if ((lane & (seg - 1)) == 0 && sj != 0.0)
          atomicAdd(&bins[(j << (2 * a.lgP)) + (by << a.lgP) + bx], sj);
        acc[j] = 0.0;
      }
    };
    // rows of one warp share ey, so the flush condition is uniform over the warp
    int by_cur = -1;
    for (int ey = row_lo + warp / nch; ey < erow_hi; ey += rstep) {
      const int by = ey >> lgm;
      if (by != by_cur) {
        if (by_cur >= 0) flush(by_cur);
        by_cur = by;
      }
      const double *tr = tile + (ey - row_lo + 1) * W + ex;
      const double sv = tr[0] + tr[1] + tr[W] + tr[W + 1];
      const int l = lc[(ex >> lgr) + ncg * (ey >> lgr)];
#pragma unroll
      for (int j = 0; j < NC; ++j) acc[j] += (l == j) ? sv : 0.0;
    }
    if (by_cur >= 0) flush(by_cur);
  }
  __syncthreads();
  for (int t = tid; t < a.nc; t += CF_THREADS)
    if (bins[t] != 0.0) atomicAdd(&a.g[((size_t)pt * a.nc + t) * a.R + r], -a.s * bins[t]);
}

constexpr int GR_THREADS = 256;

template <int R>
__global__ void __launch_bounds__(GR_THREADS) k_gram2d(int nv, int slices, const double *X,
                                                        const double *Y, double alpha, double *E) {
  constexpr int NP = R * (R + 1) / 2;
  const int pt = blockIdx.x;
  const int per = (nv + slices - 1) / slices;
  const int k0 = blockIdx.y * per, k1 = min(nv, k0 + per);
  double acc[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) acc[p] = 0.0;
  const double *Xp = X + (size_t)pt * R * nv;
  const double *Yp = Y + (size_t)pt * R * nv;
  for (int k = k0 + threadIdx.x; k < k1; k += GR_THREADS) {
    double xv[R], yv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      xv[r] = Xp[(size_t)r * nv + k];
      yv[r] = Yp[(size_t)r * nv + k];
    }
    int p = 0;
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int s = r; s < R; ++s, ++p) acc[p] += xv[r] * yv[s] + yv[r] * xv[s];
  }
  __shared__ double red[GR_THREADS / 32][NP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const double v = warp_sum(acc[p]);
    if (lane == 0) red[w][p] = v;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < NP; p += GR_THREADS) {
    double s = 0.0;
    for (int ww = 0; ww < GR_THREADS / 32; ++ww) s += red[ww][p];
    int rr = 0, cc = 0, q = p;
    while (q >= R - rr) { q -= R - rr; ++rr; }
    cc = rr + q;
    double *Ep = E + (size_t)pt * R * R;
    const double v = 0.5 * alpha * s;
    atomicAdd(&Ep[rr * R + cc], v);
    if (cc != rr) atomicAdd(&Ep[cc * R + rr], v);
  }
}

template <int RHO>
__global__ void k_restrict2d(int nf, const double *yf, int nvf, double scale, double *outc,
                             int nvc) {
  const int unit = blockIdx.y;
  const int ncg = nf / RHO, Wc = ncg + 1, Wf = nf + 1;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Wc * Wc) return;
  const int Kx = k % Wc, Ky = k / Wc;
  double *o = outc + (size_t)unit * nvc;
  if (Kx == 0 || Ky == 0 || Kx == ncg || Ky == ncg) {
    o[k] = 0.0;
    return;
  }
  const double *y = yf + (size_t)unit * nvf + (size_t)(Ky * RHO) * Wf + Kx * RHO;
  double s = 0.0;
#pragma unroll
  for (int dy = -(RHO - 1); dy <= RHO - 1; ++dy) {
    double sx = 0.0;
#pragma unroll
    for (int dx = -(RHO - 1); dx <= RHO - 1; ++dx)
      sx += double(RHO - (dx < 0 ? -dx : dx)) * y[dy * Wf + dx];
    s += double(RHO - (dy < 0 ? -dy : dy)) * sx;
  }
  o[k] = scale * s * (1.0 / (RHO * RHO));
}

// One thread per coarse cell: the cell's RHO x RHO fine nodes (lower-left corner included)
// get the bilinear interpolant of the cell's four coarse values.
template <int RHO>
__global__ void k_prolong_add2d(int nf, const double *xc, int nvc, double *phif, int nvf) {
  const int unit = blockIdx.y;
  const int ncg = nf / RHO, Wc = ncg + 1, Wf = nf + 1;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= ncg * ncg) return;
  const int Kx = cell % ncg, Ky = cell / ncg;
  const double *x = xc + (size_t)unit * nvc + Kx + Wc * Ky;
  const double x00 = x[0], x10 = x[1], x01 = x[Wc], x11 = x[Wc + 1];
  double *f = phif + (size_t)unit * nvf + (size_t)(Ky * RHO) * Wf + Kx * RHO;
  const double dl = x01 - x00, dr = x11 - x10;
#pragma unroll
  for (int j = 0; j < RHO; ++j) {
    const double ty = double(j) * (1.0 / RHO);
    const double aj = x00 + ty * dl, bj = x10 + ty * dr;
    const double dj = bj - aj;
#pragma unroll
    for (int i = 0; i < RHO; ++i) f[j * Wf + i] += aj + double(i) * (1.0 / RHO) * dj;
  }
}

}  // namespace

cudaError_t launch_child_fine2d(const ChildArgs &a, cudaStream_t st) {
  if (a.nf < 32 || a.nf > 256) return cudaErrorInvalidValue;
  dim3 grid((a.nf + 1 + CF_BR - 1) / CF_BR, a.npts * a.R);
  if (a.N <= 2) k_child_fine2d<2><<<grid, CF_THREADS, 0, st>>>(a);
  else if (a.N == 3) k_child_fine2d<3><<<grid, CF_THREADS, 0, st>>>(a);
  else k_child_fine2d<4><<<grid, CF_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gram(int npts, int R, int nv, const double *X, const double *Y,
                        double alpha, double *E, cudaStream_t st) {
  int slices = nv >= 8192 ? 8 : (nv >= 2048 ? 4 : 1);
  if (nv > 100000) {
    // 3D level-1 lattices: enough slices for every SM when the level has few points
    const int want = (4 * 152 + npts - 1) / npts;
    slices = want < 8 ? 8 : (want > nv / 4096 ? nv / 4096 : want);
  }
  dim3 grid(npts, slices);
  switch (R) {
    case 3: k_gram2d<3><<<grid, GR_THREADS, 0, st>>>(nv, slices, X, Y, alpha, E); break;
    case 4: k_gram2d<4><<<grid, GR_THREADS, 0, st>>>(nv, slices, X, Y, alpha, E); break;
    case 8: k_gram2d<8><<<grid, GR_THREADS, 0, st>>>(nv, slices, X, Y, alpha, E); break;
    case 6: k_gram2d<6><<<grid, GR_THREADS, 0, st>>>(nv, slices, X, Y, alpha, E); break;
    case 9: k_gram2d<9><<<grid, GR_THREADS, 0, st>>>(nv, slices, X, Y, alpha, E); break;
    case 12: k_gram2d<12><<<grid, GR_THREADS, 0, st>>>(nv, slices, X, Y, alpha, E); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_restrict2d(int npts, int R, int nf, int rho, const double *yf, int nvf,
                              double scale, double *outc, int nvc, cudaStream_t st) {
  const int Wc = nf / rho + 1;
  dim3 grid((Wc * Wc + 255) / 256, npts * R);
  switch (rho) {
    case 2: k_restrict2d<2><<<grid, 256, 0, st>>>(nf, yf, nvf, scale, outc, nvc); break;
    case 4: k_restrict2d<4><<<grid, 256, 0, st>>>(nf, yf, nvf, scale, outc, nvc); break;
    case 8: k_restrict2d<8><<<grid, 256, 0, st>>>(nf, yf, nvf, scale, outc, nvc); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_prolong_add2d(int npts, int R, int nf, int rho, const double *xc, int nvc,
                                 double *phif, int nvf, cudaStream_t st) {
  const int ncg = nf / rho;
  dim3 grid((ncg * ncg + 127) / 128, npts * R);
  switch (rho) {
    case 2: k_prolong_add2d<2><<<grid, 128, 0, st>>>(nf, xc, nvc, phif, nvf); break;
    case 4: k_prolong_add2d<4><<<grid, 128, 0, st>>>(nf, xc, nvc, phif, nvf); break;
    case 8: k_prolong_add2d<8><<<grid, 128, 0, st>>>(nf, xc, nvc, phif, nvf); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace mch
