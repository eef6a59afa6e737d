// Per-point constraint data for the 2D cell problems (one CTA per macropoint).
//
// Sec. 2, Eqs. (phi_avar) and (phi_grad): for continuum j and sub-block R_q the constraint
// functional is v -> int_{R_q} psi_j v and its targets are delta_ij int_{R_q} psi_j
// (constant cell function phi_i) and delta_ij int_{R_q} (x_m - c_mj) psi_j (linear cell
// function phi_i^m), with c_mj the centroid of continuum j over R_p (here the whole RVE).
// Everything is scaled by 4 / h^2 (see common.cuh): the target of row (j, q) for phi_j is
// 4 * #elements, for phi_j^m it is 4 * sum over the row's elements of (centroid_m - c_mj).
//
// The kernel also forms S = Ct M^-1 Ct^T with M = diag(A) (the Jacobi preconditioner) and
// inverts it in FP64 (Cholesky, then L^-T L^-1). S^-1 is the small dense solve of the
// constraint projection used by the PCG and by the FP64 refinement. Rows of empty
// (continuum, sub-block) pairs are decoupled with a unit diagonal, so their multiplier is 0.
#include "common.cuh"
#include "kernels.h"

namespace mch {

namespace {

constexpr int SETUP_THREADS = 512;

__global__ void __launch_bounds__(SETUP_THREADS) k_setup2d(SetupArgs a) {
  const int pt = blockIdx.x;
  const int n = a.n, P = a.P, N = a.N, R = a.R, nc = a.nc;
  const int m = n / P, nq = P * P;
  const int tid = threadIdx.x;
  const double *kap = a.kappa + (size_t)pt * n * n;
  const uint8_t *lab = a.labels + (size_t)pt * n * n;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *S = reinterpret_cast<double *>(smem_raw);      // [nc][nc]
  double *Z = S + nc * nc;                                // [nc][nc]
  double *bsy = Z + nc * nc;                              // [nc][2]
  double *bcnt = bsy + 2 * nc;                            // [nc]
  double *cen = bcnt + nc;                                // [MCH_MAX_CONT][2]
  double *dorig = cen + 2 * MCH_MAX_CONT;                 // [nc]
  __shared__ int flags;

  if (tid == 0) flags = 0;
  for (int i = tid; i < nc * nc; i += SETUP_THREADS) S[i] = 0.0;
  __syncthreads();

  // 1. validate the medium
  for (int e = tid; e < n * n; e += SETUP_THREADS) {
    const double k = kap[e];
    if (!(k > 0.0) || !(k < 1e300)) atomicOr(&flags, 1);
    if (lab[e] >= N) atomicOr(&flags, 2);
  }
  __syncthreads();
  if (flags & 3) {
    if (tid == 0) a.status[pt] = flags;
    return;
  }

  // 2. per (continuum, sub-block): element count and centroid sums; one warp per sub-block
  const int warp = tid >> 5, lane = tid & 31, nwarps = SETUP_THREADS / 32;
  for (int q = warp; q < nq; q += nwarps) {
    const int qx = q % P, qy = q / P;
    double cnt[MCH_MAX_CONT] = {0, 0, 0, 0}, sx[MCH_MAX_CONT] = {0, 0, 0, 0},
           sy[MCH_MAX_CONT] = {0, 0, 0, 0};
    for (int t = lane; t < m * m; t += 32) {
      const int ex = qx * m + t % m, ey = qy * m + t / m;
      const int l = lab[ex + n * ey];
      const double yx = -0.5 * a.len + (ex + 0.5) * a.h;
      const double yy = -0.5 * a.len + (ey + 0.5) * a.h;
      add_by_label(cnt, l, 1.0);
      add_by_label(sx, l, yx);
      add_by_label(sy, l, yy);
    }
    for (int j = 0; j < N; ++j) {
      const double c = warp_sum(cnt[j]), x = warp_sum(sx[j]), y = warp_sum(sy[j]);
      if (lane == 0) {
        bcnt[j * nq + q] = c;
        bsy[2 * (j * nq + q) + 0] = x;
        bsy[2 * (j * nq + q) + 1] = y;
      }
    }
  }
  __syncthreads();

  // 3. centroids c_mj over the whole RVE
  if (tid < N) {
    double c = 0, x = 0, y = 0;
    for (int q = 0; q < nq; ++q) {
      c += bcnt[tid * nq + q];
      x += bsy[2 * (tid * nq + q)];
      y += bsy[2 * (tid * nq + q) + 1];
    }
    if (c == 0.0) atomicOr(&flags, 8);
    cen[2 * tid] = c > 0 ? x / c : 0.0;
    cen[2 * tid + 1] = c > 0 ? y / c : 0.0;
  }
  __syncthreads();

  // 4. scaled targets G[b][r]
  double *G = a.G + (size_t)pt * nc * R;
  for (int t = tid; t < nc * R; t += SETUP_THREADS) {
    const int b = t / R, r = t % R;
    const int j = b / nq;
    double v = 0.0;
    if (r < N) {
      if (r == j) v = 4.0 * bcnt[b];
    } else {
      const int i = (r - N) / 2, mm = (r - N) % 2;
      if (i == j) v = 4.0 * (bsy[2 * b + mm] - bcnt[b] * cen[2 * j + mm]);
    }
    G[t] = v;
  }

  // M^-1 = 1 / diag(A) at interior nodes, kept for the FP64 refinement steps
  {
    double *mv = a.minv + (size_t)pt * a.nv;
    const int W = n + 1;
    for (int k = tid; k < W * W; k += SETUP_THREADS) {
      const int kx = k % W, ky = k / W;
      double v = 0.0;
      if (kx > 0 && ky > 0 && kx < n && ky < n)
        v = 1.0 / ((kap[(kx - 1) + n * (ky - 1)] + kap[kx + n * (ky - 1)] + kap[(kx - 1) + n * ky] +
                    kap[kx + n * ky]) * (2.0 / 3.0));
      mv[k] = v;
    }
  }

  // 5. S = Ct M^-1 Ct^T: per node, sum over pairs of adjacent elements of 1/diag; runs of
  // nodes with the same four adjacent rows are accumulated before the atomic flush.
  {
    const int ncol = n - 1;
    const int nstrip = SETUP_THREADS / ncol > 0 ? SETUP_THREADS / ncol : 1;
    const int rows_per = (n - 1 + nstrip - 1) / nstrip;
    for (int u = tid; u < ncol * nstrip; u += SETUP_THREADS) {
      const int kx = 1 + u % ncol, strip = u / ncol;
      const int y0 = 1 + strip * rows_per;
      const int y1 = min(n, y0 + rows_per);
      unsigned sig = 0xffffffffu;
      double acc = 0.0;
      for (int ky = y0; ky < y1; ++ky) {
        const int eSW = (kx - 1) + n * (ky - 1), eSE = kx + n * (ky - 1);
        const int eNW = (kx - 1) + n * ky, eNE = kx + n * ky;
        const int b0 = lab[eSW] * nq + ((ky - 1) / m) * P + (kx - 1) / m;
        const int b1 = lab[eSE] * nq + ((ky - 1) / m) * P + kx / m;
        const int b2 = lab[eNW] * nq + (ky / m) * P + (kx - 1) / m;
        const int b3 = lab[eNE] * nq + (ky / m) * P + kx / m;
        const unsigned key = (unsigned)b0 | ((unsigned)b1 << 8) | ((unsigned)b2 << 16) |
                             ((unsigned)b3 << 24);
        const double dg = (kap[eSW] + kap[eSE] + kap[eNW] + kap[eNE]) * (2.0 / 3.0);
        if (key != sig) {
          if (sig != 0xffffffffu) {
            int bb[4] = {int(sig & 255), int((sig >> 8) & 255), int((sig >> 16) & 255),
                         int(sig >> 24)};
            for (int e1 = 0; e1 < 4; ++e1)
              for (int e2 = 0; e2 < 4; ++e2) atomicAdd(&S[bb[e1] * nc + bb[e2]], acc);
          }
          sig = key;
          acc = 0.0;
        }
        acc += 1.0 / dg;
      }
      if (sig != 0xffffffffu) {
        int bb[4] = {int(sig & 255), int((sig >> 8) & 255), int((sig >> 16) & 255), int(sig >> 24)};
        for (int e1 = 0; e1 < 4; ++e1)
          for (int e2 = 0; e2 < 4; ++e2) atomicAdd(&S[bb[e1] * nc + bb[e2]], acc);
      }
    }
  }
  __syncthreads();
  if (tid < nc) {
    if (bcnt[tid] == 0.0) S[tid * nc + tid] = 1.0;
    dorig[tid] = S[tid * nc + tid];
  }
  __syncthreads();

  // 6. Cholesky S = L L^T in place (lower triangle)
  for (int k = 0; k < nc; ++k) {
    if (tid == 0) {
      double v = S[k * nc + k];
      if (!(v > 1e-13 * dorig[k])) {
        flags |= 4;
        v = dorig[k] > 0 ? dorig[k] : 1.0;
      }
      S[k * nc + k] = sqrt(v);
    }
    __syncthreads();
    for (int i = k + 1 + tid; i < nc; i += SETUP_THREADS) S[i * nc + k] /= S[k * nc + k];
    __syncthreads();
    const int rem = nc - k - 1;
    for (int t = tid; t < rem * rem; t += SETUP_THREADS) {
      const int i = k + 1 + t / rem, j = k + 1 + t % rem;
      if (j <= i) S[i * nc + j] -= S[i * nc + k] * S[j * nc + k];
    }
    __syncthreads();
  }

  // 7. Z = L^-1 (column j by forward substitution), then S^-1 = Z^T Z
  for (int j = tid; j < nc; j += SETUP_THREADS) {
    for (int i = 0; i < nc; ++i) {
      double v = (i == j) ? 1.0 : 0.0;
      if (i > j)
        for (int k = j; k < i; ++k) v -= S[i * nc + k] * Z[k * nc + j];
      Z[i * nc + j] = (i < j) ? 0.0 : v / S[i * nc + i];
    }
  }
  __syncthreads();
  double *Si64 = a.Sinv64 + (size_t)pt * nc * nc;
  float *Si32 = a.Sinv32 ? a.Sinv32 + (size_t)pt * nc * nc : nullptr;
  for (int t = tid; t < nc * nc; t += SETUP_THREADS) {
    const int i = t / nc, j = t % nc;
    double v = 0.0;
    for (int k = max(i, j); k < nc; ++k) v += Z[k * nc + i] * Z[k * nc + j];
    Si64[t] = v;
    if (Si32) Si32[t] = (float)v;
  }
  if (tid == 0) {
    int nd = 0;
    for (int b = 0; b < nc; ++b) nd += (bcnt[b] == 0.0);
    a.dropped[pt] = nd;
    a.status[pt] = flags;
  }
}

}  // namespace

cudaError_t launch_setup2d(const SetupArgs &a, cudaStream_t st) {
  const size_t smem = sizeof(double) * (2 * a.nc * a.nc + 4 * a.nc + 2 * MCH_MAX_CONT);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_setup2d, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_setup2d<<<a.npts, SETUP_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace mch
