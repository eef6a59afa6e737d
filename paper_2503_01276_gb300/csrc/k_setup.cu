// Per-point constraint data for the 2D cell problems.
//
// Sec. 2, Eqs. (phi_avar) and (phi_grad): for continuum j and sub-block R_q the constraint
// functional is v -> int_{R_q} psi_j v and its targets are delta_ij int_{R_q} psi_j
// (constant cell function phi_i) and delta_ij int_{R_q} (x_m - c_mj) psi_j (linear cell
// function phi_i^m), with c_mj the centroid of continuum j over R_p (here the whole RVE).
// Everything is scaled by 4 / h^2 (see common.cuh): the target of row (j, q) for phi_j is
// 4 * #elements, for phi_j^m it is 4 * sum over the row's elements of (centroid_m - c_mj).
//
// The setup also forms S = Ct M^-1 Ct^T with M = diag(A) (the Jacobi preconditioner) and
// inverts it in FP64 (Gauss-Jordan). S^-1 is the small dense solve of the
// constraint projection used by the PCG and by the FP64 refinement. Rows of empty
// (continuum, sub-block) pairs are decoupled with a unit diagonal, so their multiplier is 0.
//
// Two kernels: k_setup_nodes runs on (point, slice of node rows) and writes M^-1 and adds
// its part of S and of the per-(continuum, sub-block) element counts and centroid sums to
// zero-initialised accumulators; k_setup_point (one CTA per point) forms the targets and
// the inverse. M^-1 is an FP32 reciprocal refined by two FP64 Newton steps (a preconditioner
// only needs a fixed positive diagonal; S and every later use read the same stored value).
#include "common.cuh"
#include "kernels.h"

namespace mch {

namespace {

constexpr int SN_THREADS = 256;

__device__ __forceinline__ double fast_rcp(double d) {
  double y = (double)(1.0f / (float)d);
  y = y * (2.0 - d * y);
  y = y * (2.0 - d * y);
  return y;
}

__global__ void __launch_bounds__(SN_THREADS) k_setup_nodes(SetupArgs a, int slices) {
  const int pt = blockIdx.x, slice = blockIdx.y;
  const int n = a.n, P = a.P, N = a.N, nc = a.nc;
  const int m = n / P, nq = P * P;
  const int tid = threadIdx.x;
  const double *kap = a.kappa + (size_t)pt * n * n;
  const uint8_t *lab = a.labels + (size_t)pt * n * n;
  // node rows [y0, y1) of the lattice and element rows [y0, y1) ∩ [0, n)
  const int per = (n + 1 + slices - 1) / slices;
  const int y0 = slice * per, y1 = min(n + 1, y0 + per);
  __shared__ double S[MCH_MAX_NC * MCH_MAX_NC];
  __shared__ int bsi[MCH_MAX_NC * 3];   // element count, sum of ex, sum of ey per row
  __shared__ int flags;
  if (tid == 0) flags = 0;
  for (int i = tid; i < nc * nc; i += SN_THREADS) S[i] = 0.0;
  for (int i = tid; i < nc * 3; i += SN_THREADS) bsi[i] = 0;
  __syncthreads();

  // elements of the slice: validation, counts and centroid sums per (continuum, sub-block)
  const int e0 = y0 * n, e1 = min(y1, n) * n;
  for (int e = e0 + tid; e < e1; e += SN_THREADS) {
    const double k = kap[e];
    const int l = lab[e];
    if (!(k > 0.0) || !(k < 1e300)) atomicOr(&flags, 1);
    if (l >= N) {
      atomicOr(&flags, 2);
      continue;
    }
    const int ex = e % n, ey = e / n;
    const int b = l * nq + (ey / m) * P + ex / m;
    // lanes of the same bin add once (consecutive elements share a bin)
    const unsigned peers = __match_any_sync(__activemask(), b);
    const int cnt = __popc(peers);
    const int sx = __reduce_add_sync(peers, ex), sy = __reduce_add_sync(peers, ey);
    if ((tid & 31) == __ffs(peers) - 1) {
      atomicAdd(&bsi[3 * b + 0], cnt);
      atomicAdd(&bsi[3 * b + 1], sx);
      atomicAdd(&bsi[3 * b + 2], sy);
    }
  }
  __syncthreads();
  if (flags) {
    if (tid == 0) atomicOr(&a.status[pt], flags);
    return;
  }

  // M^-1 of the slice's nodes and the slice's part of S: per node, 1/diag times every pair
  // of its adjacent elements' rows; runs of equal row signatures along a column are summed
  // before the flush.
  double *mv = a.minv + (size_t)pt * a.nv;
  const int W = n + 1;
  for (int col = tid; col < W; col += SN_THREADS) {
    unsigned sig = 0xffffffffu;
    double acc = 0.0;
    auto flush = [&]() {
      if (sig == 0xffffffffu) return;
      const int bb[4] = {int(sig & 255), int((sig >> 8) & 255), int((sig >> 16) & 255),
                         int(sig >> 24)};
      for (int e1_ = 0; e1_ < 4; ++e1_)
        for (int e2_ = 0; e2_ < 4; ++e2_) atomicAdd(&S[bb[e1_] * nc + bb[e2_]], acc);
    };
    for (int ky = y0; ky < y1; ++ky) {
      if (col == 0 || ky == 0 || col == n || ky == n) {
        mv[col + W * ky] = 0.0;
        continue;
      }
      const int kx = col;
      const int eSW = (kx - 1) + n * (ky - 1), eSE = kx + n * (ky - 1);
      const int eNW = (kx - 1) + n * ky, eNE = kx + n * ky;
      const double dinv =
          fast_rcp((kap[eSW] + kap[eSE] + kap[eNW] + kap[eNE]) * (2.0 / 3.0));
      mv[col + W * ky] = dinv;
      // labels of the neighbouring slice are not validated here: clamp them (an invalid
      // label is reported by that slice)
      const int b0 = min((int)lab[eSW], N - 1) * nq + ((ky - 1) / m) * P + (kx - 1) / m;
      const int b1 = min((int)lab[eSE], N - 1) * nq + ((ky - 1) / m) * P + kx / m;
      const int b2 = min((int)lab[eNW], N - 1) * nq + (ky / m) * P + (kx - 1) / m;
      const int b3 = min((int)lab[eNE], N - 1) * nq + (ky / m) * P + kx / m;
      const unsigned key = (unsigned)b0 | ((unsigned)b1 << 8) | ((unsigned)b2 << 16) |
                           ((unsigned)b3 << 24);
      if (key != sig) {
        flush();
        sig = key;
        acc = 0.0;
      }
      acc += dinv;
    }
    // the column's last run: lanes with the same row signature add once
    const unsigned peers = __match_any_sync(__activemask(), sig);
    double tot = 0.0;
    for (unsigned mm = peers; mm; mm &= mm - 1) tot += __shfl_sync(peers, acc, __ffs(mm) - 1);
    if ((tid & 31) == __ffs(peers) - 1) {
      acc = tot;
      flush();
    }
  }
  __syncthreads();
  double *Sg = a.Sacc + (size_t)pt * nc * nc;
  for (int i = tid; i < nc * nc; i += SN_THREADS)
    if (S[i] != 0.0) atomicAdd(&Sg[i], S[i]);
  // counts and centroid sums: sum over elements of (-len/2 + (e + 1/2) h) from the integer
  // index sums (exact)
  double *bg = a.bacc + (size_t)pt * nc * 3;
  for (int i = tid; i < nc * 3; i += SN_THREADS) {
    const int b = i / 3, c = i % 3;
    const int cnt = bsi[3 * b];
    if (cnt == 0) continue;
    const double v = c == 0 ? (double)cnt
                            : (double)cnt * (-0.5 * a.len + 0.5 * a.h) + a.h * (double)bsi[i];
    atomicAdd(&bg[i], v);
  }
}

// One CTA per point. S^-1 by in-place Gauss-Jordan elimination, one thread per matrix entry:
// nc pivot steps of fully parallel rank-one updates (S is symmetric positive definite, so the
// diagonal pivots, the Schur-complement diagonals of the elimination, need no pivoting).
constexpr int SP_THREADS = 1024;

__global__ void __launch_bounds__(SP_THREADS) k_setup_point(SetupArgs a) {
  const int pt = blockIdx.x;
  const int P = a.P, N = a.N, R = a.R, nc = a.nc;
  const int nq = P * P;
  const int tid = threadIdx.x;
  if (a.status[pt] & 3) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *A = reinterpret_cast<double *>(smem_raw);      // [nc][nc], S then S^-1
  double *bs = A + nc * nc;                               // [nc][3] count, sum x, sum y
  double *cen = bs + 3 * nc;                              // [MCH_MAX_CONT][2]
  double *dorig = cen + 2 * MCH_MAX_CONT;                 // [nc]
  double *col = dorig + nc;                               // [nc] pivot column of a step
  double *rowk = col + nc;                                // [nc] pivot row of a step
  __shared__ int flags;
  __shared__ double rpiv;
  if (tid == 0) flags = 0;
  const double *Sg = a.Sacc + (size_t)pt * nc * nc;
  for (int i = tid; i < nc * nc; i += SP_THREADS) A[i] = Sg[i];
  for (int i = tid; i < 3 * nc; i += SP_THREADS) bs[i] = a.bacc[(size_t)pt * nc * 3 + i];
  __syncthreads();

  // centroids c_mj over the integration region R_p (the central (P - 2 overs)^2 periods;
  // the whole RVE when the continuum is absent there, or when overs = 0)
  if (tid < N) {
    double c = 0, x = 0, y = 0, ca = 0, xa = 0, ya = 0;
    for (int q = 0; q < nq; ++q) {
      const int b = tid * nq + q;
      const int qx = q % P, qy = q / P;
      ca += bs[3 * b];
      xa += bs[3 * b + 1];
      ya += bs[3 * b + 2];
      if (qx >= a.overs && qx < P - a.overs && qy >= a.overs && qy < P - a.overs) {
        c += bs[3 * b];
        x += bs[3 * b + 1];
        y += bs[3 * b + 2];
      }
    }
    if (ca == 0.0) atomicOr(&flags, 8);
    if (c == 0.0) {
      c = ca;
      x = xa;
      y = ya;
    }
    cen[2 * tid] = c > 0 ? x / c : 0.0;
    cen[2 * tid + 1] = c > 0 ? y / c : 0.0;
  }
  __syncthreads();

  // scaled targets G[b][r]
  double *G = a.G + (size_t)pt * nc * R;
  for (int t = tid; t < nc * R; t += SP_THREADS) {
    const int b = t / R, r = t % R;
    const int j = b / nq;
    double v = 0.0;
    if (r < N) {
      if (r == j) v = 4.0 * bs[3 * b];
    } else {
      const int i = (r - N) / 2, mm = (r - N) % 2;
      if (i == j) v = 4.0 * (bs[3 * b + 1 + mm] - bs[3 * b] * cen[2 * j + mm]);
    }
    G[t] = v;
  }
  if (tid < nc) {
    if (bs[3 * tid] == 0.0) A[tid * nc + tid] = 1.0;
    dorig[tid] = A[tid * nc + tid];
  }
  __syncthreads();

  // Gauss-Jordan: after step k, row k holds e_k^T times the running inverse
  for (int k = 0; k < nc; ++k) {
    if (tid == 0) {
      double v = A[k * nc + k];
      if (!(v > 1e-13 * dorig[k])) {
        flags |= 4;
        v = dorig[k] > 0 ? dorig[k] : 1.0;
      }
      rpiv = 1.0 / v;
    }
    // snapshot the pivot column and row: the update below overwrites both
    for (int i = tid; i < nc; i += SP_THREADS) {
      col[i] = A[i * nc + k];
      rowk[i] = A[k * nc + i];
    }
    __syncthreads();
    const double rp = rpiv;
    for (int t = tid; t < nc * nc; t += SP_THREADS) {
      const int i = t / nc, j = t % nc;
      // pivot row: A[k][j] / p (the pivot entry itself becomes 1 / p)
      const double akj = (j == k ? 1.0 : rowk[j]) * rp;
      if (i == k) {
        A[t] = akj;
      } else {
        const double f = col[i];
        A[t] = (j == k ? 0.0 : A[t]) - f * akj;
      }
    }
    __syncthreads();
  }

  double *Si64 = a.Sinv64 + (size_t)pt * nc * nc;
  float *Si32 = a.Sinv32 ? a.Sinv32 + (size_t)pt * nc * nc : nullptr;
  for (int t = tid; t < nc * nc; t += SP_THREADS) {
    // symmetrise (the elimination leaves round-off asymmetry)
    const int i = t / nc, j = t % nc;
    const double v = 0.5 * (A[t] + A[j * nc + i]);
    Si64[t] = v;
    if (Si32) Si32[t] = (float)v;
  }
  if (tid == 0) {
    int nd = 0;
    for (int b = 0; b < nc; ++b) nd += (bs[3 * b] == 0.0);
    a.dropped[pt] = nd;
    a.status[pt] |= flags;
  }
}

}  // namespace

cudaError_t launch_setup2d(const SetupArgs &a, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(a.Sacc, 0, sizeof(double) * a.npts * a.nc * a.nc, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.bacc, 0, sizeof(double) * a.npts * a.nc * 3, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.status, 0, sizeof(int) * a.npts, st);
  if (e != cudaSuccess) return e;
  // enough slices to give every SM a few CTAs when the level has few points
  int slices = (4 * device_sm_count() + a.npts - 1) / a.npts;
  slices = slices < 1 ? 1 : (slices > (a.n + 1) / 4 ? (a.n + 1) / 4 : slices);
  k_setup_nodes<<<dim3(a.npts, slices), SN_THREADS, 0, st>>>(a, slices);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = sizeof(double) * ((size_t)a.nc * a.nc + 6 * a.nc + 2 * MCH_MAX_CONT);
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(k_setup_point, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_setup_point<<<a.npts, SP_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace mch
