// Shared-memory-resident projected PCG for the 2D constrained cell problems (template;
// instantiated per precision in k_pcg_f32.cu and k_pcg_f64.cu).
//
// One (point, cell function) unit is one CTA, or one thread-block cluster of CL CTAs that
// split the node rows into slabs and exchange halo rows and partial sums through
// distributed shared memory. The unit's whole iteration state stays on chip for the sweep:
// the search direction p, kappa and the labels in shared memory, x, r, A p and M^-1 in
// registers. HBM is touched only to load kappa, labels, S^-1 and the initial residual, and
// to store the correction at the end.
//
// Iteration (Sec. 3, Eq. phi_abstract: minimise the energy over the constraint set; the
// method is projected conjugate gradients with the constraint preconditioner
// P r = M^-1 (r - Ct^T S^-1 Ct M^-1 r), M = diag A, S = Ct M^-1 Ct^T):
//   q = A p
//   one reduction of  p.q, z.q, q.M^-1 q, r.z, Ct z, Ct M^-1 q   (z = M^-1 r)
//   alpha = rho / p.q,  c = Ct z - alpha Ct M^-1 q,  lambda = S^-1 c
//   x += alpha p,  r <- r - alpha q - Ct^T lambda   (residual kept projected)
//   rho' = r.z - 2 alpha z.q + alpha^2 q.M^-1 q - lambda.c     (= new r.M^-1 r)
//   p = M^-1 r + (rho'/rho) p
// so every iteration has one reduction phase and two barriers (p visible, partial sums
// complete). Every warp evaluates the scalars and lambda from the reduced sums itself, so
// no warp waits on another after the reduction. Keeping r projected (rather than
// projecting only z) avoids the cancellation that otherwise pushes FP32 iterates off the
// constraint set.
//
// Constraint rows: node k contributes v_k to the row of each of its four adjacent elements.
// A thread's column strip has fixed west/east element columns, so the west and east
// contributions are accumulated per label in registers (static slots); the east slot of
// lane c belongs to column c+1, whose owner is lane c+1, and is handed over with one
// shfl_up. Rows per thread divide the sub-block size, so all south elements of a strip lie
// in one sub-block row; only the north elements of the strip's last row can fall in the
// next one, and those few go straight to shared-memory atomics.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"

namespace mch {

namespace cg = cooperative_groups;

template <typename T, int CL>
struct ClusterOps {
  __device__ static void sync() {
    if constexpr (CL > 1) cg::this_cluster().sync();
    else __syncthreads();
  }
  __device__ static int rank() {
    if constexpr (CL > 1) return (int)cg::this_cluster().block_rank();
    else return 0;
  }
  __device__ static T *remote(T *p, int rk) {
    if constexpr (CL > 1) return cg::this_cluster().map_shared_rank(p, rk);
    else return p;
  }
};

template <int NC, typename T>
__device__ __forceinline__ void add_lab(T (&acc)[NC], int lab, T v) {
#pragma unroll
  for (int j = 0; j < NC; ++j) acc[j] += (lab == j) ? v : T(0);
}

template <typename T, int NEL, int RG, int RPT, int CL, int NC>
__global__ void __launch_bounds__(NEL * RG) k_pcg2d(PcgArgs<T> a) {
  using C = ClusterOps<T, CL>;
  constexpr int THREADS = NEL * RG;
  constexpr int NWARPS = THREADS / 32;
  constexpr int ROWS = RG * RPT;
  constexpr int W = NEL + 1;
  const int n = NEL;
  const int unit = blockIdx.x / CL;
  if (a.done[unit]) return;  // uniform over the cluster: no barrier has been used yet
  const int rank = C::rank();
  const int pt = unit / a.R;
  const int nc = a.nc;
  const int NRED = 4 + 2 * nc;
  const int lgm = a.lgm, lgP = a.lgP, lgnq = 2 * a.lgP;
  const int m = 1 << lgm;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *ps = reinterpret_cast<T *>(smem_raw);   // [(ROWS+2)][W] search direction with halo rows
  T *ks = ps + (ROWS + 2) * W;               // [(ROWS+1)][NEL] kappa of element rows r_lo-1..
  T *sinv = ks + (ROWS + 1) * NEL;           // [nc][nc] (symmetric)
  T *red = sinv + nc * nc;                   // [2][NRED] partial sums (double-buffered)
  T *twarp = red + 2 * NRED;                 // [NWARPS][NRED] per-warp totals
  T *lamw = twarp + NWARPS * NRED;           // [NWARPS][nc] per-warp multipliers
  T *bc = lamw + NWARPS * nc;                // [8]
  uint8_t *ls = reinterpret_cast<uint8_t *>(bc + 8);  // [(ROWS+1)][NEL] labels

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int c = tid % NEL, g = tid / NEL;
  const int G = rank * RG + g;
  const int r_lo = 1 + rank * ROWS;
  const int kx = c + 1;
  const int kxE = kx + 1 <= n ? kx + 1 : n;   // clamp for the inactive last lane
  const int cE = c + 1 <= n - 1 ? c + 1 : n - 1;
  const bool col_active = c < n - 1;
  const int bxW = c >> lgm, bxE = cE >> lgm;
  const int bym = (G * RPT) >> lgm;
  // north elements of the strip's last row lie in the next sub-block row
  const bool next_row = (((G + 1) * RPT) & (m - 1)) == 0;
  const int baseW = (bym << lgP) + bxW, baseE = (bym << lgP) + bxE;
  const int baseWn = ((bym + 1) << lgP) + bxW, baseEn = ((bym + 1) << lgP) + bxE;

  // ---- load the unit's data
  const double *kap = a.kappa + (size_t)pt * n * n;
  const uint8_t *lab = a.labels + (size_t)pt * n * n;
  for (int t = tid; t < (ROWS + 2) * W; t += THREADS) ps[t] = T(0);
  for (int t = tid; t < (ROWS + 1) * NEL; t += THREADS) {
    const int ey = r_lo - 1 + t / NEL, ex = t % NEL;
    const bool in = ey < n;
    ks[t] = in ? T(kap[ex + n * ey]) : T(0);
    ls[t] = in ? lab[ex + n * ey] : uint8_t(0);
  }
  const T *Si = a.Sinv + (size_t)pt * nc * nc;
  for (int t = tid; t < nc * nc; t += THREADS) sinv[t] = Si[t];
  for (int t = tid; t < 2 * NRED; t += THREADS) red[t] = T(0);
  __syncthreads();

  T x[RPT], rr[RPT], q[RPT], mi[RPT];
  T *vec = a.vec + (size_t)unit * a.nv;
  T dz = T(0);
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int lr = 1 + g * RPT + i;
    const int ky = r_lo + lr - 1;
    const bool act = col_active && ky <= n - 1;
    x[i] = T(0);
    q[i] = T(0);
    rr[i] = act ? vec[kx + (n + 1) * ky] : T(0);
    const T dg = q1_diag(ks[(lr - 1) * NEL + c], ks[(lr - 1) * NEL + cE], ks[lr * NEL + c],
                         ks[lr * NEL + cE]);
    mi[i] = act ? T(1) / dg : T(0);
    const T z = mi[i] * rr[i];
    dz += rr[i] * z;
    if (act) ps[lr * W + kx] = z;
  }
  if constexpr (CL > 1) {
    if (g == 0 && rank > 0) C::remote(ps, rank - 1)[(ROWS + 1) * W + kx] = ps[1 * W + kx];
    if (g == RG - 1 && rank < CL - 1) C::remote(ps, rank + 1)[kx] = ps[ROWS * W + kx];
  }
  dz = warp_sum(dz);
  if (lane == 0) atomicAdd(&red[NRED + 0], dz);   // the initial phase uses buffer 1
  C::sync();
  T rho0 = T(0);
  for (int rk = 0; rk < CL; ++rk) rho0 += C::remote(red, rk)[NRED + 0];
  T rho = rho0;
  int it = 0;
  bool breakdown = false;
  T *tw = twarp + warp * NRED;
  T *lw = lamw + warp * nc;

  if (rho0 > T(0)) {
    for (;; ++it) {
      C::sync();  // B1: p and its halo visible; reads of the buffer zeroed below are done
      T *rb = red + (it & 1) * NRED;
      T *rn = red + ((it + 1) & 1) * NRED;
      for (int t = tid; t < NRED; t += THREADS) rn[t] = T(0);

      // ---- q = A p with a sliding 3-row window, plus the partial sums
      T pq = 0, zq = 0, qmq = 0, rz = 0;
      T azW[NC], azE[NC], aqW[NC], aqE[NC];
#pragma unroll
      for (int j = 0; j < NC; ++j) azW[j] = azE[j] = aqW[j] = aqE[j] = T(0);
      int lr = 1 + g * RPT;
      T pW0 = ps[(lr - 1) * W + kx - 1], pC0 = ps[(lr - 1) * W + kx], pE0 = ps[(lr - 1) * W + kxE];
      T pW1 = ps[lr * W + kx - 1], pC1 = ps[lr * W + kx], pE1 = ps[lr * W + kxE];
      T kS0 = ks[(lr - 1) * NEL + c], kS1 = ks[(lr - 1) * NEL + cE];
      int lS0 = ls[(lr - 1) * NEL + c], lS1 = ls[(lr - 1) * NEL + cE];
#pragma unroll
      for (int i = 0; i < RPT; ++i, ++lr) {
        const T pW2 = ps[(lr + 1) * W + kx - 1], pC2 = ps[(lr + 1) * W + kx],
                pE2 = ps[(lr + 1) * W + kxE];
        const T kN0 = ks[lr * NEL + c], kN1 = ks[lr * NEL + cE];
        const int lN0 = ls[lr * NEL + c], lN1 = ls[lr * NEL + cE];
        const int ky = r_lo + lr - 1;
        const bool act = col_active && ky <= n - 1;
        T qv = q1_apply(kS0, kS1, kN0, kN1, pW0, pC0, pE0, pW1, pC1, pE1, pW2, pC2, pE2);
        qv = act ? qv : T(0);
        q[i] = qv;
        const T z = mi[i] * rr[i];
        const T mq = mi[i] * qv;
        pq += pC1 * qv;
        zq += z * qv;
        qmq += qv * mq;
        rz += rr[i] * z;
        // inactive nodes carry z = mq = 0, so their contributions vanish
        add_lab<NC>(azW, lS0, z);
        add_lab<NC>(azE, lS1, z);
        add_lab<NC>(aqW, lS0, mq);
        add_lab<NC>(aqE, lS1, mq);
        if (i < RPT - 1 || !next_row) {
          add_lab<NC>(azW, lN0, z);
          add_lab<NC>(azE, lN1, z);
          add_lab<NC>(aqW, lN0, mq);
          add_lab<NC>(aqE, lN1, mq);
        } else if (act) {
          atomicAdd(&rb[4 + (lN0 << lgnq) + baseWn], z);
          atomicAdd(&rb[4 + (lN1 << lgnq) + baseEn], z);
          atomicAdd(&rb[4 + nc + (lN0 << lgnq) + baseWn], mq);
          atomicAdd(&rb[4 + nc + (lN1 << lgnq) + baseEn], mq);
        }
        pW0 = pW1; pC0 = pC1; pE0 = pE1;
        pW1 = pW2; pC1 = pC2; pE1 = pE2;
        kS0 = kN0; kS1 = kN1; lS0 = lN0; lS1 = lN1;
      }
      // hand the east slots to the owner of column c+1; lane 31 hands over through shared
      const int seg = m < 32 ? m : 32;
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        const T uz = __shfl_up_sync(0xffffffffu, azE[j], 1);
        const T uq = __shfl_up_sync(0xffffffffu, aqE[j], 1);
        if (lane > 0) {  // lane 0's west column gets the east slot of the previous warp's
          azW[j] += uz;  // lane 31, which adds it to shared memory itself
          aqW[j] += uq;
        }
        if (lane == 31 && (azE[j] != T(0) || aqE[j] != T(0))) {
          atomicAdd(&rb[4 + (j << lgnq) + baseE], azE[j]);
          atomicAdd(&rb[4 + nc + (j << lgnq) + baseE], aqE[j]);
        }
        const T sz = seg_sum(azW[j], seg);
        const T sq = seg_sum(aqW[j], seg);
        if ((lane & (seg - 1)) == 0) {
          atomicAdd(&rb[4 + (j << lgnq) + baseW], sz);
          atomicAdd(&rb[4 + nc + (j << lgnq) + baseW], sq);
        }
      }
      pq = warp_sum(pq);
      zq = warp_sum(zq);
      qmq = warp_sum(qmq);
      rz = warp_sum(rz);
      if (lane == 0) {
        atomicAdd(&rb[0], pq);
        atomicAdd(&rb[1], zq);
        atomicAdd(&rb[2], qmq);
        atomicAdd(&rb[3], rz);
      }
      C::sync();  // B2: every partial of every CTA is in place

      // ---- scalars and multipliers, evaluated by every warp from the same sums
      for (int t = lane; t < NRED; t += 32) {
        T v = T(0);
        for (int rk = 0; rk < CL; ++rk) v += C::remote(rb, rk)[t];
        tw[t] = v;
      }
      __syncwarp();
      const T tpq = tw[0], tzq = tw[1], tqmq = tw[2], trz = tw[3];
      T alpha = rho / tpq;
      const bool bad = !(tpq > T(0)) || !(alpha == alpha) || !(alpha < T(3.0e38));
      if (bad) alpha = T(0);
      __syncwarp();
      for (int t = lane; t < nc; t += 32) tw[4 + t] = tw[4 + t] - alpha * tw[4 + nc + t];
      __syncwarp();
      T lc = T(0);
      for (int i = lane; i < nc; i += 32) {
        // S^-1 is symmetric: column i is read so that consecutive lanes hit distinct banks
        T l0 = T(0), l1 = T(0), l2 = T(0), l3 = T(0);
        int j = 0;
        for (; j + 3 < nc; j += 4) {
          l0 += sinv[(j + 0) * nc + i] * tw[4 + j + 0];
          l1 += sinv[(j + 1) * nc + i] * tw[4 + j + 1];
          l2 += sinv[(j + 2) * nc + i] * tw[4 + j + 2];
          l3 += sinv[(j + 3) * nc + i] * tw[4 + j + 3];
        }
        for (; j < nc; ++j) l0 += sinv[j * nc + i] * tw[4 + j];
        const T l = (l0 + l1) + (l2 + l3);
        lw[i] = bad ? T(0) : l;
        lc += l * tw[4 + i];
      }
      lc = warp_sum(lc);
      __syncwarp();
      const T rho_new = trz - T(2) * alpha * tzq + alpha * alpha * tqmq - lc;
      int stop = 0;
      if (bad) stop = 2;
      else if (!(rho_new > T(a.tol) * T(a.tol) * rho0)) stop = 1;
      else if (it + 1 >= a.max_iter) stop = 1;
      const T beta = stop ? T(0) : rho_new / rho;
      rho = rho_new;

      // ---- updates (labels again through a sliding window)
      lr = 1 + g * RPT;
      lS0 = ls[(lr - 1) * NEL + c];
      lS1 = ls[(lr - 1) * NEL + cE];
#pragma unroll
      for (int i = 0; i < RPT; ++i, ++lr) {
        const int lN0 = ls[lr * NEL + c], lN1 = ls[lr * NEL + cE];
        const int ky = r_lo + lr - 1;
        const bool act = col_active && ky <= n - 1;
        const bool nr = (i == RPT - 1) && next_row && act;  // keeps inactive bins in range
        const T p0 = ps[lr * W + kx];
        x[i] += alpha * p0;
        const T cl = lw[(lS0 << lgnq) + baseW] + lw[(lS1 << lgnq) + baseE] +
                     lw[(lN0 << lgnq) + (nr ? baseWn : baseW)] +
                     lw[(lN1 << lgnq) + (nr ? baseEn : baseE)];
        rr[i] = act ? rr[i] - alpha * q[i] - cl : T(0);
        const T pn = mi[i] * rr[i] + beta * p0;
        if (act && !stop) ps[lr * W + kx] = pn;
        lS0 = lN0;
        lS1 = lN1;
      }
      if (stop) {
        breakdown = (stop == 2);
        break;
      }
      if constexpr (CL > 1) {
        if (g == 0 && rank > 0) C::remote(ps, rank - 1)[(ROWS + 1) * W + kx] = ps[1 * W + kx];
        if (g == RG - 1 && rank < CL - 1) C::remote(ps, rank + 1)[kx] = ps[ROWS * W + kx];
      }
    }
  }

  // ---- write the correction
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int lrr = 1 + g * RPT + i;
    const int ky = r_lo + lrr - 1;
    if (col_active && ky <= n - 1) vec[kx + (n + 1) * ky] = x[i];
  }
  if (rank == 0 && tid == 0) {
    a.iters[unit] += (rho0 > T(0)) ? it + 1 : 0;
    if (breakdown) a.status[unit] |= 1;
  }
  C::sync();  // no CTA leaves while a peer may still read its shared memory
}

template <typename T, int NEL, int RG, int RPT, int CL, int NC>
cudaError_t launch_pcg_cfg(const PcgArgs<T> &a, cudaStream_t st) {
  constexpr int THREADS = NEL * RG;
  constexpr int ROWS = RG * RPT;
  const int nred = 4 + 2 * a.nc;
  const size_t smem = sizeof(T) * ((ROWS + 2) * (NEL + 1) + (ROWS + 1) * NEL + a.nc * a.nc +
                                   2 * nred + (THREADS / 32) * (nred + a.nc) + 8) +
                      (ROWS + 1) * NEL + 16;
  auto kern = k_pcg2d<T, NEL, RG, RPT, CL, NC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.npts * a.R * CL);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = CL > 1 ? 1 : 0;
  e = cudaLaunchKernelEx(&cfg, kern, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename T, int NEL, int RG, int RPT, int CL>
cudaError_t launch_pcg_nc(const PcgArgs<T> &a, cudaStream_t st) {
  if (a.N <= 2) return launch_pcg_cfg<T, NEL, RG, RPT, CL, 2>(a, st);
  if (a.N == 3) return launch_pcg_cfg<T, NEL, RG, RPT, CL, 3>(a, st);
  return launch_pcg_cfg<T, NEL, RG, RPT, CL, 4>(a, st);
}

}  // namespace mch
