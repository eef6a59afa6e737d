// Shared-memory-resident projected PCG for the 2D constrained cell problems.
//
// One (point, cell function) unit is one CTA, or one thread-block cluster of CL CTAs that
// split the node rows into slabs and exchange halo rows and partial sums through
// distributed shared memory. The unit's whole iteration state stays on chip for the sweep:
// the search direction p and kappa in shared memory, x, r, A p and M^-1 in registers. HBM
// is touched only to load kappa, labels, S^-1 and the initial residual, and to store the
// correction at the end.
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
// so every iteration has a single reduction phase. Keeping r projected (rather than
// projecting only z) avoids the cancellation that otherwise pushes FP32 iterates off the
// constraint set.
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace mch {

namespace {

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

template <typename T>
__device__ __forceinline__ T rcp(T v) { return T(1) / v; }

template <typename T, int NEL, int RG, int RPT, int CL>
__global__ void __launch_bounds__(NEL * RG) k_pcg2d(PcgArgs<T> a) {
  using C = ClusterOps<T, CL>;
  constexpr int THREADS = NEL * RG;
  constexpr int ROWS = RG * RPT;
  constexpr int W = NEL + 1;
  const int n = NEL;
  const int unit = blockIdx.x / CL;
  if (a.done[unit]) return;  // uniform over the cluster: no barrier has been used yet
  const int rank = C::rank();
  const int pt = unit / a.R;
  const int nc = a.nc;
  const int NRED = 4 + 2 * nc;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *ps = reinterpret_cast<T *>(smem_raw);   // [(ROWS+2)][W] search direction with halo rows
  T *ks = ps + (ROWS + 2) * W;               // [(ROWS+1)][NEL] kappa of element rows r_lo-1..
  T *sinv = ks + (ROWS + 1) * NEL;           // [nc][nc]
  T *red = sinv + nc * nc;                   // [2][NRED] partial sums (double-buffered)
  T *lam = red + 2 * NRED;                   // [nc]
  T *tot = lam + nc;                         // [NRED]
  T *bc = tot + NRED;                        // [8] broadcast scalars
  uint8_t *ls = reinterpret_cast<uint8_t *>(bc + 8);  // [(ROWS+1)][NEL] labels

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int c = tid % NEL, g = tid / NEL;
  const int G = rank * RG + g;
  const int r_lo = 1 + rank * ROWS;
  Strip s;
  s.init(n, a.P, c, G, RPT);
  const int kx = c + 1;
  const int kxE = kx + 1 <= n ? kx + 1 : n;   // clamp for the inactive last lane
  const int cE = c + 1 <= n - 1 ? c + 1 : n - 1;
  const bool col_active = c < n - 1;

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
    mi[i] = act ? rcp(dg) : T(0);
    const T z = mi[i] * rr[i];
    dz += rr[i] * z;
    if (act) ps[lr * W + kx] = z;
  }
  // halo push of the initial direction
  if constexpr (CL > 1) {
    if (g == 0 && rank > 0) C::remote(ps, rank - 1)[(ROWS + 1) * W + kx] = ps[1 * W + kx];
    if (g == RG - 1 && rank < CL - 1) C::remote(ps, rank + 1)[kx] = ps[ROWS * W + kx];
  }
  dz = warp_sum(dz);
  if (lane == 0) atomicAdd(&red[NRED + 0], dz);   // initial phase uses buffer 1
  C::sync();
  if (warp == 0) {
    T v = T(0);
    for (int rk = 0; rk < CL; ++rk) v += C::remote(red, rk)[NRED + 0];
    if (lane == 0) bc[4] = v;
  }
  __syncthreads();
  const T rho0 = bc[4];
  T rho = rho0;
  int it = 0;
  bool breakdown = false;

  if (rho0 > T(0)) {
    for (;; ++it) {
      C::sync();  // B1: p and its halo visible; reads of the buffer zeroed below are done
      T *rb = red + (it & 1) * NRED;
      T *rn = red + ((it + 1) & 1) * NRED;
      for (int t = tid; t < NRED; t += THREADS) rn[t] = T(0);

      // ---- q = A p with a sliding 3-row window, plus the partial sums
      T pq = 0, zq = 0, qmq = 0, rz = 0;
      T accz[MCH_MAX_CONT] = {0, 0, 0, 0}, accq[MCH_MAX_CONT] = {0, 0, 0, 0};
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
        if (act) {
          scatter_node(s, ky, lS0, lS1, lN0, lN1, z, accz, rb + 4);
          scatter_node(s, ky, lS0, lS1, lN0, lN1, mq, accq, rb + 4 + nc);
        }
        pW0 = pW1; pC0 = pC1; pE0 = pE1;
        pW1 = pW2; pC1 = pC2; pE1 = pE2;
        kS0 = kN0; kS1 = kN1; lS0 = lN0; lS1 = lN1;
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
      flush_acc(s, accz, a.N, rb + 4, true);
      flush_acc(s, accq, a.N, rb + 4 + nc, true);
      C::sync();  // B2: every partial of every CTA is in place

      // ---- scalars and multipliers (warp 0 of each CTA, identical on every rank)
      if (warp == 0) {
        for (int t = lane; t < NRED; t += 32) {
          T v = T(0);
          for (int rk = 0; rk < CL; ++rk) v += C::remote(rb, rk)[t];
          tot[t] = v;
        }
        __syncwarp();
        const T tpq = tot[0], tzq = tot[1], tqmq = tot[2], trz = tot[3];
        T alpha = rho / tpq;
        const bool bad = !(tpq > T(0)) || !(alpha == alpha) || !(alpha < T(3.0e38));
        if (bad) alpha = T(0);
        for (int t = lane; t < nc; t += 32) tot[4 + t] = tot[4 + t] - alpha * tot[4 + nc + t];
        __syncwarp();
        T lc = T(0);
        for (int i = lane; i < nc; i += 32) {
          T l = T(0);
          for (int j = 0; j < nc; ++j) l += sinv[i * nc + j] * tot[4 + j];
          lam[i] = bad ? T(0) : l;
          lc += l * tot[4 + i];
        }
        lc = warp_sum(lc);
        const T rho_new = trz - T(2) * alpha * tzq + alpha * alpha * tqmq - lc;
        if (lane == 0) {
          int stop = 0;
          if (bad) stop = 2;
          else if (!(rho_new > a.tol * a.tol * rho0)) stop = 1;
          else if (it + 1 >= a.max_iter) stop = 1;
          bc[0] = alpha;
          bc[1] = stop ? T(0) : rho_new / rho;
          bc[2] = T(stop);
          bc[3] = rho_new;
        }
      }
      __syncthreads();  // B3
      const T alpha = bc[0], beta = bc[1];
      const int stop = (int)bc[2];
      rho = bc[3];

      // ---- updates
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int lrr = 1 + g * RPT + i;
        const int ky = r_lo + lrr - 1;
        const bool act = col_active && ky <= n - 1;
        if (!act) continue;
        const T p0 = ps[lrr * W + kx];
        x[i] += alpha * p0;
        const T cl = ct_lambda(s, ky, ls[(lrr - 1) * NEL + c], ls[(lrr - 1) * NEL + cE],
                               ls[lrr * NEL + c], ls[lrr * NEL + cE], lam);
        rr[i] = rr[i] - alpha * q[i] - cl;
        const T pn = mi[i] * rr[i] + beta * p0;
        if (!stop) ps[lrr * W + kx] = pn;
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

template <typename T, int NEL, int RG, int RPT, int CL>
cudaError_t launch_cfg(const PcgArgs<T> &a, cudaStream_t st) {
  constexpr int THREADS = NEL * RG;
  constexpr int ROWS = RG * RPT;
  const int nred = 4 + 2 * a.nc;
  const size_t smem = sizeof(T) * ((ROWS + 2) * (NEL + 1) + (ROWS + 1) * NEL + a.nc * a.nc +
                                   2 * nred + a.nc + nred + 8) +
                      (ROWS + 1) * NEL + 16;
  auto kern = k_pcg2d<T, NEL, RG, RPT, CL>;
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
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace

bool pcg2d_supported(int n, int P, bool fp64) {
  if (P < 1 || n % P) return false;
  const int m = n / P;
  if (m < 2 || (m & (m - 1))) return false;
  int rpt;
  switch (n) {
    case 16: rpt = 1; break;
    case 32: rpt = 4; break;
    case 64: rpt = fp64 ? 4 : 8; break;
    case 128: rpt = fp64 ? 8 : 16; break;
    case 256: if (fp64) return false; rpt = 16; break;
    default: return false;
  }
  return m % rpt == 0;
}

template <>
cudaError_t launch_pcg2d<float>(const PcgArgs<float> &a, cudaStream_t st, int *launches) {
  if (launches) ++*launches;
  switch (a.n) {
    case 16: return launch_cfg<float, 16, 16, 1, 1>(a, st);
    case 32: return launch_cfg<float, 32, 8, 4, 1>(a, st);
    case 64: return launch_cfg<float, 64, 8, 8, 1>(a, st);
    case 128: return launch_cfg<float, 128, 4, 16, 2>(a, st);
    case 256: return launch_cfg<float, 256, 2, 16, 8>(a, st);
  }
  return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_pcg2d<double>(const PcgArgs<double> &a, cudaStream_t st, int *launches) {
  if (launches) ++*launches;
  switch (a.n) {
    case 16: return launch_cfg<double, 16, 16, 1, 1>(a, st);
    case 32: return launch_cfg<double, 32, 8, 4, 1>(a, st);
    case 64: return launch_cfg<double, 64, 8, 4, 2>(a, st);
    case 128: return launch_cfg<double, 128, 4, 8, 4>(a, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mch
