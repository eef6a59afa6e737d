// Persistent level kernel for the 2D constrained cell problems (template; instantiated per
// inner precision in k_level_f32.cu and k_level_f64.cu).
//
// One launch solves every (point, cell function) unit of a level to the refinement
// tolerance. A unit is one CTA, or one thread-block cluster of CL CTAs that split the node
// rows into slabs and exchange halo rows and partial sums through distributed shared memory.
// Its whole state stays on chip for the launch: the FP32 (or FP64) search direction, the
// FP64 solution with halo rows, kappa and the labels in shared memory; the inner-precision
// correction, residual, A p and M^-1 in registers. HBM is read for the inputs and, in the
// FP64 steps, for kappa, M^-1 and the right-hand side, and written once for the solution.
//
// The unit minimises 1/2 x'A x - b'x subject to Ct x = g (Sec. 3, Eq. phi_abstract; at
// level 1 b = 0 and g are the targets of Eqs. phi_avar / phi_grad, at level n > 1 they are
// the correction data of Eqs. phi_avar_corrector / phi_grad_corrector). Loop:
//   FP64 refinement step: x += delta; x += M^-1 Ct^T S^-1 (g - Ct x)  (constraints exact);
//     r = b - A x; r <- r - Ct^T S^-1 Ct M^-1 r; rho64 = r'M^-1 r; stop when
//     sqrt(rho64 / rho64_ref) < rtol, else hand r to the next sweep as its residual.
//     rho64_ref = max(rho64 of the first step, b'M^-1 b): for a correction problem (n > 1)
//     the right-hand side b = -P^T A_1 I carries the scale of the cell function I + P Xi,
//     so the test bounds the error of the cell function, not of the (possibly tiny)
//     correction.
//   inner sweep (projected PCG, inner precision, from delta = 0):
//     q = A p
//     one reduction of  p.q, z.q, q.M^-1 q, r.z, Ct z, Ct M^-1 q   (z = M^-1 r)
//     alpha = rho / p.q,  c = Ct z - alpha Ct M^-1 q,  lambda = S^-1 c
//     delta += alpha p,  r <- r - alpha q - Ct^T lambda   (residual kept projected)
//     rho' = r.z - 2 alpha z.q + alpha^2 q.M^-1 q - lambda.c     (= new r.M^-1 r)
//     p = M^-1 r + (rho'/rho) p,   until sqrt(rho' / rho_first) < tol.
// Every sweep iteration has one reduction phase and two barriers; every warp evaluates the
// scalars and lambda from the reduced sums itself. Keeping r projected (rather than
// projecting only z) avoids the cancellation that otherwise pushes FP32 iterates off the
// constraint set; the FP64 steps restore the constraints and the true residual.
//
// Constraint rows: node k contributes v_k to the row of each of its four adjacent elements.
// A thread's column strip has fixed west/east element columns, so west and east
// contributions are accumulated per label in registers (static slots); the east slot of
// lane c belongs to column c+1, whose owner is lane c+1, and is handed over with one
// shfl_up. Rows per thread divide the sub-block size, so all south elements of a strip lie
// in one sub-block row; only the north elements of the strip's last row can fall in the
// next one, and those go straight to shared-memory atomics.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"

namespace mch {

namespace cg = cooperative_groups;

template <int CL>
struct ClusterOps {
  __device__ static void sync() {
    if constexpr (CL > 1) cg::this_cluster().sync();
    else __syncthreads();
  }
  __device__ static int rank() {
    if constexpr (CL > 1) return (int)cg::this_cluster().block_rank();
    else return 0;
  }
  template <typename V>
  __device__ static V *remote(V *p, int rk) {
    if constexpr (CL > 1) return cg::this_cluster().map_shared_rank(p, rk);
    else return p;
  }
};

template <int NC, typename V>
__device__ __forceinline__ void add_lab(V (&acc)[NC], int lab, V v) {
#pragma unroll
  for (int j = 0; j < NC; ++j) acc[j] += (lab == j) ? v : V(0);
}

// Adds a node value to the per-label west/east slots of its four adjacent elements; the
// north elements of an aligned strip's last row (to_next) go to `bins` directly.
template <int NC, typename V>
__device__ __forceinline__ void acc_node(V (&aW)[NC], V (&aE)[NC], int lS0, int lS1, int lN0,
                                         int lN1, V v, bool to_next, V *bins, int lgnq,
                                         int baseWn, int baseEn) {
  add_lab<NC>(aW, lS0, v);
  add_lab<NC>(aE, lS1, v);
  if (!to_next) {
    add_lab<NC>(aW, lN0, v);
    add_lab<NC>(aE, lN1, v);
  } else {
    atomicAdd(&bins[(lN0 << lgnq) + baseWn], v);
    atomicAdd(&bins[(lN1 << lgnq) + baseEn], v);
  }
}

// East slots to the owner lane of column c+1 (lane 31 adds its own directly), then sums over
// the lanes that share the west sub-block; the group leader adds to `bins`.
template <int NC, typename V>
__device__ __forceinline__ void flush_bins(V (&aW)[NC], V (&aE)[NC], V *bins, int lane, int seg,
                                           int lgnq, int baseW, int baseE) {
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    const V up = __shfl_up_sync(0xffffffffu, aE[j], 1);
    if (lane > 0) aW[j] += up;
    if (lane == 31 && aE[j] != V(0)) atomicAdd(&bins[(j << lgnq) + baseE], aE[j]);
    const V s = seg_sum(aW[j], seg);
    if ((lane & (seg - 1)) == 0 && s != V(0)) atomicAdd(&bins[(j << lgnq) + baseW], s);
  }
}

template <typename T, int NEL, int RG, int RPT, int CL, int NC, int MINB, bool SR>
__global__ void __launch_bounds__(NEL * RG, MINB) k_level2d(LevelArgs<T> a) {
  using C = ClusterOps<CL>;
  constexpr int THREADS = NEL * RG;
  constexpr int NWARPS = THREADS / 32;
  constexpr int ROWS = RG * RPT;
  constexpr int W = NEL + 1;
  const int n = NEL;
  const int unit = blockIdx.x / CL;
  const int rank = C::rank();
  const int pt = unit / a.R, rfun = unit % a.R;
  const int nc = a.nc;
  const int NRED = 4 + 2 * nc;
  const int lgm = a.lgm, lgP = a.lgP, lgnq = 2 * a.lgP;
  const int m = 1 << lgm;
  const int seg = m < 32 ? m : 32;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *xs = reinterpret_cast<double *>(smem_raw);  // [(ROWS+2)][W] FP64 solution + halo
  double *sinv64 = xs + (ROWS + 2) * W;               // [nc][nc]
  double *red64 = sinv64 + nc * nc;                   // [2 nc + 1] FP64 partial sums
  double *v64 = red64 + 2 * nc + 1;                   // [2 nc] mu, lambda
  double *sc64 = v64 + 2 * nc;                        // [2] scalars
  T *ps = reinterpret_cast<T *>(sc64 + 2);            // [(ROWS+2)][W] search direction
  T *ks = ps + (ROWS + 2) * W;                        // [(ROWS+1)][NEL] kappa rows r_lo-1..
  T *sinv = ks + (ROWS + 1) * NEL;                    // [nc][nc] (symmetric)
  T *red = sinv + nc * nc;                            // [2][NRED] (double-buffered)
  T *twarp = red + 2 * NRED;                          // [NWARPS][NRED]
  T *lamw = twarp + NWARPS * NRED;                    // [NWARPS][nc]
  T *mis = lamw + NWARPS * nc;                        // [ROWS][W] M^-1 of own rows
  uint8_t *ls = reinterpret_cast<uint8_t *>(mis + ROWS * W);  // [(ROWS+1)][NEL]
  // FP64 residual of the own rows between steps (d) and (e) when SR (8-byte aligned)
  double *rs = reinterpret_cast<double *>(
      (reinterpret_cast<uintptr_t>(ls + (ROWS + 1) * NEL) + 15) & ~uintptr_t(15));

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int c = tid % NEL, g = tid / NEL;
  const int G = rank * RG + g;
  const int r_lo = 1 + rank * ROWS;
  const int kx = c + 1;
  const int kxE = kx + 1 <= n ? kx + 1 : n;   // clamp for the inactive last lane
  const int cE = c + 1 <= n - 1 ? c + 1 : n - 1;
  const bool col_active = c < n - 1;
  (void)r_lo;
  const int bxW = c >> lgm, bxE = cE >> lgm;
  const int bym = (G * RPT) >> lgm;
  const bool next_row = (((G + 1) * RPT) & (m - 1)) == 0;
  const int baseW = (bym << lgP) + bxW, baseE = (bym << lgP) + bxE;
  const int baseWn = ((bym + 1) << lgP) + bxW, baseEn = ((bym + 1) << lgP) + bxE;

  // ---- load the unit's data
  const double *kap = a.kappa + (size_t)pt * n * n;
  const uint8_t *lab = a.labels + (size_t)pt * n * n;
  const double *mv64 = a.minv64 + (size_t)pt * a.nv;
  const double *bvec = a.b ? a.b + (size_t)unit * a.nv : nullptr;
  const double *gt = a.g + (size_t)pt * nc * a.R + rfun;  // stride R
  for (int t = tid; t < (ROWS + 2) * W; t += THREADS) {
    ps[t] = T(0);
    xs[t] = 0.0;
  }
  for (int t = tid; t < (ROWS + 1) * NEL; t += THREADS) {
    const int ey = r_lo - 1 + t / NEL, ex = t % NEL;
    const bool in = ey < n;
    ks[t] = in ? T(kap[ex + n * ey]) : T(0);
    // labels >= N (invalid input, reported by the setup) are clamped so that no row index
    // leaves the multiplier table
    ls[t] = in ? (uint8_t)min((int)lab[ex + n * ey], a.N - 1) : uint8_t(0);
  }
  {
    const T *Si = a.Sinv + (size_t)pt * nc * nc;
    const double *Si64 = a.Sinv64 + (size_t)pt * nc * nc;
    for (int t = tid; t < nc * nc; t += THREADS) {
      sinv[t] = Si[t];
      sinv64[t] = Si64[t];
    }
  }
  for (int t = tid; t < 2 * NRED; t += THREADS) red[t] = T(0);
  for (int t = tid; t < 2 * nc + 1; t += THREADS) red64[t] = 0.0;
  __syncthreads();

  // Per-thread base pointers: row i of the strip is at a compile-time offset from these.
  const int row0 = 1 + g * RPT;                    // first own row in the local arrays
  const int dEx = kxE - kx;                        // 1, or 0 for the inactive last lane
  const int dEc = cE - c;
  const int ky0 = r_lo + row0 - 1;                 // global node row of local row row0
  const int nact = col_active ? max(0, min(RPT, n - ky0)) : 0;  // active rows of the strip
  T *pb = ps + row0 * W + kx;                      // p at (row i, own column): pb[i*W]
  double *xb = xs + row0 * W + kx;
  T *mb = mis + (row0 - 1) * W + kx;               // M^-1 of row i: mb[i*W]
  const T *kb = ks + (row0 - 1) * NEL + c;         // kappa of element row (ky-1): kb[i*NEL]
  const uint8_t *lb = ls + (row0 - 1) * NEL + c;   // labels likewise
  const double *kg = kap + c + n * (ky0 - 1);      // FP64 kappa of element row (ky-1): kg[i*n]
  const double *mg = mv64 + kx + (n + 1) * ky0;    // FP64 M^-1 of row i: mg[i*(n+1)]
  const double *bg = bvec ? bvec + kx + (n + 1) * ky0 : nullptr;

  T x[RPT], rr[RPT], q[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    x[i] = T(0);
    rr[i] = T(0);
    q[i] = T(0);
    const T dg = q1_diag(kb[i * NEL], kb[i * NEL + dEc], kb[(i + 1) * NEL], kb[(i + 1) * NEL + dEc]);
    mb[i * W] = (i < nact) ? T(1) / dg : T(0);   // each thread reads only its own entries
  }
  T *tw = twarp + warp * NRED;
  T *lw = lamw + warp * nc;

  auto push_halo_x = [&]() {
    if constexpr (CL > 1) {
      if (g == 0 && rank > 0) C::remote(xs, rank - 1)[(ROWS + 1) * W + kx] = xs[1 * W + kx];
      if (g == RG - 1 && rank < CL - 1) C::remote(xs, rank + 1)[kx] = xs[ROWS * W + kx];
    }
  };
  auto push_halo_p = [&]() {
    if constexpr (CL > 1) {
      if (g == 0 && rank > 0) C::remote(ps, rank - 1)[(ROWS + 1) * W + kx] = ps[1 * W + kx];
      if (g == RG - 1 && rank < CL - 1) C::remote(ps, rank + 1)[kx] = ps[ROWS * W + kx];
    }
  };
  // small FP64 product out = S^-1 v by warp 0 (v, out in shared memory)
  auto small64 = [&](const double *v, double *out) {
    if (warp == 0) {
      for (int i = lane; i < nc; i += 32) {
        double s0 = 0.0, s1 = 0.0;
        int j = 0;
        for (; j + 1 < nc; j += 2) {
          s0 += sinv64[j * nc + i] * v[j];
          s1 += sinv64[(j + 1) * nc + i] * v[j + 1];
        }
        for (; j < nc; ++j) s0 += sinv64[j * nc + i] * v[j];
        out[i] = s0 + s1;
      }
    }
  };
  // sum of a per-row vector over the row's four adjacent constraint rows (Ct^T v at a node)
  auto ctv = [&](const auto *v, int lS0, int lS1, int lN0, int lN1, bool nr) {
    return v[(lS0 << lgnq) + baseW] + v[(lS1 << lgnq) + baseE] +
           v[(lN0 << lgnq) + (nr ? baseWn : baseW)] + v[(lN1 << lgnq) + (nr ? baseEn : baseE)];
  };
  // FP64 residual b - A x at row i from a sliding window (caller keeps the window)
  double rho64_first = 0.0, ratio = 0.0;
  int sweeps = 0, iters = 0;
  bool breakdown = false, done = false;

  for (int step = 0;; ++step) {
    // ================= FP64 refinement step =================
    // (a) fold the correction; (b) Ct x by element rows (column sums of node pairs)
    {
      double aW[NC], aE[NC];
#pragma unroll
      for (int j = 0; j < NC; ++j) aW[j] = aE[j] = 0.0;
      int lS0 = lb[0], lS1 = lb[dEc];
      double vprev = 0.0;
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int lN0 = lb[(i + 1) * NEL], lN1 = lb[(i + 1) * NEL + dEc];
        double v = 0.0;
        if (i < nact) {
          v = xb[i * W] + (double)x[i];
          xb[i * W] = v;
        }
        x[i] = T(0);
        const double u = v + vprev;
        add_lab<NC>(aW, lS0, u);
        add_lab<NC>(aE, lS1, u);
        vprev = v;
        lS0 = lN0;
        lS1 = lN1;
      }
      if (!next_row) {
        add_lab<NC>(aW, lS0, vprev);
        add_lab<NC>(aE, lS1, vprev);
      } else if (nact == RPT) {
        atomicAdd(&red64[(lS0 << lgnq) + baseWn], vprev);
        atomicAdd(&red64[(lS1 << lgnq) + baseEn], vprev);
      }
      flush_bins<NC>(aW, aE, red64, lane, seg, lgnq, baseW, baseE);
    }
    C::sync();
    // mu = S^-1 (g - Ct x)
    if (warp == 0) {
      for (int b = lane; b < nc; b += 32) {
        double s = 0.0;
        for (int rk = 0; rk < CL; ++rk) s += C::remote(red64, rk)[b];
        v64[nc + b] = gt[(size_t)b * a.R] - s;
      }
      __syncwarp();
    }
    small64(v64 + nc, v64);
    __syncthreads();
    // (c) x += M^-1 Ct^T mu
    {
      double wprev = v64[(lb[0] << lgnq) + baseW] + v64[(lb[dEc] << lgnq) + baseE];
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int lN0 = lb[(i + 1) * NEL], lN1 = lb[(i + 1) * NEL + dEc];
        const bool act = i < nact;
        const bool nr = (i == RPT - 1) && next_row && act;
        const double wcur = v64[(lN0 << lgnq) + (nr ? baseWn : baseW)] +
                            v64[(lN1 << lgnq) + (nr ? baseEn : baseE)];
        if (act) xb[i * W] += mg[i * (n + 1)] * (wprev + wcur);
        wprev = wcur;
      }
    }
    push_halo_x();
    C::sync();  // x and its halo final for this step; every rank has read red64[0..nc)
    // (d) Ct M^-1 r with r = b - A x (FP64); r kept in shared memory when SR, else formed
    // again in (e)
    {
      double aW[NC], aE[NC];
#pragma unroll
      for (int j = 0; j < NC; ++j) aW[j] = aE[j] = 0.0;
      double xW0 = xb[-W - 1], xC0 = xb[-W], xE0 = xb[-W + dEx];
      double xW1 = xb[-1], xC1 = xb[0], xE1 = xb[dEx];
      double kS0 = kg[0], kS1 = kg[dEc];
      int lS0 = lb[0], lS1 = lb[dEc];
      double zprev = 0.0;
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const bool act = i < nact;
        const double xW2 = xb[(i + 1) * W - 1], xC2 = xb[(i + 1) * W], xE2 = xb[(i + 1) * W + dEx];
        const double kN0 = act ? kg[(i + 1) * n] : 0.0, kN1 = act ? kg[(i + 1) * n + dEc] : 0.0;
        const int lN0 = lb[(i + 1) * NEL], lN1 = lb[(i + 1) * NEL + dEc];
        double zm = 0.0;
        if (act) {
          const double ax = q1_apply(kS0, kS1, kN0, kN1, xW0, xC0, xE0, xW1, xC1, xE1, xW2, xC2, xE2);
          const double rv = (bg ? bg[i * (n + 1)] : 0.0) - ax;
          if constexpr (SR) rs[(g * RPT + i) * W + kx] = rv;
          zm = mg[i * (n + 1)] * rv;
        }
        const double u = zm + zprev;
        add_lab<NC>(aW, lS0, u);
        add_lab<NC>(aE, lS1, u);
        zprev = zm;
        xW0 = xW1; xC0 = xC1; xE0 = xE1;
        xW1 = xW2; xC1 = xC2; xE1 = xE2;
        kS0 = kN0; kS1 = kN1; lS0 = lN0; lS1 = lN1;
      }
      if (!next_row) {
        add_lab<NC>(aW, lS0, zprev);
        add_lab<NC>(aE, lS1, zprev);
      } else if (nact == RPT) {
        atomicAdd(&red64[nc + (lS0 << lgnq) + baseWn], zprev);
        atomicAdd(&red64[nc + (lS1 << lgnq) + baseEn], zprev);
      }
      flush_bins<NC>(aW, aE, red64 + nc, lane, seg, lgnq, baseW, baseE);
    }
    C::sync();
    if (warp == 0) {
      for (int b = lane; b < nc; b += 32) {
        double s = 0.0;
        for (int rk = 0; rk < CL; ++rk) s += C::remote(red64, rk)[nc + b];
        v64[nc + b] = s;
      }
      __syncwarp();
    }
    small64(v64 + nc, v64);
    __syncthreads();
    // (e) projected residual, its M^-1 norm; the next sweep's residual
    {
      double rho_p = 0.0;
      double xW0 = 0, xC0 = 0, xE0 = 0, xW1 = 0, xC1 = 0, xE1 = 0, kS0 = 0, kS1 = 0;
      if constexpr (!SR) {
        xW0 = xb[-W - 1]; xC0 = xb[-W]; xE0 = xb[-W + dEx];
        xW1 = xb[-1]; xC1 = xb[0]; xE1 = xb[dEx];
        kS0 = kg[0]; kS1 = kg[dEc];
      }
      double wprev = v64[(lb[0] << lgnq) + baseW] + v64[(lb[dEc] << lgnq) + baseE];
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const bool act = i < nact;
        const int lN0 = lb[(i + 1) * NEL], lN1 = lb[(i + 1) * NEL + dEc];
        const bool nr = (i == RPT - 1) && next_row && act;
        const double wcur = v64[(lN0 << lgnq) + (nr ? baseWn : baseW)] +
                            v64[(lN1 << lgnq) + (nr ? baseEn : baseE)];
        double rv = 0.0;
        if constexpr (SR) {
          if (act) rv = rs[(g * RPT + i) * W + kx];
        } else {
          const double xW2 = xb[(i + 1) * W - 1], xC2 = xb[(i + 1) * W], xE2 = xb[(i + 1) * W + dEx];
          const double kN0 = act ? kg[(i + 1) * n] : 0.0, kN1 = act ? kg[(i + 1) * n + dEc] : 0.0;
          if (act)
            rv = (bg ? bg[i * (n + 1)] : 0.0) -
                 q1_apply(kS0, kS1, kN0, kN1, xW0, xC0, xE0, xW1, xC1, xE1, xW2, xC2, xE2);
          xW0 = xW1; xC0 = xC1; xE0 = xE1;
          xW1 = xW2; xC1 = xC2; xE1 = xE2;
          kS0 = kN0; kS1 = kN1;
        }
        double rt = 0.0;
        if (act) {
          rt = rv - (wprev + wcur);
          rho_p += rt * rt * mg[i * (n + 1)];
        }
        rr[i] = T(rt);
        wprev = wcur;
      }
      rho_p = warp_sum(rho_p);
      if (lane == 0) atomicAdd(&red64[2 * nc], rho_p);
    }
    C::sync();
    {
      double sum = 0.0;
      for (int rk = 0; rk < CL; ++rk) sum += C::remote(red64, rk)[2 * nc];
      if (step == 0) rho64_first = a.bnorm ? fmax(sum, a.bnorm[unit]) : sum;
      ratio = rho64_first > 0.0 ? sqrt(sum / rho64_first) : 0.0;
      if (!(ratio >= a.rtol)) done = true;
      if (!(ratio == ratio)) breakdown = true;
    }
    if (done || breakdown || step >= a.max_refine) break;

    // ================= inner PCG sweep =================
    C::sync();  // every rank has read red64; clear it and the inner buffers for reuse
    for (int t = tid; t < 2 * nc + 1; t += THREADS) red64[t] = 0.0;
    for (int t = tid; t < 2 * NRED; t += THREADS) red[t] = T(0);
    __syncthreads();
    ++sweeps;
    T dz = T(0);
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const T z = mb[i * W] * rr[i];
      dz += rr[i] * z;
      if (i < nact) pb[i * W] = z;
    }
    push_halo_p();
    dz = warp_sum(dz);
    if (lane == 0) atomicAdd(&red[NRED + 0], dz);   // the sweep's first sum uses buffer 1
    C::sync();
    T rho0 = T(0);
    for (int rk = 0; rk < CL; ++rk) rho0 += C::remote(red, rk)[NRED + 0];
    T rho = rho0;
    int it = 0;
    if (rho0 > T(0)) {
      for (;; ++it) {
        C::sync();  // B1: p and its halo visible; reads of the buffer zeroed below are done
        T *rb = red + (it & 1) * NRED;
        T *rn = red + ((it + 1) & 1) * NRED;
        for (int t = tid; t < NRED; t += THREADS) rn[t] = T(0);

        T pq = 0, zq = 0, qmq = 0, rz = 0;
        T azW[NC], azE[NC], aqW[NC], aqE[NC];
#pragma unroll
        for (int j = 0; j < NC; ++j) azW[j] = azE[j] = aqW[j] = aqE[j] = T(0);
        T pW0 = pb[-W - 1], pC0 = pb[-W], pE0 = pb[-W + dEx];
        T pW1 = pb[-1], pC1 = pb[0], pE1 = pb[dEx];
        T kS0 = kb[0], kS1 = kb[dEc];
        int lS0 = lb[0], lS1 = lb[dEc];
        T zprev = T(0), mqprev = T(0);
        // Element row ky-1 (south of row i) gets this thread's column sum of the node pair
        // (ky-1, ky): only row i's value for i = 0 (the row below belongs to the strip
        // underneath), both for i > 0. The strip's last element row is added after the loop.
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const T pW2 = pb[(i + 1) * W - 1], pC2 = pb[(i + 1) * W], pE2 = pb[(i + 1) * W + dEx];
          const T kN0 = kb[(i + 1) * NEL], kN1 = kb[(i + 1) * NEL + dEc];
          const int lN0 = lb[(i + 1) * NEL], lN1 = lb[(i + 1) * NEL + dEc];
          const bool act = i < nact;
          T qv = q1_apply(kS0, kS1, kN0, kN1, pW0, pC0, pE0, pW1, pC1, pE1, pW2, pC2, pE2);
          qv = act ? qv : T(0);
          q[i] = qv;
          const T mii = mb[i * W];
          const T z = mii * rr[i];
          const T mq = mii * qv;
          pq += pC1 * qv;
          zq += z * qv;
          qmq += qv * mq;
          rz += rr[i] * z;
          const T uz = z + zprev, uq = mq + mqprev;
          add_lab<NC>(azW, lS0, uz);
          add_lab<NC>(azE, lS1, uz);
          add_lab<NC>(aqW, lS0, uq);
          add_lab<NC>(aqE, lS1, uq);
          zprev = z;
          mqprev = mq;
          pW0 = pW1; pC0 = pC1; pE0 = pE1;
          pW1 = pW2; pC1 = pC2; pE1 = pE2;
          kS0 = kN0; kS1 = kN1; lS0 = lN0; lS1 = lN1;
        }
        // element row of the strip's top: lS0/lS1 now hold its labels
        if (!next_row) {
          add_lab<NC>(azW, lS0, zprev);
          add_lab<NC>(azE, lS1, zprev);
          add_lab<NC>(aqW, lS0, mqprev);
          add_lab<NC>(aqE, lS1, mqprev);
        } else if (nact == RPT) {
          atomicAdd(&rb[4 + (lS0 << lgnq) + baseWn], zprev);
          atomicAdd(&rb[4 + (lS1 << lgnq) + baseEn], zprev);
          atomicAdd(&rb[4 + nc + (lS0 << lgnq) + baseWn], mqprev);
          atomicAdd(&rb[4 + nc + (lS1 << lgnq) + baseEn], mqprev);
        }
        flush_bins<NC>(azW, azE, rb + 4, lane, seg, lgnq, baseW, baseE);
        flush_bins<NC>(aqW, aqE, rb + 4 + nc, lane, seg, lgnq, baseW, baseE);
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

        // scalars and multipliers, evaluated by every warp from the same sums
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

        // Ct^T lambda at node (ky) = w(ky-1) + w(ky), w(ey) = lambda of the element row ey's
        // west and east elements of this column
        T wprev = lw[(lb[0] << lgnq) + baseW] + lw[(lb[dEc] << lgnq) + baseE];
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const int lN0 = lb[(i + 1) * NEL], lN1 = lb[(i + 1) * NEL + dEc];
          const bool act = i < nact;
          const bool nr = (i == RPT - 1) && next_row && act;
          const T wcur = lw[(lN0 << lgnq) + (nr ? baseWn : baseW)] +
                         lw[(lN1 << lgnq) + (nr ? baseEn : baseE)];
          const T p0 = pb[i * W];
          x[i] += alpha * p0;
          rr[i] = act ? rr[i] - alpha * q[i] - (wprev + wcur) : T(0);
          const T pn = mb[i * W] * rr[i] + beta * p0;
          if (act && !stop) pb[i * W] = pn;
          wprev = wcur;
        }
        if (stop) {
          if (stop == 2) breakdown = true;
          break;
        }
        push_halo_p();
      }
    }
    iters += (rho0 > T(0)) ? it + 1 : 0;
    C::sync();  // all inner reads finished before the refinement step reuses the buffers
    if (breakdown) break;
  }

  // ---- write the solution
  double *xo = a.x + (size_t)unit * a.nv + kx + (n + 1) * ky0;
#pragma unroll
  for (int i = 0; i < RPT; ++i)
    if (i < nact) xo[i * (n + 1)] = xb[i * W];
  if (a.lam && rank == 0)
    for (int i = tid; i < nc; i += THREADS) a.lam[(size_t)unit * nc + i] = v64[i];
  if (rank == 0 && tid == 0) {
    a.iters[unit] = iters;
    a.sweeps[unit] = sweeps;
    a.ratio[unit] = ratio;
    a.status[unit] = breakdown ? 1 : 0;
  }
  C::sync();  // no CTA leaves while a peer may still read its shared memory
}

template <typename T, int NEL, int RG, int RPT, int CL, bool SR>
size_t level_smem_bytes(int nc) {
  constexpr int THREADS = NEL * RG;
  constexpr int ROWS = RG * RPT;
  const int nred = 4 + 2 * nc;
  return sizeof(double) * ((ROWS + 2) * (NEL + 1) + nc * nc + 2 * nc + 1 + 2 * nc + 2) +
         sizeof(T) * ((ROWS + 2) * (NEL + 1) + (ROWS + 1) * NEL + nc * nc + 2 * nred +
                      (THREADS / 32) * (nred + nc) + ROWS * (NEL + 1)) +
         (ROWS + 1) * NEL + 16 + (SR ? sizeof(double) * ROWS * (NEL + 1) : 0);
}

template <typename T, int NEL, int RG, int RPT, int CL, int NC, int MINB>
cudaError_t launch_level_cfg(const LevelArgs<T> &a, cudaStream_t st) {
  constexpr int THREADS = NEL * RG;
  // keep the FP64 residual on chip when it fits beside everything else
  constexpr bool SR = (size_t)RG * RPT * (NEL + 1) * 8 + 40 * 1024 +
                          (size_t)(RG * RPT + 2) * (NEL + 1) * (8 + sizeof(T)) * 2 <=
                      200 * 1024;
  const size_t smem = level_smem_bytes<T, NEL, RG, RPT, CL, SR>(a.nc);
  auto kern = k_level2d<T, NEL, RG, RPT, CL, NC, MINB, SR>;
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

template <typename T, int NEL, int RG, int RPT, int CL, int MINB>
cudaError_t launch_level_nc(const LevelArgs<T> &a, cudaStream_t st) {
  if (a.N <= 2) return launch_level_cfg<T, NEL, RG, RPT, CL, 2, MINB>(a, st);
  if (a.N == 3) return launch_level_cfg<T, NEL, RG, RPT, CL, 3, MINB>(a, st);
  return launch_level_cfg<T, NEL, RG, RPT, CL, 4, MINB>(a, st);
}

}  // namespace mch
