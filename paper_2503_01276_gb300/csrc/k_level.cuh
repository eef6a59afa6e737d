// Persistent level kernel for the 2D constrained cell problems (template; instantiated per
// inner precision in k_level_f32.cu, k_level_f32_alt.cu and k_level_f64.cu).
//
// One launch solves every (point, cell function) unit of a level to the refinement
// tolerance. A unit is one CTA, or one thread-block cluster of CL CTAs that split the node
// rows into slabs and exchange halo rows and partial sums through distributed shared memory.
// The inner-precision iterates stay on chip for the launch: the search direction (and the
// Chebyshev iterates) with halo rows, kappa, the labels and M^-1 in shared memory; the
// correction, residual and A p in registers. The FP64 solution lives in the output buffer
// (global memory, L2-resident while the unit runs) and is touched only by the refinement
// steps.
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
//   inner sweep: projected PCG in the inner precision from delta = 0 on the constraint
//     null space, S = Ct M^-1 Ct^T, M = diag(A), with the residual kept projected
//     (Ct M^-1 r = 0, so Pi^T r = r for Pi^T = I - Ct^T S^-1 Ct M^-1). Preconditioner
//     B = Pi p(M^-1 A) M^-1 Pi^T, where p(M^-1 A) M^-1 r is NCH steps of the Chebyshev
//     iteration for M^-1 A y = M^-1 r on the fixed interval [1/50, 2] (the Gershgorin bound
//     of M^-1 A for the Q1 stencil is 2), which needs NCH - 1 stencil applications and no
//     reduction; with NCH = 1 it is the Jacobi-weighted projection Pi M^-1 Pi^T.
//     NCH = 1 (one reduction phase and two barriers per iteration):
//       q = A p; one reduction of p.q, z.q, q.M^-1 q, r.z, Ct z, Ct M^-1 q (z = M^-1 r)
//       alpha = rho / p.q,  c = Ct z - alpha Ct M^-1 q,  lambda = S^-1 c
//       delta += alpha p,  r <- r - alpha q - Ct^T lambda
//       rho' = r.z - 2 alpha z.q + alpha^2 q.M^-1 q - lambda.c     (= new r.M^-1 r)
//       p = M^-1 r + (rho'/rho) p
//     NCH > 1 (two reduction phases; NCH + 2 barriers per iteration):
//       y = p(M^-1 A) M^-1 r (Chebyshev, iterates double-buffered in shared memory);
//       reduce r.y and Ct y; mu = S^-1 Ct y; z = y - M^-1 Ct^T mu; rho' = r.z = r.y
//       (because Ct M^-1 r = 0); p = z + (rho'/rho) p;
//       q = A p; reduce p.q and Ct M^-1 q; alpha = rho' / p.q;
//       lambda = alpha S^-1 Ct M^-1 q; delta += alpha p; r <- r - alpha q + Ct^T lambda.
//     The sweep ends when sqrt(rho' / rho_first) < max(tol, 0.3 rtol / ratio), ratio the
//     refinement step's residual ratio: the last sweep stops once rtol is within reach.
// After a reduction's barrier the scalars and multipliers come from the same summed values
// everywhere: in the Jacobi sweep every warp evaluates them itself; in the Chebyshev sweep and
// the refinement steps the CTA gathers the CL partial vectors once and forms the small
// products S^-1 c cooperatively (a row per power-of-two group of threads), then shares them
// through shared memory. Keeping r projected avoids the cancellation that otherwise pushes
// FP32 iterates off the constraint set; the FP64 steps restore the constraints and the true
// residual.
//
// Constraint rows: node k contributes v_k to the row of each of its four adjacent elements;
// row (j, q) of continuum j and sub-block q = by P + bx has index j P^2 + q. A thread's
// column strip has fixed west/east element columns, so west and east contributions are
// accumulated per label in registers (static slots); the east slot of lane c belongs to
// column c+1, whose owner is lane c+1, and is handed over with one shfl_up. Rows per thread
// divide the sub-block size m = n / P (a power of two; P need not be), so all south elements
// of a strip lie in one sub-block row; only the north elements of the strip's last row can
// fall in the next one, and those go through the same warp reduction with the next row's
// bins (flush_next).
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

// Adds a node value to the per-label west/east slots of its four adjacent elements; the
// north elements of an aligned strip's last row (to_next) go to `bins` directly.
// Per-label sums over the element rows of a column strip of the node-pair sums
// v_(i-1) + v_i, for the west and the east element of the column at once, from one running
// prefix Q of the node values: a run of element rows s..e with one label adds
// (Q_e + Q_(e-1)) - (Q_(s-1) + Q_(s-2)), so a node costs one add instead of three (used for
// the FP64 sums of the refinement steps, whose FP64 adds run at a small fraction of the FP32
// rate). Element row i lies between node rows i-1 and i; node row -1 belongs to the strip
// below (its value is added there), so Q starts at zero.
template <int NC>
struct PairRuns {
  double aW[NC], aE[NC];
  double q1, q2;   // Q_(i-1), Q_(i-2)
  double sW, sE;   // Q_(s-1) + Q_(s-2) where the current west / east run started
  int lW, lE;      // labels of the current runs
  __device__ __forceinline__ void init(int lw, int le) {
#pragma unroll
    for (int j = 0; j < NC; ++j) aW[j] = aE[j] = 0.0;
    q1 = q2 = sW = sE = 0.0;
    lW = lw;
    lE = le;
  }
  // element row i, labels (lw, le), gets v_(i-1) + v_i
  __device__ __forceinline__ void step(int lw, int le, double v) {
    if (lw != lW) {
      add_lab<NC>(aW, lW, (q1 + q2) - sW);
      sW = q1 + q2;
      lW = lw;
    }
    if (le != lE) {
      add_lab<NC>(aE, lE, (q1 + q2) - sE);
      sE = q1 + q2;
      lE = le;
    }
    q2 = q1;
    q1 += v;
  }
  __device__ __forceinline__ void close() {
    const double t = q1 + q2;
    add_lab<NC>(aW, lW, t - sW);
    add_lab<NC>(aE, lE, t - sE);
  }
};

// East slots to the owner lane of column c+1 (lane 31 adds its own directly), then sums over
// the lanes that share the west sub-block; the group leader adds to `bins`.
template <int NC, typename V>
__device__ __forceinline__ void flush_bins(V (&aW)[NC], V (&aE)[NC], V *bins, int lane, int seg,
                                           int nq, int baseW, int baseE) {
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    const V up = __shfl_up_sync(0xffffffffu, aE[j], 1);
    if (lane > 0) aW[j] += up;
    if (lane == 31 && aE[j] != V(0)) atomicAdd(&bins[j * nq + baseE], aE[j]);
    const V s = seg_sum(aW[j], seg);
    if ((lane & (seg - 1)) == 0 && s != V(0)) atomicAdd(&bins[j * nq + baseW], s);
  }
}

// The north element row of a strip that ends a sub-block row (pred: next_row with every row
// of the strip active) lies in the next sub-block row: its per-label west/east values go
// through the same warp reduction as the strip's own sums, so that one atomic per segment,
// not one per thread, reaches a bin. Lanes without the predicate add zero; the call is skipped
// by warps where no lane has it.
template <int NC, typename V>
__device__ __forceinline__ void flush_next(bool pred, int lW, int lE, V v, V *bins, int lane,
                                           int seg, int nq, int baseWn, int baseEn) {
  if (!__any_sync(0xffffffffu, pred)) return;
  V nW[NC], nE[NC];
#pragma unroll
  for (int j = 0; j < NC; ++j) nW[j] = nE[j] = V(0);
  const V u = pred ? v : V(0);
  add_lab<NC>(nW, lW, u);
  add_lab<NC>(nE, lE, u);
  flush_bins<NC>(nW, nE, bins, lane, seg, nq, baseWn, baseEn);
}

// Chebyshev coefficients of the preconditioner on [1/50, 2]: y_1 = c0 M^-1 r and, for step
// j = 1 .. NCH-1, d_j = c1[j] d_{j-1} + c2[j] M^-1 (r - A y_j), y_{j+1} = y_j + d_j.
struct ChebCoef {
  float c0, c1[16], c2[16];
};
__host__ __device__ inline ChebCoef cheb_coef(int nch) {
  const double lo = 1.0 / 50.0, hi = 2.0;
  const double th = 0.5 * (hi + lo), de = 0.5 * (hi - lo), sig = th / de;
  ChebCoef c{};
  c.c0 = (float)(1.0 / th);
  double rc = 1.0 / sig;
  for (int j = 1; j < nch && j < 16; ++j) {
    const double rn = 1.0 / (2.0 * sig - rc);
    c.c1[j] = (float)(rn * rc);
    c.c2[j] = (float)(2.0 * rn / de);
    rc = rn;
  }
  return c;
}

template <typename T, int NEL, int RG, int RPT, int CL, int NC, int MINB, bool SR, int NCH>
__global__ void __launch_bounds__(NEL * RG, MINB) k_level2d(LevelArgs<T> a) {
  using C = ClusterOps<CL>;
  constexpr int THREADS = NEL * RG;
  constexpr int NWARPS = THREADS / 32;
  static_assert(THREADS >= MCH_MAX_NC, "the small products give every row a thread");
  constexpr int ROWS = RG * RPT;
  constexpr int W = NEL + 1;
  constexpr int YB = (ROWS + 2) * W;                  // one halo-padded slab
  constexpr int NYB = NCH > 1 ? 2 : 0;                // Chebyshev iterate buffers
  const int n = NEL;
  const int XW = n + 1;                               // lattice row stride of x, b, M^-1
  const int unit = blockIdx.x / CL;
  const int rank = C::rank();
  const int pt = unit / a.R, rfun = unit % a.R;
  const int nc = a.nc;
  const int NRED = NCH > 1 ? 1 + nc : 4 + 2 * nc;
  const int P = a.P, nq = a.P * a.P;
  const int m = n / P;
  const int seg = m < 32 ? m : 32;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *sinv64 = reinterpret_cast<double *>(smem_raw);  // [nc][nc]
  double *red64 = sinv64 + nc * nc;                   // [2 nc + 1] FP64 partial sums
  double *v64 = red64 + 2 * nc + 1;                   // [2 nc] mu, lambda
  double *rs = v64 + 2 * nc;                          // [ROWS][W] FP64 residual when SR
  T *ps = reinterpret_cast<T *>(rs + (SR ? ROWS * W : 0));  // [(ROWS+2)][W] search direction
  T *yb = ps + YB;                                    // [NYB][(ROWS+2)][W] Chebyshev iterates
  T *ks = yb + NYB * YB;                              // [(ROWS+1)][NEL] kappa rows r_lo-1..
  T *sinv = ks + (ROWS + 1) * NEL;                    // [nc][nc] (symmetric)
  T *red = sinv + nc * nc;                            // [2][NRED] (two reduction buffers)
  constexpr int NSC = NCH > 1 ? 1 : NWARPS;            // copies of the gathered sums
  T *twarp = red + 2 * NRED;                          // [NSC][NRED]
  T *lamw = twarp + NSC * NRED;                       // [NSC][nc]
  T *mis = lamw + NSC * nc;                           // [ROWS][W] M^-1 of own rows
  T *chc = mis + ROWS * W;                            // [2][16] Chebyshev coefficients
  uint8_t *ls = reinterpret_cast<uint8_t *>(chc + 32);  // [(ROWS+1)][NEL]

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int c = tid % NEL, g = tid / NEL;
  const int G = rank * RG + g;
  const int r_lo = 1 + rank * ROWS;
  const int kx = c + 1;
  const int kxE = kx + 1 <= n ? kx + 1 : n;   // clamp for the inactive last lane
  const int cE = c + 1 <= n - 1 ? c + 1 : n - 1;
  const bool col_active = c < n - 1;
  const int bxW = c / m, bxE = cE / m;
  const int bym = (G * RPT) / m;
  const bool next_row = ((G + 1) * RPT) % m == 0;
  const int baseW = bym * P + bxW, baseE = bym * P + bxE;
  const int baseWn = (bym + 1) * P + bxW, baseEn = (bym + 1) * P + bxE;

  // ---- load the unit's data; the FP64 solution starts at zero everywhere (boundary and
  // padding entries included)
  const double *kap = a.kappa + (size_t)pt * n * n;
  const uint8_t *lab = a.labels + (size_t)pt * n * n;
  const double *mv64 = a.minv64 + (size_t)pt * a.nv;
  const double *bvec = a.b ? a.b + (size_t)unit * a.nv : nullptr;
  const double *gt = a.g + (size_t)pt * nc * a.R + rfun;  // stride R
  double *xg = a.x + (size_t)unit * a.nv;
  // FP64 residual of step (d) kept for step (e) when it does not fit in shared memory (else
  // the FP64 stencil runs twice per refinement step)
  double *r64g = (!SR && a.r64) ? a.r64 + (size_t)unit * a.nv : nullptr;
  for (int t = rank * THREADS + tid; t < a.nv; t += CL * THREADS) xg[t] = 0.0;
  for (int t = tid; t < (1 + NYB) * YB; t += THREADS) ps[t] = T(0);
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
  if (tid == 0) {
    const ChebCoef cc = cheb_coef(NCH);
    chc[0] = T(cc.c0);
    for (int j = 1; j < 16; ++j) {
      chc[j] = T(cc.c1[j]);
      chc[16 + j] = T(cc.c2[j]);
    }
  }
  for (int t = tid; t < 2 * NRED; t += THREADS) red[t] = T(0);
  for (int t = tid; t < 2 * nc + 1; t += THREADS) red64[t] = 0.0;
  C::sync();  // x zeroed cluster-wide, shared data in place

  // Per-thread base pointers: row i of the strip is at a compile-time offset from these.
  const int row0 = 1 + g * RPT;                    // first own row in the local arrays
  const int dEx = kxE - kx;                        // 1, or 0 for the inactive last lane
  const int dEc = cE - c;
  const int ky0 = r_lo + row0 - 1;                 // global node row of local row row0
  const int nact = col_active ? max(0, min(RPT, n - ky0)) : 0;  // active rows of the strip
  T *pb = ps + row0 * W + kx;                      // p at (row i, own column): pb[i*W]
  double *xb = xg + kx + XW * ky0;                 // FP64 x at row i: xb[i*XW]
  T *mb = mis + (row0 - 1) * W + kx;               // M^-1 of row i: mb[i*W]
  const T *kb = ks + (row0 - 1) * NEL + c;         // kappa of element row (ky-1): kb[i*NEL]
  const uint8_t *lb = ls + (row0 - 1) * NEL + c;   // labels likewise
  const double *kg = kap + c + n * (ky0 - 1);      // FP64 kappa of element row (ky-1): kg[i*n]
  const double *mg = mv64 + kx + XW * ky0;         // FP64 M^-1 of row i: mg[i*XW]
  const double *bg = bvec ? bvec + kx + XW * ky0 : nullptr;

  T x[RPT], rr[RPT], q[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    x[i] = T(0);
    rr[i] = T(0);
    q[i] = T(0);
    const T dg = q1_diag(kb[i * NEL], kb[i * NEL + dEc], kb[(i + 1) * NEL], kb[(i + 1) * NEL + dEc]);
    mb[i * W] = (i < nact) ? T(1) / dg : T(0);   // each thread reads only its own entries
  }
  // gathered sums and multipliers: per warp in the Jacobi sweep (every warp evaluates them
  // itself), shared by the CTA in the Chebyshev sweep (evaluated cooperatively)
  T *tw = twarp + (NCH > 1 ? 0 : warp) * NRED;
  T *lw = lamw + (NCH > 1 ? 0 : warp) * nc;

  // halo rows of a shared-memory slab (p or a Chebyshev iterate) to the neighbouring CTAs
  auto push_halo = [&](T *slab) {
    if constexpr (CL > 1) {
      if (g == 0 && rank > 0) C::remote(slab, rank - 1)[(ROWS + 1) * W + kx] = slab[1 * W + kx];
      if (g == RG - 1 && rank < CL - 1) C::remote(slab, rank + 1)[kx] = slab[ROWS * W + kx];
    }
  };
  // Small products S^-1 v by the whole CTA: row i of S^-1 (symmetric) goes to KS consecutive
  // threads (KS a power of two with KS nc <= THREADS, at most 32), each summing every KS-th
  // term, then a KS-lane butterfly; so the work is spread over the CTA instead of repeated
  // by every warp, and no row is a long serial chain.
  const int KS = [&] {
    int k = 1;
    while (k < 32 && 2 * k * nc <= THREADS) k *= 2;
    return k;
  }();
  const int srow = tid / KS, spart = tid % KS;
  // small FP64 product out = S^-1 v (v, out in shared memory)
  auto small64 = [&](const double *v, double *out) {
    double s = 0.0;
    if (srow < nc)
      for (int j = spart; j < nc; j += KS) s += sinv64[srow * nc + j] * v[j];
    for (int o = KS >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (spart == 0 && srow < nc) out[srow] = s;
  };
  // the CL partial vectors of buffer rb summed into tw[0..cnt) by the CTA (one thread per
  // entry; the caller synchronises the CTA before tw is read)
  auto gather_cta = [&](const T *rb, int cnt) {
    for (int t = tid; t < cnt; t += THREADS) {
      T v = T(0);
#pragma unroll
      for (int rk = 0; rk < CL; ++rk) v += C::remote(rb, rk)[t];
      tw[t] = v;
    }
  };
  // lw = scale S^-1 tw[off ..) (or 0 when zero) by the CTA, rows as in small64
  auto small_cta = [&](int off, T scale, bool zero) {
    T s = T(0);
    if (srow < nc)
      for (int j = spart; j < nc; j += KS) s += sinv[srow * nc + j] * tw[off + j];
    for (int o = KS >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (spart == 0 && srow < nc) lw[srow] = zero ? T(0) : scale * s;
  };
  // inner-precision product lw = scale * S^-1 v (v = tw + off) by every warp for itself;
  // returns scale * lw . v summed over the warp (used by the Jacobi sweep)
  auto small_warp = [&](int off, T scale, bool zero) {
    T lc = T(0);
    for (int i = lane; i < nc; i += 32) {
      // S^-1 is symmetric: column i is read so that consecutive lanes hit distinct banks
      T l0 = T(0), l1 = T(0), l2 = T(0), l3 = T(0);
      int j = 0;
      for (; j + 3 < nc; j += 4) {
        l0 += sinv[(j + 0) * nc + i] * tw[off + j + 0];
        l1 += sinv[(j + 1) * nc + i] * tw[off + j + 1];
        l2 += sinv[(j + 2) * nc + i] * tw[off + j + 2];
        l3 += sinv[(j + 3) * nc + i] * tw[off + j + 3];
      }
      for (; j < nc; ++j) l0 += sinv[j * nc + i] * tw[off + j];
      const T l = scale * ((l0 + l1) + (l2 + l3));
      lw[i] = zero ? T(0) : l;
      lc += l * tw[off + i];
    }
    return warp_sum(lc);
  };
  // every warp sums the CL partial vectors of buffer rb into tw[0..cnt)
  auto gather = [&](const T *rb, int cnt) {
    for (int t = lane; t < cnt; t += 32) {
      T v = T(0);
      for (int rk = 0; rk < CL; ++rk) v += C::remote(rb, rk)[t];
      tw[t] = v;
    }
    __syncwarp();
  };
  // Ct^T w at own row i from the element-row values w(ky-1) (wprev) and w(ky) (wcur):
  // wcur(i) = w[label W] + w[label E] of element row ky, in the next sub-block row for the
  // strip's last row when it ends a sub-block
  auto wrow = [&](const auto *w, int lN0, int lN1, bool nr) {
    return w[lN0 * nq + (nr ? baseWn : baseW)] + w[lN1 * nq + (nr ? baseEn : baseE)];
  };
  // Ct v of a node vector held per own row in registers: per-label element-row sums into
  // the bins (shared memory), plus the dot product sum_i da[i] db[i] into *dot
  auto ct_reduce = [&](const T (&v)[RPT], const T (&da)[RPT], const T (&db)[RPT], T *bins,
                       T *dot) {
    T aW[NC], aE[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) aW[j] = aE[j] = T(0);
    T dsum = T(0);
    int lS0 = lb[0], lS1 = lb[dEc];
    T vprev = T(0);
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int lN0 = lb[(i + 1) * NEL], lN1 = lb[(i + 1) * NEL + dEc];
      dsum += da[i] * db[i];
      const T u = v[i] + vprev;
      add_lab<NC>(aW, lS0, u);
      add_lab<NC>(aE, lS1, u);
      vprev = v[i];
      lS0 = lN0;
      lS1 = lN1;
    }
    if (!next_row) {
      add_lab<NC>(aW, lS0, vprev);
      add_lab<NC>(aE, lS1, vprev);
    }
    flush_next<NC>(next_row && nact == RPT, lS0, lS1, vprev, bins, lane, seg, nq,
                   baseWn, baseEn);
    flush_bins<NC>(aW, aE, bins, lane, seg, nq, baseW, baseE);
    dsum = warp_sum(dsum);
    if (lane == 0) atomicAdd(dot, dsum);
  };

  double rho64_first = 0.0, ratio = 0.0;
  int sweeps = 0, iters = 0;
  bool breakdown = false, done = false;

  for (int step = 0;; ++step) {
    // ================= FP64 refinement step =================
    // (a) fold the correction; (b) Ct x by element rows (column sums of node pairs). The
    // first step starts from x = 0, where both are zero.
    if (step > 0) {
      PairRuns<NC> pr;
      pr.init(lb[0], lb[dEc]);
      double vprev = 0.0;
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        double v = 0.0;
        if (i < nact) {
          v = xb[i * XW] + (double)x[i];
          xb[i * XW] = v;
        }
        x[i] = T(0);
        pr.step(lb[i * NEL], lb[i * NEL + dEc], v);
        vprev = v;
      }
      const int lT0 = lb[RPT * NEL], lT1 = lb[RPT * NEL + dEc];
      if (!next_row) pr.step(lT0, lT1, 0.0);
      flush_next<NC>(next_row && nact == RPT, lT0, lT1, vprev, red64, lane, seg, nq,
                     baseWn, baseEn);
      pr.close();
      flush_bins<NC>(pr.aW, pr.aE, red64, lane, seg, nq, baseW, baseE);
    }
    C::sync();
    // mu = S^-1 (g - Ct x)
    for (int b = tid; b < nc; b += THREADS) {
      double s = 0.0;
      for (int rk = 0; rk < CL; ++rk) s += C::remote(red64, rk)[b];
      v64[nc + b] = gt[(size_t)b * a.R] - s;
    }
    __syncthreads();
    small64(v64 + nc, v64);
    __syncthreads();
    // (c) x += M^-1 Ct^T mu
    {
      double wprev = v64[lb[0] * nq + baseW] + v64[lb[dEc] * nq + baseE];
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int lN0 = lb[(i + 1) * NEL], lN1 = lb[(i + 1) * NEL + dEc];
        const bool act = i < nact;
        const bool nr = (i == RPT - 1) && next_row && act;
        const double wcur = wrow(v64, lN0, lN1, nr);
        if (act) xb[i * XW] += mg[i * XW] * (wprev + wcur);
        wprev = wcur;
      }
    }
    C::sync();  // x final for this step cluster-wide; every rank has read red64[0..nc)
    // (d) Ct M^-1 r with r = b - A x (FP64); r kept in shared memory when SR, else formed
    // again in (e)
    {
      // strips wholly beyond the last node row (nact = 0) read nothing from global memory
      const bool any = nact > 0;
      double xW0 = any ? xb[-XW - 1] : 0.0, xC0 = any ? xb[-XW] : 0.0;
      double xE0 = any ? xb[-XW + dEx] : 0.0, xW1 = any ? xb[-1] : 0.0;
      double xC1 = any ? xb[0] : 0.0, xE1 = any ? xb[dEx] : 0.0;
      double kS0 = any ? kg[0] : 0.0, kS1 = any ? kg[dEc] : 0.0;
      double sS = kS0 + kS1;      // kappa sum of the south element pair (the previous north)
      PairRuns<NC> pr;
      pr.init(lb[0], lb[dEc]);
      double zprev = 0.0;
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const bool act = i < nact;
        double xW2 = 0.0, xC2 = 0.0, xE2 = 0.0;
        if (act) {
          xW2 = xb[(i + 1) * XW - 1];
          xC2 = xb[(i + 1) * XW];
          xE2 = xb[(i + 1) * XW + dEx];
        }
        const double kN0 = act ? kg[(i + 1) * n] : 0.0, kN1 = act ? kg[(i + 1) * n + dEc] : 0.0;
        const double sN = kN0 + kN1;
        double zm = 0.0;
        if (act) {
          // the Q1 stencil (as q1_apply) with the element-pair kappa sums carried over rows
          const double t = 4.0 * (sS + sN) * xC1 - (kS1 + kN1) * xE1 - (kS0 + kN0) * xW1 -
                           sN * xC2 - sS * xC0 -
                           2.0 * (kN1 * xE2 + kN0 * xW2 + kS1 * xE0 + kS0 * xW0);
          const double rv = (bg ? bg[i * XW] : 0.0) - t * (1.0 / 6.0);
          if constexpr (SR) rs[(g * RPT + i) * W + kx] = rv;
          else if (r64g) r64g[kx + XW * (ky0 + i)] = rv;
          zm = mg[i * XW] * rv;
        }
        pr.step(lb[i * NEL], lb[i * NEL + dEc], zm);
        zprev = zm;
        xW0 = xW1; xC0 = xC1; xE0 = xE1;
        xW1 = xW2; xC1 = xC2; xE1 = xE2;
        kS0 = kN0; kS1 = kN1; sS = sN;
      }
      const int lT0 = lb[RPT * NEL], lT1 = lb[RPT * NEL + dEc];
      if (!next_row) pr.step(lT0, lT1, 0.0);
      flush_next<NC>(next_row && nact == RPT, lT0, lT1, zprev, red64 + nc, lane, seg, nq,
                     baseWn, baseEn);
      pr.close();
      flush_bins<NC>(pr.aW, pr.aE, red64 + nc, lane, seg, nq, baseW, baseE);
    }
    C::sync();
    for (int b = tid; b < nc; b += THREADS) {
      double s = 0.0;
      for (int rk = 0; rk < CL; ++rk) s += C::remote(red64, rk)[nc + b];
      v64[nc + b] = s;
    }
    __syncthreads();
    small64(v64 + nc, v64);
    __syncthreads();
    // (e) projected residual, its M^-1 norm; the next sweep's residual
    {
      double rho_p = 0.0;
      double xW0 = 0, xC0 = 0, xE0 = 0, xW1 = 0, xC1 = 0, xE1 = 0, kS0 = 0, kS1 = 0;
      if constexpr (!SR) {
        if (nact > 0 && !r64g) {
          xW0 = xb[-XW - 1]; xC0 = xb[-XW]; xE0 = xb[-XW + dEx];
          xW1 = xb[-1]; xC1 = xb[0]; xE1 = xb[dEx];
          kS0 = kg[0]; kS1 = kg[dEc];
        }
      }
      double wprev = v64[lb[0] * nq + baseW] + v64[lb[dEc] * nq + baseE];
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const bool act = i < nact;
        const int lN0 = lb[(i + 1) * NEL], lN1 = lb[(i + 1) * NEL + dEc];
        const bool nr = (i == RPT - 1) && next_row && act;
        const double wcur = wrow(v64, lN0, lN1, nr);
        double rv = 0.0;
        if constexpr (SR) {
          if (act) rv = rs[(g * RPT + i) * W + kx];
        } else if (r64g) {
          if (act) rv = r64g[kx + XW * (ky0 + i)];
        } else {
          double xW2 = 0.0, xC2 = 0.0, xE2 = 0.0;
          if (act) {
            xW2 = xb[(i + 1) * XW - 1];
            xC2 = xb[(i + 1) * XW];
            xE2 = xb[(i + 1) * XW + dEx];
          }
          const double kN0 = act ? kg[(i + 1) * n] : 0.0, kN1 = act ? kg[(i + 1) * n + dEc] : 0.0;
          if (act)
            rv = (bg ? bg[i * XW] : 0.0) -
                 q1_apply(kS0, kS1, kN0, kN1, xW0, xC0, xE0, xW1, xC1, xE1, xW2, xC2, xE2);
          xW0 = xW1; xC0 = xC1; xE0 = xE1;
          xW1 = xW2; xC1 = xC2; xE1 = xE2;
          kS0 = kN0; kS1 = kN1;
        }
        double rt = 0.0;
        if (act) {
          rt = rv - (wprev + wcur);
          rho_p += rt * rt * mg[i * XW];
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
    // the sweep's reduction target: the inner tolerance, relaxed once the refinement
    // tolerance is within reach (0.3 rtol / ratio), so that the last sweep does not solve
    // further than the refinement step needs
    const T tol_s = T(fmax((double)a.tol, fmin(0.5, 0.3 * a.rtol / ratio)));

    // ================= inner PCG sweep =================
    C::sync();  // every rank has read red64; clear it and the inner buffers for reuse
    for (int t = tid; t < 2 * nc + 1; t += THREADS) red64[t] = 0.0;
    for (int t = tid; t < 2 * NRED; t += THREADS) red[t] = T(0);
    __syncthreads();
    ++sweeps;
    if constexpr (NCH == 1) {
      T dz = T(0);
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const T z = mb[i * W] * rr[i];
        dz += rr[i] * z;
        if (i < nact) pb[i * W] = z;
      }
      push_halo(ps);
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
          }
          flush_next<NC>(next_row && nact == RPT, lS0, lS1, zprev, rb + 4, lane, seg, nq, baseWn,
                         baseEn);
          flush_next<NC>(next_row && nact == RPT, lS0, lS1, mqprev, rb + 4 + nc, lane, seg, nq,
                         baseWn, baseEn);
          flush_bins<NC>(azW, azE, rb + 4, lane, seg, nq, baseW, baseE);
          flush_bins<NC>(aqW, aqE, rb + 4 + nc, lane, seg, nq, baseW, baseE);
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
          gather(rb, NRED);
          const T tpq = tw[0], tzq = tw[1], tqmq = tw[2], trz = tw[3];
          T alpha = rho / tpq;
          const bool bad = !(tpq > T(0)) || !(alpha == alpha) || !(alpha < T(3.0e38));
          if (bad) alpha = T(0);
          __syncwarp();
          for (int t = lane; t < nc; t += 32) tw[4 + t] = tw[4 + t] - alpha * tw[4 + nc + t];
          __syncwarp();
          const T lc = small_warp(4, T(1), bad);
          __syncwarp();
          const T rho_new = trz - T(2) * alpha * tzq + alpha * alpha * tqmq - lc;
          int stop = 0;
          if (bad) stop = 2;
          else if (!(rho_new > tol_s * tol_s * rho0)) stop = 1;
          else if (it + 1 >= a.max_iter) stop = 1;
          const T beta = stop ? T(0) : rho_new / rho;
          rho = rho_new;

          // Ct^T lambda at node (ky) = w(ky-1) + w(ky), w(ey) = lambda of the element row ey's
          // west and east elements of this column
          T wprev = lw[lb[0] * nq + baseW] + lw[lb[dEc] * nq + baseE];
#pragma unroll
          for (int i = 0; i < RPT; ++i) {
            const int lN0 = lb[(i + 1) * NEL], lN1 = lb[(i + 1) * NEL + dEc];
            const bool act = i < nact;
            const bool nr = (i == RPT - 1) && next_row && act;
            const T wcur = wrow(lw, lN0, lN1, nr);
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
          push_halo(ps);
        }
      }
      iters += (rho0 > T(0)) ? it + 1 : 0;
    } else {
      // Chebyshev-preconditioned sweep: red[0..NRED) holds p.q and Ct M^-1 q, red[NRED..)
      // holds r.y and Ct y
      T *r1 = red, *r2 = red + NRED;
      T rho = T(0), rho0 = T(0);
      int it = 0;
      for (;; ++it) {
        // ---- y = p(M^-1 A) M^-1 r: y_1 = c0 M^-1 r, then NCH - 1 stencil steps
        T yv[RPT], dv[RPT];
        {
          const T c0 = chc[0];
          T *yo = yb + row0 * W + kx;
#pragma unroll
          for (int i = 0; i < RPT; ++i) {
            dv[i] = c0 * mb[i * W] * rr[i];     // 0 on inactive rows (M^-1 entry 0)
            yv[i] = dv[i];
            if (i < nact) yo[i * W] = yv[i];
          }
          push_halo(yb);
        }
#pragma unroll 1
        for (int j = 1; j < NCH; ++j) {
          C::sync();  // y_j and its halo visible; the other buffer's readers are done
          const T *ys = yb + ((j - 1) & 1) * YB + row0 * W + kx;
          T *yd = yb + (j & 1) * YB + row0 * W + kx;
          const T c1 = chc[j], c2 = chc[16 + j];
          const bool keep = j < NCH - 1;
          T yW0 = ys[-W - 1], yC0 = ys[-W], yE0 = ys[-W + dEx];
          T yW1 = ys[-1], yC1 = ys[0], yE1 = ys[dEx];
          T kS0 = kb[0], kS1 = kb[dEc];
#pragma unroll
          for (int i = 0; i < RPT; ++i) {
            const T yW2 = ys[(i + 1) * W - 1], yC2 = ys[(i + 1) * W], yE2 = ys[(i + 1) * W + dEx];
            const T kN0 = kb[(i + 1) * NEL], kN1 = kb[(i + 1) * NEL + dEc];
            const T ay = q1_apply(kS0, kS1, kN0, kN1, yW0, yC0, yE0, yW1, yC1, yE1, yW2, yC2, yE2);
            const T res = mb[i * W] * (rr[i] - ay);
            dv[i] = c1 * dv[i] + c2 * res;
            yv[i] += dv[i];
            if (keep && i < nact) yd[i * W] = yv[i];
            yW0 = yW1; yC0 = yC1; yE0 = yE1;
            yW1 = yW2; yC1 = yC2; yE1 = yE2;
            kS0 = kN0; kS1 = kN1;
          }
          if (keep) push_halo(yb + (j & 1) * YB);
        }
        // ---- r.y and Ct y
        ct_reduce(yv, rr, yv, r2 + 1, r2);
        C::sync();  // B3: sums in place; every CTA has read the previous r1
        for (int t = tid; t < NRED; t += THREADS) r1[t] = T(0);
        gather_cta(r2, NRED);
        __syncthreads();
        const T rho_new = tw[0];
        small_cta(1, T(1), false);    // lw = mu = S^-1 Ct y
        __syncthreads();
        int stop = 0;
        if (!(rho_new >= T(0)) || !(rho_new < T(3.0e38))) stop = 2;
        else if (it == 0) {
          rho0 = rho_new;
          if (!(rho0 > T(0))) stop = 1;
        } else if (!(rho_new > tol_s * tol_s * rho0)) stop = 1;
        if (!stop && it >= a.max_iter) stop = 1;
        if (stop) {
          if (stop == 2) breakdown = true;
          break;
        }
        const T beta = it == 0 ? T(0) : rho_new / rho;
        rho = rho_new;
        // ---- z = y - M^-1 Ct^T mu; p = z + beta p
        {
          T wprev = lw[lb[0] * nq + baseW] + lw[lb[dEc] * nq + baseE];
#pragma unroll
          for (int i = 0; i < RPT; ++i) {
            const int lN0 = lb[(i + 1) * NEL], lN1 = lb[(i + 1) * NEL + dEc];
            const bool act = i < nact;
            const bool nr = (i == RPT - 1) && next_row && act;
            const T wcur = wrow(lw, lN0, lN1, nr);
            const T z = yv[i] - mb[i * W] * (wprev + wcur);
            const T pn = it == 0 ? z : z + beta * pb[i * W];
            if (act) pb[i * W] = pn;
            wprev = wcur;
          }
          push_halo(ps);
        }
        C::sync();  // B1: p and its halo visible; r1 cleared
        // ---- q = A p; p.q and Ct M^-1 q, accumulated in the same pass over the rows (no
        // per-row arrays of M^-1 q and p are kept)
        {
          T aW[NC], aE[NC];
#pragma unroll
          for (int j = 0; j < NC; ++j) aW[j] = aE[j] = T(0);
          T pq = T(0), mqprev = T(0);
          int lS0 = lb[0], lS1 = lb[dEc];
          T pW0 = pb[-W - 1], pC0 = pb[-W], pE0 = pb[-W + dEx];
          T pW1 = pb[-1], pC1 = pb[0], pE1 = pb[dEx];
          T kS0 = kb[0], kS1 = kb[dEc];
#pragma unroll
          for (int i = 0; i < RPT; ++i) {
            const T pW2 = pb[(i + 1) * W - 1], pC2 = pb[(i + 1) * W], pE2 = pb[(i + 1) * W + dEx];
            const T kN0 = kb[(i + 1) * NEL], kN1 = kb[(i + 1) * NEL + dEc];
            const int lN0 = lb[(i + 1) * NEL], lN1 = lb[(i + 1) * NEL + dEc];
            T qv = q1_apply(kS0, kS1, kN0, kN1, pW0, pC0, pE0, pW1, pC1, pE1, pW2, pC2, pE2);
            qv = i < nact ? qv : T(0);
            q[i] = qv;
            const T mq = mb[i * W] * qv;
            pq += pC1 * qv;
            const T u = mq + mqprev;
            add_lab<NC>(aW, lS0, u);
            add_lab<NC>(aE, lS1, u);
            mqprev = mq;
            pW0 = pW1; pC0 = pC1; pE0 = pE1;
            pW1 = pW2; pC1 = pC2; pE1 = pE2;
            kS0 = kN0; kS1 = kN1;
            lS0 = lN0; lS1 = lN1;
          }
          if (!next_row) {
            add_lab<NC>(aW, lS0, mqprev);
            add_lab<NC>(aE, lS1, mqprev);
          }
          flush_next<NC>(next_row && nact == RPT, lS0, lS1, mqprev, r1 + 1, lane, seg, nq,
                         baseWn, baseEn);
          flush_bins<NC>(aW, aE, r1 + 1, lane, seg, nq, baseW, baseE);
          pq = warp_sum(pq);
          if (lane == 0) atomicAdd(&r1[0], pq);
        }
        // every CTA read r2 (after B3) before B1, so it can be cleared for the next use
        for (int t = tid; t < NRED; t += THREADS) r2[t] = T(0);
        C::sync();  // B2
        gather_cta(r1, NRED);
        __syncthreads();
        const T tpq = tw[0];
        T alpha = rho / tpq;
        const bool bad = !(tpq > T(0)) || !(alpha == alpha) || !(alpha < T(3.0e38));
        if (bad) alpha = T(0);
        small_cta(1, alpha, bad);     // lw = lambda = alpha S^-1 Ct M^-1 q
        __syncthreads();
        {
          T wprev = lw[lb[0] * nq + baseW] + lw[lb[dEc] * nq + baseE];
#pragma unroll
          for (int i = 0; i < RPT; ++i) {
            const int lN0 = lb[(i + 1) * NEL], lN1 = lb[(i + 1) * NEL + dEc];
            const bool act = i < nact;
            const bool nr = (i == RPT - 1) && next_row && act;
            const T wcur = wrow(lw, lN0, lN1, nr);
            x[i] += alpha * pb[i * W];
            rr[i] = act ? rr[i] - alpha * q[i] + (wprev + wcur) : T(0);
            wprev = wcur;
          }
        }
        if (bad) {
          breakdown = true;
          break;
        }
      }
      iters += it;
    }
    C::sync();  // all inner reads finished before the refinement step reuses the buffers
    if (breakdown) break;
  }

  // ---- the solution is in place (xg); multipliers and the convergence record
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

// Dynamic shared memory of a launch shape for nc constraint rows.
template <typename T, int NEL, int RG, int RPT, int CL, bool SR, int NCH>
constexpr size_t level_smem_bytes(int nc) {
  constexpr int THREADS = NEL * RG;
  constexpr int ROWS = RG * RPT;
  constexpr int W = NEL + 1;
  const int nred = NCH > 1 ? 1 + nc : 4 + 2 * nc;
  return sizeof(double) * ((size_t)nc * nc + 2 * nc + 1 + 2 * nc + (SR ? ROWS * W : 0)) +
         sizeof(T) * ((size_t)(NCH > 1 ? 3 : 1) * (ROWS + 2) * W + (ROWS + 1) * NEL + nc * nc +
                      2 * nred + (NCH > 1 ? 1 : THREADS / 32) * (nred + nc) + ROWS * W + 32) +
         (size_t)(ROWS + 1) * NEL;
}

// Keep the FP64 residual on chip when the shape still fits MINB CTAs per SM with the
// largest constraint count (228 KB of shared memory per SM, 1 KB reserved per CTA).
template <typename T, int NEL, int RG, int RPT, int CL, int MINB, int NCH>
constexpr bool level_keeps_residual() {
  return (level_smem_bytes<T, NEL, RG, RPT, CL, true, NCH>(MCH_MAX_NC) + 1024) * MINB <=
         228 * 1024;
}

template <typename T, int NEL, int RG, int RPT, int CL, int NC, int MINB, int NCH>
cudaError_t launch_level_cfg(const LevelArgs<T> &a, cudaStream_t st) {
  constexpr int THREADS = NEL * RG;
  constexpr bool SR = level_keeps_residual<T, NEL, RG, RPT, CL, MINB, NCH>();
  const size_t smem = level_smem_bytes<T, NEL, RG, RPT, CL, SR, NCH>(a.nc);
  auto kern = k_level2d<T, NEL, RG, RPT, CL, NC, MINB, SR, NCH>;
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

template <typename T, int NEL, int RG, int RPT, int CL, int MINB, int NCH = 1>
cudaError_t launch_level_nc(const LevelArgs<T> &a, cudaStream_t st) {
  if (a.N <= 2) return launch_level_cfg<T, NEL, RG, RPT, CL, 2, MINB, NCH>(a, st);
  if (a.N == 3) return launch_level_cfg<T, NEL, RG, RPT, CL, 3, MINB, NCH>(a, st);
  return launch_level_cfg<T, NEL, RG, RPT, CL, 4, MINB, NCH>(a, st);
}

}  // namespace mch
