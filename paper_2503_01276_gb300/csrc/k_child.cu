// Level-1-grid (fine) work of a child level and the Gram reductions.
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
//
// Every kernel is a template over the storage of the level-1-grid vectors: FP64 (the FP64
// mode) or float-float planes (ff.cuh; the mixed mode), whose arithmetic runs on the FP32
// pipes. Level-grid vectors (x, b), kappa, the targets and E stay FP64.
#include <type_traits>

#include "common.cuh"
#include "ff.cuh"
#include "kernels.h"

namespace mch {

namespace {

template <class S>
__device__ __forceinline__ typename S::V seg_sum_s(typename S::V v, int seg) {
  for (int o = seg >> 1; o > 0; o >>= 1) v = v + S::shfl_xor(v, o);
  return v;
}

template <int NC, class S>
__device__ __forceinline__ void add_lab_s(typename S::V (&acc)[NC], int lab, typename S::V v) {
#pragma unroll
  for (int j = 0; j < NC; ++j) acc[j] += (lab == j) ? v : S::zero();
}

constexpr int CF_THREADS = 256;
constexpr int CF_BR = 16;   // fine rows per band

// A_1 x at a level-1 node: the Q1 stencil (element matrix entries 2/3 on the diagonal, -1/6
// for an edge neighbour, -1/3 for the opposite corner; h^(d-2) = 1 in 2D) from the kappa of
// the node's four elements (a SW, b SE, c NW, d NE) and the 3x3 values around it (tr points
// at the node, rows W apart), as one sum of nine products:
//   4 (a+b+c+d) x0 - (b+d) xE - (a+c) xW - (c+d) xN - (a+b) xS
//   - 2 (d xNE + c xNW + b xSE + a xSW), times 1/6.
template <class S>
__device__ __forceinline__ typename S::V q1_dot(typename S::V a, typename S::V b,
                                                typename S::V c, typename S::V d,
                                                const typename S::V *tr, int W,
                                                typename S::V sixth) {
  using V = typename S::V;
  const V ab = a + b, cd = c + d;
  typename S::D t = S::dzero();
  S::dadd(t, S::scale2(ab + cd, 4.f), tr[0]);
  S::dadd(t, -(b + d), tr[1]);
  S::dadd(t, -(a + c), tr[-1]);
  S::dadd(t, -cd, tr[W]);
  S::dadd(t, -ab, tr[-W]);
  S::dadd(t, S::scale2(d, -2.f), tr[W + 1]);
  S::dadd(t, S::scale2(c, -2.f), tr[W - 1]);
  S::dadd(t, S::scale2(b, -2.f), tr[-W + 1]);
  S::dadd(t, S::scale2(a, -2.f), tr[-W - 1]);
  return S::dget(t) * sixth;
}

template <int NC, class S>
__global__ void __launch_bounds__(CF_THREADS, 4) k_child_fine2d(ChildArgs a) {
  using V = typename S::V;
  const int unit = blockIdx.y;
  const int pt = unit / a.R, r = unit % a.R;
  const int nf = a.nf, W = nf + 1, lgr = a.lgr, ncg = nf >> lgr;
  const int band = blockIdx.x;
  const int row_lo = band * CF_BR;                 // first own lattice row
  const int row_hi = min(row_lo + CF_BR, nf + 1);  // one past the last own row
  __shared__ V tile[(CF_BR + 2) * 257];
  __shared__ double bins[MCH_MAX_NC];
  __shared__ typename S::P pp[4];
  __shared__ V pw[4];
  __shared__ int nslot;
  const int tid = threadIdx.x;
  if (tid == 0) {
    // the parents with a cell function, packed to the front
    int ns = 0;
    for (int s = 0; s < a.slots && s < 4; ++s) {
      const double *b = a.par_ptr[pt * a.slots + s];
      if (!b) continue;
      pp[ns] = S::vec(b, r, a.nvf);
      pw[ns] = S::from(a.par_w[pt * a.slots + s]);
      ++ns;
    }
    nslot = ns;
  }
  for (int t = tid; t < a.nc; t += CF_THREADS) bins[t] = 0.0;
  __syncthreads();

  // I on rows row_lo-1 .. row_lo+CF_BR (rows outside the lattice are zero); (row, col) of
  // entry t advance without divisions
  {
    const int ns = nslot;
    int row = row_lo - 1 + tid / W, col = tid % W;
    for (int t = tid; t < (CF_BR + 2) * W; t += CF_THREADS) {
      V v = S::zero();
      if (row >= 0 && row <= nf) {
        const int k = col + W * row;
        // the (at most four) parents' loads are issued together
        V pv[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) pv[s] = s < ns ? S::ldv(pp[s], a.nvf, k) : S::zero();
        typename S::D acc = S::dzero();
#pragma unroll
        for (int s = 0; s < 4; ++s)
          if (s < ns) S::dadd(acc, pw[s], pv[s]);
        v = S::dget(acc);
      }
      tile[t] = v;
      col += CF_THREADS;
      while (col >= W) {
        col -= W;
        ++row;
      }
    }
  }
  __syncthreads();

  const double *kc = a.kappa_c + (size_t)pt * ncg * ncg;
  const V sixth = S::from(1.0 / 6.0);
  const typename S::P phv = S::vec(a.phi, unit, a.nvf), yv = S::vec(a.y, unit, a.nvf);
  const typename S::P yrv = a.yR ? S::vec(a.yR, unit, a.nvf) : nullptr;
  // kappa of a level-n element in V: float-float storage reads the prepared planes (a
  // double -> float conversion runs on the FP64 pipe, about 1/100 of the FP32 rate here)
  auto kval = [&](int e) -> V {
    if constexpr (std::is_same<V, ff>::value) return ff_load(a.kappa_ff, pt, ncg * ncg, e);
    else return kc[e];
  };
  {
    int row = row_lo + tid / W, col = tid % W;
    for (int t = tid; t < (row_hi - row_lo) * W; t += CF_THREADS) {
      const int k = col + W * row;
      const V *tr = tile + (row - row_lo + 1) * W + col;
      S::stv(phv, a.nvf, k, tr[0]);
      V v = S::zero(), vR = S::zero();
      if (row > 0 && row < nf && col > 0 && col < nf) {
        const int e0x = (col - 1) >> lgr, e1x = col >> lgr;
        const int e0y = (row - 1) >> lgr, e1y = row >> lgr;
        const V kSW = kval(e0x + ncg * e0y), kSE = kval(e1x + ncg * e0y);
        const V kNW = kval(e0x + ncg * e1y), kNE = kval(e1x + ncg * e1y);
        v = q1_dot<S>(kSW, kSE, kNW, kNE, tr, W, sixth);
        if (a.yR) {
          // the same with kappa zero outside the integration region (period index of each
          // adjacent fine element)
          const int P = a.P, o = a.overs;
          auto in = [&](int ex, int ey) {
            const int px = ex >> a.lgmf, py = ey >> a.lgmf;
            return px >= o && px < P - o && py >= o && py < P - o;
          };
          const V z = S::zero();
          vR = q1_dot<S>(in(col - 1, row - 1) ? kSW : z, in(col, row - 1) ? kSE : z,
                         in(col - 1, row) ? kNW : z, in(col, row) ? kNE : z, tr, W, sixth);
        }
      }
      S::stv(yv, a.nvf, k, v);
      if (yrv) S::stv(yrv, a.nvf, k, vR);
      col += CF_THREADS;
      while (col >= W) {
        col -= W;
        ++row;
      }
    }
  }

  // C_1 I on the band's element rows: element corner sums per (label, sub-block). Warp w
  // takes column chunk w % nch (32 element columns: whole sub-block columns or aligned parts
  // of one; lanes past the last column add nothing) and a contiguous range of the band's
  // element rows (group w / nch). A lane walks its element column upwards with the sum of
  // the node pair (ex, ex+1) of the previous node row, so an element costs two adds, and sums
  // the elements of one level-n element (one label, one sub-block: the level-n element size
  // 2^lgr divides the sub-block size) before adding them to its label's slot.
  {
    const int warp = tid >> 5, lane = tid & 31;
    const int nch = (nf + 31) >> 5;                // nf <= 256
    const int ngrp = (CF_THREADS / 32) / nch;
    const int chunk = warp % nch, grp = warp / nch;
    const int ex = chunk * 32 + lane;
    const bool lane_ok = ex < nf;
    const int exs = lane_ok ? ex : 0;
    const int lgm = a.lgmf, m = 1 << lgm;
    const int seg = m < 32 ? m : 32;
    const int rho_m = (1 << lgr) - 1;
    const uint8_t *lc = a.labels_c + (size_t)pt * ncg * ncg + (exs >> lgr);
    const int bx = exs >> lgm;
    V acc[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) acc[j] = S::zero();
    auto flush = [&](int by) {
#pragma unroll
      for (int j = 0; j < NC; ++j) {
        const double sj = S::to(seg_sum_s<S>(acc[j], seg));
        if ((lane & (seg - 1)) == 0 && sj != 0.0)
          atomicAdd(&bins[j * a.P * a.P + by * a.P + bx], sj);
        acc[j] = S::zero();
      }
    };
    const int erow_hi = min(row_lo + CF_BR, nf);
    const int rpg = (CF_BR + ngrp - 1) / ngrp;
    const int ey_lo = grp < ngrp ? min(row_lo + grp * rpg, erow_hi) : erow_hi;
    const int ey_hi = min(ey_lo + rpg, erow_hi);
    if (ey_lo < ey_hi) {                           // uniform over the warp
      const V *tc = tile + (ey_lo - row_lo + 1) * W + exs;
      V cprev = lane_ok ? tc[0] + tc[1] : S::zero();
      V cur = S::zero();
      int lab = lc[ncg * (ey_lo >> lgr)];
      int by_cur = ey_lo >> lgm;
      for (int ey = ey_lo; ey < ey_hi; ++ey) {
        if (ey > ey_lo && (ey & rho_m) == 0) {     // a new level-n element row
          add_lab_s<NC, S>(acc, lab, cur);
          cur = S::zero();
          const int by = ey >> lgm;
          if (by != by_cur) {
            flush(by_cur);
            by_cur = by;
          }
          lab = lc[ncg * (ey >> lgr)];
        }
        tc += W;
        const V cn = lane_ok ? tc[0] + tc[1] : S::zero();
        cur += cprev + cn;
        cprev = cn;
      }
      add_lab_s<NC, S>(acc, lab, cur);
      flush(by_cur);
    }
  }
  __syncthreads();
  for (int t = tid; t < a.nc; t += CF_THREADS)
    if (bins[t] != 0.0) atomicAdd(&a.g[((size_t)pt * a.nc + t) * a.R + r], -a.s * bins[t]);
}

constexpr int GR_THREADS = 256;

// E += alpha sym(X^T Y) per point (R vectors each). SYM: Y is the image of X under a
// symmetric operator (Y = A_1 X), so X^T Y is symmetric and one product per pair suffices.
// Each thread's pair sums are sums of products (S::D: Dot2 in float-float storage).
template <int R, class S, bool SYM>
__global__ void __launch_bounds__(GR_THREADS) k_gram2d(int nv, int slices, const double *X,
                                                        const double *Y, double alpha, double *E) {
  using V = typename S::V;
  constexpr int NP = R * (R + 1) / 2;
  const int pt = blockIdx.x;
  const int per = (nv + slices - 1) / slices;
  const int k0 = blockIdx.y * per, k1 = min(nv, k0 + per);
  typename S::D acc[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) acc[p] = S::dzero();
  const typename S::P x0 = S::vec(X, (size_t)pt * R, nv), y0 = S::vec(Y, (size_t)pt * R, nv);
  // vector r of the point starts r * (entries of one vector) after vector 0
  const int vstride = (int)(S::vec(X, 1, nv) - S::vec(X, 0, nv));
  for (int k = k0 + threadIdx.x; k < k1; k += GR_THREADS) {
    V xv[R], yv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      xv[r] = S::ldv(x0 + r * vstride, nv, k);
      yv[r] = S::ldv(y0 + r * vstride, nv, k);
    }
    int p = 0;
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int s = r; s < R; ++s, ++p) {
        S::dadd(acc[p], xv[r], yv[s]);
        if constexpr (!SYM) S::dadd(acc[p], yv[r], xv[s]);
      }
  }
  __shared__ double red[GR_THREADS / 32][NP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const V v = seg_sum_s<S>(S::dget(acc[p]), 32);
    if (lane == 0) red[w][p] = S::to(v);
  }
  __syncthreads();
  for (int p = threadIdx.x; p < NP; p += GR_THREADS) {
    double s = 0.0;
    for (int ww = 0; ww < GR_THREADS / 32; ++ww) s += red[ww][p];
    int rr = 0, cc = 0, q = p;
    while (q >= R - rr) { q -= R - rr; ++rr; }
    cc = rr + q;
    double *Ep = E + (size_t)pt * R * R;
    const double v = (SYM ? 1.0 : 0.5) * alpha * s;
    atomicAdd(&Ep[rr * R + cc], v);
    if (cc != rr) atomicAdd(&Ep[cc * R + rr], v);
  }
}

// The symmetric Gram (Y = A_1 X) in float-float storage with the pairs split over two warp
// sets: rows r and R-1-r carry R+1 pairs together, and such row pairs alternate between the
// sets (the middle row of an odd R joins set 0), so a warp keeps about half of the pair sums
// and loads Y and its own rows of X. Warps 2g and 2g+1 take the same nodes with the two sets:
// twice the resident warps of k_gram2d at the same loads per pair (the point's R (R+1) / 2
// pair sums in registers otherwise hold a CTA per SM).
template <int R>
struct GramSplit {
  static constexpr int set_of(int r) { return (r < R - 1 - r ? r : R - 1 - r) & 1; }
  static constexpr int np(int set) {
    int c = 0;
    for (int r = 0; r < R; ++r)
      if (set_of(r) == set) c += R - r;
    return c;
  }
  static constexpr int NPMAX = np(0) > np(1) ? np(0) : np(1);
  // index of pair (r, s), r <= s, among its set's pairs, and in the full upper triangle
  static constexpr int local(int r, int s) {
    int c = 0;
    for (int q = 0; q < r; ++q)
      if (set_of(q) == set_of(r)) c += R - q;
    return c + (s - r);
  }
  static constexpr int global(int r, int s) { return r * R - r * (r - 1) / 2 + (s - r); }
};

template <int R, class S, int SET>
__device__ __forceinline__ void gram_split_walk(typename S::D (&acc)[GramSplit<R>::NPMAX],
                                                typename S::P x0, typename S::P y0, int vstride,
                                                int nv, int k0, int k1, int node0, int nstep) {
  using V = typename S::V;
  using G = GramSplit<R>;
  for (int k = k0 + node0; k < k1; k += nstep) {
    V yv[R], xv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      yv[r] = S::ldv(y0 + r * vstride, nv, k);
      if (G::set_of(r) == SET) xv[r] = S::ldv(x0 + r * vstride, nv, k);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (G::set_of(r) != SET) continue;
#pragma unroll
      for (int s = r; s < R; ++s) S::dadd(acc[G::local(r, s)], xv[r], yv[s]);
    }
  }
}

template <int R, class S>
__global__ void __launch_bounds__(GR_THREADS, 2) k_gram2d_split(int nv, int slices,
                                                                const double *X, const double *Y,
                                                                double alpha, double *E) {
  using V = typename S::V;
  using G = GramSplit<R>;
  constexpr int NP = R * (R + 1) / 2;
  __shared__ double red[GR_THREADS / 32][NP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < (GR_THREADS / 32) * NP; i += GR_THREADS) (&red[0][0])[i] = 0.0;
  const int pt = blockIdx.x;
  const int per = (nv + slices - 1) / slices;
  const int k0 = blockIdx.y * per, k1 = min(nv, k0 + per);
  typename S::D acc[G::NPMAX];
#pragma unroll
  for (int p = 0; p < G::NPMAX; ++p) acc[p] = S::dzero();
  const typename S::P x0 = S::vec(X, (size_t)pt * R, nv), y0 = S::vec(Y, (size_t)pt * R, nv);
  const int vstride = (int)(S::vec(X, 1, nv) - S::vec(X, 0, nv));
  const int node0 = (w >> 1) * 32 + lane, nstep = GR_THREADS / 2;
  const int set = w & 1;                                  // uniform over the warp
  if (set == 0) gram_split_walk<R, S, 0>(acc, x0, y0, vstride, nv, k0, k1, node0, nstep);
  else gram_split_walk<R, S, 1>(acc, x0, y0, vstride, nv, k0, k1, node0, nstep);
  __syncthreads();                                        // red zeroed
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int s = r; s < R; ++s) {
      if (G::set_of(r) != set) continue;
      const V v = seg_sum_s<S>(S::dget(acc[G::local(r, s)]), 32);
      if (lane == 0) red[w][G::global(r, s)] = S::to(v);
    }
  __syncthreads();
  for (int p = threadIdx.x; p < NP; p += GR_THREADS) {
    double sum = 0.0;
    for (int ww = 0; ww < GR_THREADS / 32; ++ww) sum += red[ww][p];
    int rr = 0, q = p;
    while (q >= R - rr) { q -= R - rr; ++rr; }
    const int cc = rr + q;
    double *Ep = E + (size_t)pt * R * R;
    const double v = alpha * sum;
    atomicAdd(&Ep[rr * R + cc], v);
    if (cc != rr) atomicAdd(&Ep[cc * R + rr], v);
  }
}

// b = scale * P^T y on the level grid (zero on its boundary nodes): P^T sums the fine values
// around coarse node K with the separable hat weights (RHO - |d|) / RHO per axis. One CTA per
// (unit, 32 / RHO coarse rows): the fine rows those coarse rows reach (32 + RHO - 1) are
// staged in shared memory with coalesced loads, so a fine row is read about once, then summed
// along y per fine column and along x per coarse node (sums of products as in the Gram).
constexpr int RS_FINE_ROWS = 32;

template <int RHO>
constexpr int restrict_rows() { return (RS_FINE_ROWS / RHO - 1) * RHO + 2 * RHO - 1; }

template <int RHO, class S>
__global__ void __launch_bounds__(256) k_restrict2d(int nf, const double *yf, int nvf,
                                                     double scale, double *outc, int nvc) {
  using V = typename S::V;
  constexpr int KB = RS_FINE_ROWS / RHO;               // coarse rows per CTA
  constexpr int NR = restrict_rows<RHO>();             // staged fine rows
  extern __shared__ __align__(16) unsigned char rs_smem[];
  V *rows = reinterpret_cast<V *>(rs_smem);            // [NR][257]
  V *cs = rows + NR * 257;                             // [257]
  const int unit = blockIdx.y, tid = threadIdx.x;
  const int ncg = nf / RHO, Wc = ncg + 1, Wf = nf + 1;
  const int K0 = blockIdx.x * KB;
  const int fr0 = K0 * RHO - (RHO - 1);                // first staged fine row (may be < 0)
  const typename S::P yb = S::vec(yf, unit, nvf);
  {
    // NB loads in flight per thread before their shared-memory stores; (fine row, column)
    // advanced without divisions
    constexpr int NB = 8;
    int fr = fr0 + tid / Wf, col = tid % Wf;
    for (int t0 = tid; t0 < NR * Wf; t0 += 256 * NB) {
      V buf[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        const int t = t0 + 256 * j;
        buf[j] = (t < NR * Wf && fr >= 0 && fr <= nf) ? S::ldv(yb, nvf, fr * Wf + col)
                                                       : S::zero();
        col += 256;
        while (col >= Wf) {
          col -= Wf;
          ++fr;
        }
      }
#pragma unroll
      for (int j = 0; j < NB; ++j)
        if (t0 + 256 * j < NR * Wf) rows[t0 + 256 * j] = buf[j];
    }
  }
  __syncthreads();
  double *o = outc + (size_t)unit * nvc;
  for (int kk = 0; kk < KB; ++kk) {
    const int Ky = K0 + kk;
    if (Ky > ncg) break;                               // uniform over the CTA
    if (Ky == 0 || Ky == ncg) {
      for (int t = tid; t < Wc; t += 256) o[Ky * Wc + t] = 0.0;
      continue;
    }
    for (int col = tid; col < Wf; col += 256) {
      const V *rc = rows + (kk * RHO) * Wf + col;      // fine row Ky RHO - (RHO - 1)
      typename S::D sy = S::dzero();
#pragma unroll
      for (int d = 0; d < 2 * RHO - 1; ++d)
        S::dadd(sy, rc[d * Wf],
                S::fromf(float(RHO - (d < RHO - 1 ? RHO - 1 - d : d - (RHO - 1)))));
      cs[col] = S::dget(sy);
    }
    __syncthreads();
    for (int Kx = tid; Kx < Wc; Kx += 256) {
      double v = 0.0;
      if (Kx > 0 && Kx < ncg) {
        const V *cc = cs + Kx * RHO - (RHO - 1);
        typename S::D sx = S::dzero();
#pragma unroll
        for (int d = 0; d < 2 * RHO - 1; ++d)
          S::dadd(sx, cc[d], S::fromf(float(RHO - (d < RHO - 1 ? RHO - 1 - d : d - (RHO - 1)))));
        v = scale * S::to(S::dget(sx)) * (1.0 / (RHO * RHO));
      }
      o[Ky * Wc + Kx] = v;
    }
    __syncthreads();                                   // cs is rewritten for the next row
  }
}

// phi += P x: every fine node of the cells' lower-left quadrants (rows and columns 0 .. nf-1)
// gets the bilinear interpolant of its coarse cell's four values. One CTA per (unit, KB
// coarse rows = 8 fine rows), one thread per fine node (coalesced); the coarse values of the
// CTA's KB + 1 coarse rows are converted once into shared memory.
template <int RHO, class S>
__global__ void __launch_bounds__(256) k_prolong_add2d(int nf, const double *xc, int nvc,
                                                        double *phif, int nvf) {
  using V = typename S::V;
  constexpr int KB = RHO >= 8 ? 1 : 8 / RHO;
  __shared__ V xs[(KB + 1) * 129];
  const int unit = blockIdx.y, tid = threadIdx.x;
  const int ncg = nf / RHO, Wc = ncg + 1, Wf = nf + 1;
  const int K0 = blockIdx.x * KB;
  const int kb = min(KB, ncg - K0);                    // coarse cell rows of this CTA
  const double *x = xc + (size_t)unit * nvc + (size_t)K0 * Wc;
  for (int t = tid; t < (kb + 1) * Wc; t += 256) xs[t] = S::from(x[t]);
  __syncthreads();
  const typename S::P pf = S::vec(phif, unit, nvf);
  // at most 8 fine rows x 256 columns: PB nodes per thread, all loaded before any store so
  // that the loads are in flight together
  constexpr int PB = 8;
  const int total = kb * RHO * nf;
  int jr = tid / nf, col = tid % nf;                  // fine row K0 RHO + jr, column col
  int kk[PB], jj[PB], cc[PB];
  V old[PB];
#pragma unroll
  for (int u = 0; u < PB; ++u) {
    jj[u] = jr;
    cc[u] = col;
    kk[u] = (K0 * RHO + jr) * Wf + col;
    old[u] = tid + 256 * u < total ? S::ldv(pf, nvf, kk[u]) : S::zero();
    col += 256;
    while (col >= nf) {
      col -= nf;
      ++jr;
    }
  }
#pragma unroll
  for (int u = 0; u < PB; ++u) {
    if (tid + 256 * u >= total) break;
    const int kr = jj[u] / RHO, j = jj[u] % RHO;
    const int Kx = cc[u] / RHO, i = cc[u] % RHO;
    const V *xr = xs + kr * Wc + Kx;
    const V x00 = xr[0], x10 = xr[1], x01 = xr[Wc], x11 = xr[Wc + 1];
    const float ty = float(j) * (1.0f / RHO);          // exact: RHO is a power of two
    const V aj = x00 + (x01 - x00) * ty, bj = x10 + (x11 - x10) * ty;
    S::stv(pf, nvf, kk[u], old[u] + (aj + (bj - aj) * (float(i) * (1.0f / RHO))));
  }
}

// FP64 <-> float-float planes, `count` vectors of nv entries (only the first `len` of each)
__global__ void k_to_ff(const double *src, int nvs, double *dst, int nvd, int len) {
  const int v = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nvd) return;
  ff_store(dst, v, nvd, k, ff_from(k < len ? src[(size_t)v * nvs + k] : 0.0));
}
__global__ void k_from_ff(const double *src, int nvs, double *dst, int nvd, int len) {
  const int v = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= len) return;
  dst[(size_t)v * nvd + k] = ff_to(ff_load(src, v, nvs, k));
}

}  // namespace

cudaError_t launch_child_fine2d(const ChildArgs &a, bool ffs, cudaStream_t st) {
  if (a.nf < 32 || a.nf > 256 || (ffs && !a.kappa_ff)) return cudaErrorInvalidValue;
  dim3 grid((a.nf + 1 + CF_BR - 1) / CF_BR, a.npts * a.R);
#define CF_LAUNCH(NCV)                                                             \
  (ffs ? (k_child_fine2d<NCV, FFS><<<grid, CF_THREADS, 0, st>>>(a), 0)            \
       : (k_child_fine2d<NCV, F64S><<<grid, CF_THREADS, 0, st>>>(a), 0))
  if (a.N <= 2) CF_LAUNCH(2);
  else if (a.N == 3) CF_LAUNCH(3);
  else CF_LAUNCH(4);
#undef CF_LAUNCH
  return cudaGetLastError();
}

template <class S, bool SYM>
cudaError_t gram_s(int npts, int R, int nv, const double *X, const double *Y, double alpha,
                   double *E, cudaStream_t st) {
  int slices = nv >= 8192 ? 8 : (nv >= 2048 ? 4 : 1);
  if (nv > 100000) {
    // 3D level-1 lattices: enough slices for every SM when the level has few points
    const int want = (4 * device_sm_count() + npts - 1) / npts;
    slices = want < 8 ? 8 : (want > nv / 4096 ? nv / 4096 : want);
  }
  dim3 grid(npts, slices);
  if constexpr (SYM && std::is_same<S, FFS>::value) {
    switch (R) {
      case 3: k_gram2d_split<3, S><<<grid, GR_THREADS, 0, st>>>(nv, slices, X, Y, alpha, E); break;
      case 4: k_gram2d_split<4, S><<<grid, GR_THREADS, 0, st>>>(nv, slices, X, Y, alpha, E); break;
      case 6: k_gram2d_split<6, S><<<grid, GR_THREADS, 0, st>>>(nv, slices, X, Y, alpha, E); break;
      case 8: k_gram2d_split<8, S><<<grid, GR_THREADS, 0, st>>>(nv, slices, X, Y, alpha, E); break;
      case 9: k_gram2d_split<9, S><<<grid, GR_THREADS, 0, st>>>(nv, slices, X, Y, alpha, E); break;
      default: break;                                   // R = 12: the pair sums do not fit
    }
    if (R <= 9) return cudaGetLastError();
  }
  switch (R) {
    case 3: k_gram2d<3, S, SYM><<<grid, GR_THREADS, 0, st>>>(nv, slices, X, Y, alpha, E); break;
    case 4: k_gram2d<4, S, SYM><<<grid, GR_THREADS, 0, st>>>(nv, slices, X, Y, alpha, E); break;
    case 6: k_gram2d<6, S, SYM><<<grid, GR_THREADS, 0, st>>>(nv, slices, X, Y, alpha, E); break;
    case 8: k_gram2d<8, S, SYM><<<grid, GR_THREADS, 0, st>>>(nv, slices, X, Y, alpha, E); break;
    case 9: k_gram2d<9, S, SYM><<<grid, GR_THREADS, 0, st>>>(nv, slices, X, Y, alpha, E); break;
    case 12: k_gram2d<12, S, SYM><<<grid, GR_THREADS, 0, st>>>(nv, slices, X, Y, alpha, E); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_gram(int npts, int R, int nv, const double *X, const double *Y,
                        double alpha, double *E, cudaStream_t st, bool ffs, bool sym) {
  if (sym)
    return ffs ? gram_s<FFS, true>(npts, R, nv, X, Y, alpha, E, st)
               : gram_s<F64S, true>(npts, R, nv, X, Y, alpha, E, st);
  return ffs ? gram_s<FFS, false>(npts, R, nv, X, Y, alpha, E, st)
             : gram_s<F64S, false>(npts, R, nv, X, Y, alpha, E, st);
}

template <class S>
cudaError_t restrict_s(int npts, int R, int nf, int rho, const double *yf, int nvf, double scale,
                       double *outc, int nvc, cudaStream_t st) {
  if (nf > 256) return cudaErrorInvalidValue;
  const int Wc = nf / rho + 1, kb = RS_FINE_ROWS / rho;
  dim3 grid((Wc + kb - 1) / kb, npts * R);
  auto run = [&](auto kern, int nr) {
    const int smem = (nr + 1) * 257 * (int)sizeof(typename S::V);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 256, smem, st>>>(nf, yf, nvf, scale, outc, nvc);
    return cudaGetLastError();
  };
  switch (rho) {
    case 2: return run(k_restrict2d<2, S>, restrict_rows<2>());
    case 4: return run(k_restrict2d<4, S>, restrict_rows<4>());
    case 8: return run(k_restrict2d<8, S>, restrict_rows<8>());
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_restrict2d(int npts, int R, int nf, int rho, const double *yf, int nvf,
                              double scale, double *outc, int nvc, cudaStream_t st, bool ffs) {
  return ffs ? restrict_s<FFS>(npts, R, nf, rho, yf, nvf, scale, outc, nvc, st)
             : restrict_s<F64S>(npts, R, nf, rho, yf, nvf, scale, outc, nvc, st);
}

template <class S>
cudaError_t prolong_s(int npts, int R, int nf, int rho, const double *xc, int nvc, double *phif,
                      int nvf, cudaStream_t st) {
  if (nf > 256) return cudaErrorInvalidValue;
  const int ncg = nf / rho, kb = rho >= 8 ? 1 : 8 / rho;
  dim3 grid((ncg + kb - 1) / kb, npts * R);
  switch (rho) {
    case 2: k_prolong_add2d<2, S><<<grid, 256, 0, st>>>(nf, xc, nvc, phif, nvf); break;
    case 4: k_prolong_add2d<4, S><<<grid, 256, 0, st>>>(nf, xc, nvc, phif, nvf); break;
    case 8: k_prolong_add2d<8, S><<<grid, 256, 0, st>>>(nf, xc, nvc, phif, nvf); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_prolong_add2d(int npts, int R, int nf, int rho, const double *xc, int nvc,
                                 double *phif, int nvf, cudaStream_t st, bool ffs) {
  return ffs ? prolong_s<FFS>(npts, R, nf, rho, xc, nvc, phif, nvf, st)
             : prolong_s<F64S>(npts, R, nf, rho, xc, nvc, phif, nvf, st);
}

cudaError_t launch_to_ff(int count, const double *src, int nvs, double *dst, int nvd, int len,
                         cudaStream_t st) {
  dim3 grid((nvd + 255) / 256, count);
  k_to_ff<<<grid, 256, 0, st>>>(src, nvs, dst, nvd, len);
  return cudaGetLastError();
}

cudaError_t launch_from_ff(int count, const double *src, int nvs, double *dst, int nvd, int len,
                           cudaStream_t st) {
  dim3 grid((len + 255) / 256, count);
  k_from_ff<<<grid, 256, 0, st>>>(src, nvs, dst, nvd, len);
  return cudaGetLastError();
}

}  // namespace mch
