// Persistent level solve for the 3D constrained cell problems.
//
// Same method as the 2D level kernel (Sec. 3, Eq. phi_abstract: minimise 1/2 x'A x - b'x
// subject to Ct x = g, FP64 refinement steps around projected Jacobi-PCG sweeps in the inner
// precision T), but the 3D RVEs are too large to keep on chip (a 64^3 RVE has 250k unknowns
// per cell function), so the vectors stream through L2 and HBM. One cooperative launch
// covers the level: the interior node columns (kx, ky) of all (point, function) units are
// split into contiguous ranges, one per CTA; a thread walks a column along z with sliding
// windows of the 3x3x3 neighbourhood, of the 8 adjacent elements' kappa and of their labels.
//
// Per-unit reductions (dot products and the constraint functionals, which a column adds
// for each adjacent element row from its own nodes) are summed per CTA in shared memory and
// then atomically in FP64 into per-unit accumulators. Accumulators rotate over three buffers
// (written in a phase, read in the next, cleared in the one before), so every phase ends
// with exactly one grid barrier. After a barrier every CTA recomputes the scalars and the
// small constraint solves of its own units from the same sums in the same order, so all CTAs
// take the same decisions without further communication; loop exits use counters that the
// units' leader CTAs increment.
//
// Refinement step (FP64): x += delta; x += M^-1 Ct^T S^-1 (g - Ct x); r = b - A x;
//   r <- r - Ct^T S^-1 Ct M^-1 r; rho64 = r'M^-1 r; stop at sqrt(rho64 / rho64_ref) < rtol
//   with rho64_ref = max(rho64 of the first step, b'M^-1 b) (the scale of the cell function
//   for a correction problem).
// Inner iteration (T): q = A p; sums p.q, z.q, q.M^-1 q, r.z, Ct z, Ct M^-1 q;
//   alpha = rho / p.q; c = Ct z - alpha Ct M^-1 q; lambda = S^-1 c;
//   delta += alpha p; r <- r - alpha q - Ct^T lambda; rho' = r.z - 2 alpha z.q
//   + alpha^2 q.M^-1 q - lambda.c; p = M^-1 r + (rho' / rho) p.
// Every loop is bounded by max_refine and max_iter.
#include <cooperative_groups.h>

#include "k3d.cuh"
#include "kernels.h"

namespace mch {

namespace cg = cooperative_groups;

namespace {

constexpr int L3_THREADS = 256;
constexpr int NACC_S = 8;  // scalar sums per unit: pq, zq, qMq, rz, rho64

struct L3Smem {
  int kmax, nc;
  double *sums;   // [kmax][8]
  double *bins;   // [kmax][2 nc]
  double *vec;    // [kmax][nc] multipliers of the current phase
  double *rho, *rho_first, *rho64_first, *ratio, *alpha, *beta;  // [kmax]
  int *flags, *iters, *sweeps;                                   // [kmax]
};

// flags bits
constexpr int F_DONE = 1;    // unit finished (converged, capped or broken down)
constexpr int F_INNER = 2;   // unit active in the current inner sweep
constexpr int F_BREAK = 4;   // breakdown

template <typename V>
__device__ __forceinline__ void load_plane9(V (&v)[3][3], const V *p, size_t node, int W) {
#pragma unroll
  for (int dy = 0; dy < 3; ++dy)
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) v[dy][dx] = p[node + (dx - 1) + (size_t)W * (dy - 1)];
}

template <typename V>
__device__ __forceinline__ void load_kplane(V (&k)[2][2], const V *kap, int kx, int ky, int ez,
                                            int n) {
#pragma unroll
  for (int sy = 0; sy < 2; ++sy)
#pragma unroll
    for (int sx = 0; sx < 2; ++sx)
      k[sy][sx] = kap[(kx - 1 + sx) + (size_t)n * ((ky - 1 + sy) + (size_t)n * ez)];
}

// Labels of the four elements of element plane ez around node column (kx, ky), one byte per
// element column c = 2 sy + sx. Labels >= N (invalid input, reported by the setup) are
// clamped so that no row index leaves the multiplier tables; N <= 128 keeps the key >= 0.
__device__ __forceinline__ int lkey(const uint8_t *lab, int kx, int ky, int ez, int n, int nm1) {
  const uint8_t *l = lab + (kx - 1) + (size_t)n * ((ky - 1) + (size_t)n * ez);
  return min((int)l[0], nm1) | (min((int)l[1], nm1) << 8) | (min((int)l[n], nm1) << 16) |
         (min((int)l[n + 1], nm1) << 24);
}

// The same four labels (clamped likewise) as l[sy][sx].
__device__ __forceinline__ void load_lplane(int (&l)[2][2], const uint8_t *lab, int kx, int ky,
                                            int ez, int n, int nm1) {
#pragma unroll
  for (int sy = 0; sy < 2; ++sy)
#pragma unroll
    for (int sx = 0; sx < 2; ++sx)
      l[sy][sx] = min((int)lab[(kx - 1 + sx) + (size_t)n * ((ky - 1 + sy) + (size_t)n * ez)], nm1);
}

// Sub-block offsets along a node column, advanced without divisions: for node kz, lo and up
// are (z-block of the element plane below, resp. above) * P^2, and boundary() says that kz is
// a multiple of m (the two planes lie in different z-blocks).
struct ZBlk {
  int rem, lo, up, m, pp;
  __device__ __forceinline__ void init(int m_, int pp_) {  // kz = 1
    m = m_;
    pp = pp_;
    rem = m_ == 1 ? 0 : 1;
    lo = 0;
    up = m_ == 1 ? pp_ : 0;
  }
  __device__ __forceinline__ bool boundary() const { return rem == 0; }
  __device__ __forceinline__ void next() {  // kz -> kz + 1
    lo = up;
    if (++rem == m) {
      rem = 0;
      up += pp;
    }
  }
};

// Per-column accumulation of node values into the constraint rows of the adjacent elements
// (node-based form of Ct v): element plane ez of each of the four element columns c = 2 sy +
// sx around the node column gets the values of node planes ez and ez + 1. NV value streams
// share one set of runs: each stream keeps one running prefix Q of the column's node values,
// and a run of elements with one label and z-block adds (Q_e + Q_(e-1)) - (Q_(s-1) +
// Q_(s-2)) to shared memory when it ends (labels and z-blocks change rarely along a column),
// so a node costs one add per stream instead of one per element column. bins[k] is stream
// k's constraint rows, bxy[c] the element column's sub-block index within a z-block, zoff
// the current z-block * P^2.
template <typename V, int NV>
struct ColRuns {
  V q1[NV], q2[NV], st[4][NV];
  int lab[4];
  int zoff, nq;
  double *bins[NV];
  const int *bxy;
  // labels of element plane 0
  __device__ __forceinline__ void init(double *const (&b)[NV], const int *bxy_, int nq_,
                                       const int (&l)[2][2]) {
    bxy = bxy_;
    nq = nq_;
    zoff = 0;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      bins[k] = b[k];
      q1[k] = q2[k] = V(0);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      lab[c] = l[c >> 1][c & 1];
#pragma unroll
      for (int k = 0; k < NV; ++k) st[c][k] = V(0);
    }
  }
  __device__ __forceinline__ void close(int c) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const V t = q1[k] + q2[k];
      const V d = t - st[c][k];
      if (d != V(0)) atomicAdd(&bins[k][lab[c] * nq + zoff + bxy[c]], (double)d);
      st[c][k] = t;
    }
  }
  // element plane i (labels l, z-block offset zo) gets v, the values of node plane i + 1
  __device__ __forceinline__ void step(const int (&l)[2][2], int zo, const V (&v)[NV]) {
    if (zo != zoff) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        close(c);
        lab[c] = l[c >> 1][c & 1];
      }
      zoff = zo;
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (l[c >> 1][c & 1] != lab[c]) {
          close(c);
          lab[c] = l[c >> 1][c & 1];
        }
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      q2[k] = q1[k];
      q1[k] += v[k];
    }
  }
  // the top element plane (its upper node plane is the boundary, value 0), then every run out
  __device__ __forceinline__ void finish(const int (&l)[2][2], int zo) {
    V zero[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) zero[k] = V(0);
    step(l, zo, zero);
#pragma unroll
    for (int c = 0; c < 4; ++c) close(c);
  }
};

// Ct^T vec restricted to one element plane: the multipliers of its four elements' rows.
template <typename V>
__device__ __forceinline__ V plane_ctt(const V *vec, int key, int zoff, const int (&bxy)[4],
                                       int nq) {
  return (vec[(key & 255) * nq + zoff + bxy[0]] + vec[((key >> 8) & 255) * nq + zoff + bxy[1]]) +
         (vec[((key >> 16) & 255) * nq + zoff + bxy[2]] +
          vec[((key >> 24) & 255) * nq + zoff + bxy[3]]);
}

// Ct^T vec along a node column: the value at node kz is the sum of the plane sums below and
// above; the plane below is the previous node's plane above, and a plane sum is recomputed
// only when its labels or z-block change.
template <typename V>
struct ColCtt {
  V below, above;
  int key, zoff;
  // node 1: planes 0 and 1
  __device__ __forceinline__ void init(const V *vec, int key0, int key1, const ZBlk &zb,
                                       const int (&bxy)[4], int nq) {
    below = plane_ctt(vec, key0, zb.lo, bxy, nq);
    above = plane_ctt(vec, key1, zb.up, bxy, nq);
    key = key1;
    zoff = zb.up;
  }
  // moves to the next node, whose plane above has labels key_up and offset zup
  __device__ __forceinline__ void next(const V *vec, int key_up, int zup, const int (&bxy)[4],
                                       int nq) {
    below = above;
    if (key_up != key || zup != zoff) {
      above = plane_ctt(vec, key_up, zup, bxy, nq);
      key = key_up;
      zoff = zup;
    }
  }
  __device__ __forceinline__ V value() const { return below + above; }
};

// The two passes of an inner iteration over one node column (kz = 1..n-1) of a unit, with the
// vectors passed as restrict-qualified pointers to the column's base.

// q = h A p; the column's sums p.q, z.q, q.M^-1 q, r.z (z = M^-1 r) and its constraint
// functionals Ct z, Ct M^-1 q into the bins.
template <typename T>
__device__ __forceinline__ void p1_column(const T *__restrict__ p, T *__restrict__ q,
                                          const T *__restrict__ rv, const T *__restrict__ mi,
                                          const T *__restrict__ kap,
                                          const uint8_t *__restrict__ lab, int n, int kx, int ky,
                                          int m, int pp, int nm1, T h, double *bz,
                                          double *bq, const int *bxy, int nq, T (&sum)[4]) {
  const int W = n + 1, W2 = W * W;
  T v[3][3][3], k[2][2][2];
  load_plane9(v[0], p, 0, W);
  load_plane9(v[1], p, W2, W);
  load_kplane(k[0], kap, kx, ky, 0, n);
  int lo[2][2], up[2][2];
  load_lplane(lo, lab, kx, ky, 0, n, nm1);
  ColRuns<T, 2> cr;
  cr.init({bz, bq}, bxy, nq, lo);
  ZBlk zb;
  zb.init(m, pp);
  for (int kz = 1; kz < n; ++kz, zb.next()) {
    load_plane9(v[2], p, (size_t)W2 * (kz + 1), W);
    load_kplane(k[1], kap, kx, ky, kz, n);
    load_lplane(up, lab, kx, ky, kz, n, nm1);
    const int o = W2 * kz;
    const T qv = h * q1_apply3d<T>(v, k);
    q[o] = qv;
    const T mv = mi[o], r = rv[o];
    const T z = mv * r, qm = mv * qv;
    sum[0] += v[1][1][1] * qv;
    sum[1] += z * qv;
    sum[2] += qv * qm;
    sum[3] += r * z;
    cr.step(lo, zb.lo, {z, qm});
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        v[0][i][j] = v[1][i][j];
        v[1][i][j] = v[2][i][j];
      }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        k[0][i][j] = k[1][i][j];
        lo[i][j] = up[i][j];
      }
  }
  cr.finish(lo, zb.lo);
}

// delta += alpha p; r <- r - alpha q - Ct^T lambda; p = M^-1 r + beta p (unless last).
// Software-pipelined: node kz+1's operands are loaded before node kz is computed, so that
// two z steps of loads are in flight.
template <typename T>
__device__ __forceinline__ void p2_column(T *__restrict__ d, T *__restrict__ r,
                                          T *__restrict__ p, const T *__restrict__ q,
                                          const T *__restrict__ mi,
                                          const uint8_t *__restrict__ lab,
                                          const T *__restrict__ vec, int n, int kx, int ky,
                                          const int (&bxy)[4], int m, int pp, int nq, int nm1,
                                          T al, T be, bool last) {
  const int W = n + 1, W2 = W * W;
  ZBlk zb;
  zb.init(m, pp);
  ColCtt<T> ct;
  ct.init(vec, lkey(lab, kx, ky, 0, n, nm1), lkey(lab, kx, ky, 1, n, nm1), zb, bxy, nq);
  int o = W2;
  T pv = p[o], dv = d[o], rv = r[o], qv = q[o], mv = mi[o];
  for (int kz = 1; kz < n; ++kz) {
    const int on = o + W2;
    const bool more = kz + 1 < n;
    T pn = 0, dn = 0, rn = 0, qn = 0, mn = 0;
    int kn = 0;
    if (more) {
      pn = p[on];
      dn = d[on];
      rn = r[on];
      qn = q[on];
      mn = mi[on];
      kn = lkey(lab, kx, ky, kz + 1, n, nm1);
    }
    d[o] = dv + al * pv;
    const T rr = rv - al * qv - ct.value();
    r[o] = rr;
    if (!last) p[o] = mv * rr + be * pv;
    if (more) {
      zb.next();
      ct.next(vec, kn, zb.up, bxy, nq);
    }
    o = on;
    pv = pn;
    dv = dn;
    rv = rn;
    qv = qn;
    mv = mn;
  }
}

template <typename T>
struct Col {
  int u, slot, pt, kx, ky;
  int bxy[4];  // sub-block index (within a z-block) of the element columns c = 2 sy + sx
};

template <typename T>
__global__ void __launch_bounds__(L3_THREADS, 2) k_level3d(Level3Args<T> a) {
  cg::grid_group grid = cg::this_grid();
  const int n = a.n, W = n + 1, ni = n - 1, R = a.R, nc = a.nc, P = a.P, m = a.m;
  const int nq = P * P * P;
  const long long cpu = (long long)ni * ni;
  const long long units = (long long)a.npts * R;
  const long long total = units * cpu;
  const long long c0 = (long long)blockIdx.x * a.cols_per_cta;
  const long long c1 = min(total, c0 + a.cols_per_cta);
  const int u0 = (int)(c0 / cpu);
  const int K = c1 > c0 ? (int)((c1 - 1) / cpu) - u0 + 1 : 0;
  const int tid = threadIdx.x;
  const int NACC = NACC_S + 2 * nc;
  const size_t bufsz = (size_t)units * NACC;
  const size_t W2 = (size_t)W * W;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  L3Smem S;
  {
    double *d = reinterpret_cast<double *>(smem_raw);
    const int km = a.kmax;
    S.kmax = km;
    S.nc = nc;
    S.sums = d;
    d += km * 8;
    S.bins = d;
    d += km * 2 * nc;
    S.vec = d;
    d += km * nc;
    S.rho = d;
    d += km;
    S.rho_first = d;
    d += km;
    S.rho64_first = d;
    d += km;
    S.ratio = d;
    d += km;
    S.alpha = d;
    d += km;
    S.beta = d;
    d += km;
    int *ip = reinterpret_cast<int *>(d);
    S.flags = ip;
    ip += km;
    S.iters = ip;
    ip += km;
    S.sweeps = ip;
  }
  // multipliers of the inner update pass in the inner precision: they live in the second half
  // of the slot's bins, which that pass does not use (it is cleared before the next q = A p)
  auto vecT = [&](int s) { return reinterpret_cast<T *>(S.bins + (size_t)s * 2 * nc + nc); };
  for (int s = tid; s < K; s += L3_THREADS) {
    S.flags[s] = 0;
    S.iters[s] = 0;
    S.sweeps[s] = 0;
    S.ratio[s] = 0.0;
  }
  int ph = 0;
  auto wbuf = [&]() { return a.acc + (size_t)(ph % 3) * bufsz; };
  auto rbuf = [&]() { return a.acc + (size_t)((ph + 2) % 3) * bufsz; };
  auto leader = [&](int u) { return (long long)blockIdx.x == ((long long)u * cpu) / a.cols_per_cta; };
  // clears the buffer of the next phase (units whose leader this CTA is) and its counter
  auto clear_next = [&]() {
    double *z = a.acc + (size_t)((ph + 1) % 3) * bufsz;
    for (int s = 0; s < K; ++s) {
      const int u = u0 + s;
      if (!leader(u)) continue;
      for (int i = tid; i < NACC; i += L3_THREADS) z[(size_t)u * NACC + i] = 0.0;
    }
    if (blockIdx.x == 0 && tid == 0) a.cnt[(ph + 1) % 3] = 0;
  };
  auto zero_local = [&]() {
    for (int i = tid; i < K * 8; i += L3_THREADS) S.sums[i] = 0.0;
    for (int i = tid; i < K * 2 * nc; i += L3_THREADS) S.bins[i] = 0.0;
  };
  // adds the CTA's shared sums of slot s to the unit's accumulator (nonzero entries only)
  auto push_local = [&](int nbins) {
    double *w = wbuf();
    for (int s = 0; s < K; ++s) {
      const size_t ub = (size_t)(u0 + s) * NACC;
      for (int i = tid; i < NACC_S + nbins; i += L3_THREADS) {
        const double v = i < NACC_S ? S.sums[s * 8 + i] : S.bins[s * 2 * nc + (i - NACC_S)];
        if (v != 0.0) atomicAdd(&w[ub + i], v);
      }
    }
  };
  auto sync = [&]() {
    grid.sync();
    ++ph;
  };
  auto col_of = [&](long long c, Col<T> &cl) {
    cl.u = (int)(c / cpu);
    cl.slot = cl.u - u0;
    const int t = (int)(c % cpu);
    cl.kx = 1 + t % ni;
    cl.ky = 1 + t / ni;
    cl.pt = cl.u / R;
#pragma unroll
    for (int c = 0; c < 4; ++c)
      cl.bxy[c] = ((cl.ky - 1 + (c >> 1)) / m) * P + (cl.kx - 1 + (c & 1)) / m;
  };
  // lambda = S^-1 v for every active slot at once, one (slot, row) pair per thread (FP64; S^-1
  // is symmetric, so its rows are read column-wise, coalesced across rows). v = the slot's
  // constraint functionals of the previous phase, or g - those when with_g.
  auto small_solve64_all = [&](bool with_g) {
    const double *rb = rbuf();
    for (int i = tid; i < K * nc; i += L3_THREADS) {
      const int s = i / nc, row = i - s * nc;
      if (S.flags[s] & F_DONE) continue;
      const int u = u0 + s, pt = u / R;
      const double *src = rb + (size_t)u * NACC + NACC_S;
      const double *Si = a.Sinv64 + (size_t)pt * nc * nc;
      const double *gs = with_g ? a.g + (size_t)pt * nc * R + u % R : nullptr;
      double acc = 0.0;
      for (int j = 0; j < nc; ++j) {
        const double cj = gs ? gs[(size_t)j * R] - src[j] : src[j];
        acc += Si[(size_t)j * nc + row] * cj;
      }
      S.vec[s * nc + row] = acc;
    }
  };

  const int max_refine = a.max_refine;
  bool finished = false;
  for (int sweep = 0; sweep <= max_refine && !finished; ++sweep) {
    // ---- F1: x += delta, delta = 0; Ct x
    clear_next();
    zero_local();
    __syncthreads();
    for (long long c = c0 + tid; c < c1; c += L3_THREADS) {
      Col<T> cl;
      col_of(c, cl);
      if (S.flags[cl.slot] & F_DONE) continue;
      const size_t ub = (size_t)cl.u * a.nv + cl.kx + (size_t)W * cl.ky;
      const uint8_t *lab = a.labels + (size_t)cl.pt * n * n * n;
      int lo[2][2], up[2][2];
      load_lplane(lo, lab, cl.kx, cl.ky, 0, n, a.N - 1);
      ColRuns<double, 1> cr;
      cr.init({S.bins + cl.slot * 2 * nc}, cl.bxy, nq, lo);
      ZBlk zb;
      zb.init(m, P * P);
      for (int kz = 1; kz < n; ++kz, zb.next()) {
        load_lplane(up, lab, cl.kx, cl.ky, kz, n, a.N - 1);
        const size_t o = ub + W2 * kz;
        double xv = a.x[o];
        if (sweep > 0) {
          xv += (double)a.d[o];
          a.x[o] = xv;
          a.d[o] = T(0);
        }
        cr.step(lo, zb.lo, {xv});
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j) lo[i][j] = up[i][j];
      }
      cr.finish(lo, zb.lo);
    }
    __syncthreads();
    push_local(nc);
    sync();

    // ---- F2: mu = S^-1 (g - Ct x); x += M^-1 Ct^T mu
    clear_next();
    small_solve64_all(true);
    __syncthreads();
    for (long long c = c0 + tid; c < c1; c += L3_THREADS) {
      Col<T> cl;
      col_of(c, cl);
      if (S.flags[cl.slot] & F_DONE) continue;
      const size_t ub = (size_t)cl.u * a.nv + cl.kx + (size_t)W * cl.ky;
      const size_t mb = (size_t)cl.pt * a.nv + cl.kx + (size_t)W * cl.ky;
      const uint8_t *lab = a.labels + (size_t)cl.pt * n * n * n;
      const double *vec = S.vec + cl.slot * nc;
      ZBlk zb;
      zb.init(m, P * P);
      ColCtt<double> ct;
      ct.init(vec, lkey(lab, cl.kx, cl.ky, 0, n, a.N - 1), lkey(lab, cl.kx, cl.ky, 1, n, a.N - 1),
              zb, cl.bxy, nq);
      for (int kz = 1; kz < n; ++kz) {
        const size_t o = ub + W2 * kz;
        a.x[o] += a.minv64[mb + W2 * kz] * ct.value();
        if (kz + 1 < n) {
          zb.next();
          ct.next(vec, lkey(lab, cl.kx, cl.ky, kz + 1, n, a.N - 1), zb.up, cl.bxy, nq);
        }
      }
    }
    sync();

    // ---- F3: r = b - A x (FP64); Ct M^-1 r
    clear_next();
    zero_local();
    __syncthreads();
    for (long long c = c0 + tid; c < c1; c += L3_THREADS) {
      Col<T> cl;
      col_of(c, cl);
      if (S.flags[cl.slot] & F_DONE) continue;
      const size_t ub = (size_t)cl.u * a.nv + cl.kx + (size_t)W * cl.ky;
      const size_t mb = (size_t)cl.pt * a.nv + cl.kx + (size_t)W * cl.ky;
      const uint8_t *lab = a.labels + (size_t)cl.pt * n * n * n;
      const double *kap = a.kappa + (size_t)cl.pt * n * n * n;
      const double *bb = a.b ? a.b + (size_t)cl.u * a.nv : nullptr;
      double v[3][3][3], k[2][2][2];
      load_plane9(v[0], a.x, ub, W);
      load_plane9(v[1], a.x, ub + W2, W);
      load_kplane(k[0], kap, cl.kx, cl.ky, 0, n);
      int lo[2][2], up[2][2];
      load_lplane(lo, lab, cl.kx, cl.ky, 0, n, a.N - 1);
      ColRuns<double, 1> cr;
      cr.init({S.bins + cl.slot * 2 * nc}, cl.bxy, nq, lo);
      ZBlk zb;
      zb.init(m, P * P);
      for (int kz = 1; kz < n; ++kz, zb.next()) {
        load_plane9(v[2], a.x, ub + W2 * (kz + 1), W);
        load_kplane(k[1], kap, cl.kx, cl.ky, kz, n);
        load_lplane(up, lab, cl.kx, cl.ky, kz, n, a.N - 1);
        const size_t o = ub + W2 * kz;
        double r = -a.h * q1_apply3d<double>(v, k);
        if (bb) r += bb[o - (size_t)cl.u * a.nv];
        a.r64[o] = r;
        const double mr = a.minv64[mb + W2 * kz] * r;
        cr.step(lo, zb.lo, {mr});
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            v[0][i][j] = v[1][i][j];
            v[1][i][j] = v[2][i][j];
          }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            k[0][i][j] = k[1][i][j];
            lo[i][j] = up[i][j];
          }
      }
      cr.finish(lo, zb.lo);
    }
    __syncthreads();
    push_local(nc);
    sync();

    // ---- F4: lambda = S^-1 Ct M^-1 r; r -= Ct^T lambda; rho64; inner vectors
    clear_next();
    zero_local();
    small_solve64_all(false);
    __syncthreads();
    for (int s = 0; s < K; ++s) {
      const int u = u0 + s;
      if ((S.flags[s] & F_DONE) || !a.lam || !leader(u)) continue;
      for (int i = tid; i < nc; i += L3_THREADS) a.lam[(size_t)u * nc + i] = S.vec[s * nc + i];
    }
    for (long long c = c0 + tid; c < c1; c += L3_THREADS) {
      Col<T> cl;
      col_of(c, cl);
      if (S.flags[cl.slot] & F_DONE) continue;
      const size_t ub = (size_t)cl.u * a.nv + cl.kx + (size_t)W * cl.ky;
      const size_t mb = (size_t)cl.pt * a.nv + cl.kx + (size_t)W * cl.ky;
      const uint8_t *lab = a.labels + (size_t)cl.pt * n * n * n;
      const double *vec = S.vec + cl.slot * nc;
      double rho = 0.0;
      ZBlk zb;
      zb.init(m, P * P);
      ColCtt<double> ct;
      ct.init(vec, lkey(lab, cl.kx, cl.ky, 0, n, a.N - 1), lkey(lab, cl.kx, cl.ky, 1, n, a.N - 1),
              zb, cl.bxy, nq);
      for (int kz = 1; kz < n; ++kz) {
        const size_t o = ub + W2 * kz;
        const double r = a.r64[o] - ct.value();
        const double mi = a.minv64[mb + W2 * kz];
        rho += r * mi * r;
        const T rt = (T)r;
        a.r[o] = rt;
        a.p[o] = a.minvT[mb + W2 * kz] * rt;
        if (kz + 1 < n) {
          zb.next();
          ct.next(vec, lkey(lab, cl.kx, cl.ky, kz + 1, n, a.N - 1), zb.up, cl.bxy, nq);
        }
      }
      atomicAdd(&S.sums[cl.slot * 8 + 4], rho);
    }
    __syncthreads();
    push_local(0);
    sync();

    // ---- F5 (no barrier of its own): refinement decisions; then the inner sweep
    {
      const double *rb = rbuf();
      if (tid == 0) {
        for (int s = 0; s < K; ++s) {
          if (S.flags[s] & F_DONE) continue;
          const int u = u0 + s;
          const double r64 = rb[(size_t)u * NACC + 4];
          if (sweep == 0) S.rho64_first[s] = a.bnorm ? fmax(r64, a.bnorm[u]) : r64;
          const double f = S.rho64_first[s];
          const double ratio = f > 0.0 ? sqrt(r64 / f) : 0.0;
          S.ratio[s] = ratio;
          S.sweeps[s] = sweep;
          if (!(ratio >= a.rtol) || sweep == max_refine || !(ratio == ratio)) {
            S.flags[s] |= F_DONE;
          } else {
            S.flags[s] |= F_INNER;
            S.rho[s] = r64;
            S.rho_first[s] = r64;
          }
        }
      }
    }
    __syncthreads();
    for (int it = 0;; ++it) {
      // ---- P1: q = A p; sums and constraint functionals
      clear_next();
      zero_local();
      if (it == 0) {
        for (int s = 0; s < K; ++s)
          if ((S.flags[s] & F_INNER) && leader(u0 + s) && tid == 0) atomicAdd(&a.cnt[ph % 3], 1);
      }
      __syncthreads();
      for (long long c = c0 + tid; c < c1; c += L3_THREADS) {
        Col<T> cl;
        col_of(c, cl);
        if (!(S.flags[cl.slot] & F_INNER)) continue;
        const size_t ub = (size_t)cl.u * a.nv + cl.kx + (size_t)W * cl.ky;
        const size_t mb = (size_t)cl.pt * a.nv + cl.kx + (size_t)W * cl.ky;
        double *sb = S.bins + cl.slot * 2 * nc;
        T sum[4] = {0, 0, 0, 0};
        p1_column<T>(a.p + ub, a.q + ub, a.r + ub, a.minvT + mb,
                     a.kapT + (size_t)cl.pt * n * n * n, a.labels + (size_t)cl.pt * n * n * n, n,
                     cl.kx, cl.ky, m, P * P, a.N - 1, (T)a.h, sb, sb + nc, cl.bxy, nq, sum);
        const T pq = sum[0], zq = sum[1], qmq = sum[2], rz = sum[3];
        double *ss = S.sums + cl.slot * 8;
        {
          // one atomic per warp when all its lanes walk columns of the same unit
          const unsigned act = __activemask();
          if (act == 0xffffffffu && __match_any_sync(act, cl.slot) == act) {
            double w0 = pq, w1 = zq, w2 = qmq, w3 = rz;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
              w0 += __shfl_xor_sync(act, w0, o);
              w1 += __shfl_xor_sync(act, w1, o);
              w2 += __shfl_xor_sync(act, w2, o);
              w3 += __shfl_xor_sync(act, w3, o);
            }
            if ((tid & 31) == 0) {
              atomicAdd(&ss[0], w0);
              atomicAdd(&ss[1], w1);
              atomicAdd(&ss[2], w2);
              atomicAdd(&ss[3], w3);
            }
            continue;
          }
        }
        atomicAdd(&ss[0], (double)pq);
        atomicAdd(&ss[1], (double)zq);
        atomicAdd(&ss[2], (double)qmq);
        atomicAdd(&ss[3], (double)rz);
      }
      __syncthreads();
      push_local(2 * nc);
      sync();
      if (it == 0 && *(volatile int *)&a.cnt[(ph + 2) % 3] == 0) {
        finished = true;
        break;
      }

      // ---- P2: scalars, lambda, updates (all slots of the CTA at once)
      clear_next();
      {
        const double *rb = rbuf();
        // c = Ct z - alpha Ct M^-1 q into the first half of the slot's bins
        for (int i = tid; i < K * nc; i += L3_THREADS) {
          const int s = i / nc, j = i - s * nc;
          if (!(S.flags[s] & F_INNER)) continue;
          const double *acc = rb + (size_t)(u0 + s) * NACC;
          const double alpha = S.rho[s] / acc[0];
          S.bins[s * 2 * nc + j] = acc[NACC_S + j] - alpha * acc[NACC_S + nc + j];
        }
        __syncthreads();
        // lambda = S^-1 c in the inner precision, one (slot, row) pair per thread
        for (int i = tid; i < K * nc; i += L3_THREADS) {
          const int s = i / nc, row = i - s * nc;
          if (!(S.flags[s] & F_INNER)) continue;
          const T *Si = a.SinvT + (size_t)((u0 + s) / R) * nc * nc;
          const double *cs = S.bins + s * 2 * nc;
          T l = 0;
          for (int j = 0; j < nc; ++j) l += Si[(size_t)j * nc + row] * (T)cs[j];
          S.vec[s * nc + row] = (double)l;
          vecT(s)[row] = l;
        }
        __syncthreads();
        // scalars: one warp per slot (the same lane order in every CTA, so every CTA that
        // holds a unit takes the same decisions)
        const int lane = tid & 31;
        for (int s = tid >> 5; s < K; s += L3_THREADS / 32) {
          if (!(S.flags[s] & F_INNER)) continue;
          double lc = 0.0;
          for (int i = lane; i < nc; i += 32) lc += S.vec[s * nc + i] * S.bins[s * 2 * nc + i];
#pragma unroll
          for (int o = 16; o; o >>= 1) lc += __shfl_xor_sync(0xffffffffu, lc, o);
          if (lane == 0) {
            const double *acc = rb + (size_t)(u0 + s) * NACC;
            const double alpha = S.rho[s] / acc[0];
            const double rn = acc[3] - 2.0 * alpha * acc[1] + alpha * alpha * acc[2] - lc;
            S.alpha[s] = alpha;
            S.beta[s] = rn / S.rho[s];
            S.iters[s] += 1;
            const bool bad = !(acc[0] > 0.0) || !(rn == rn);
            if (bad) {
              S.flags[s] = (S.flags[s] & ~F_INNER) | F_DONE | F_BREAK;
            } else {
              S.rho[s] = rn;
              // the sweep's target: the inner tolerance, relaxed once the refinement
              // tolerance is within reach (0.3 rtol / ratio)
              const double ts = fmax((double)a.tol, fmin(0.5, 0.3 * a.rtol / S.ratio[s]));
              if (!(rn >= ts * ts * S.rho_first[s]) || it + 1 >= a.max_iter)
                S.flags[s] |= 8;  // last update of this sweep
            }
          }
        }
        __syncthreads();
      }
      for (long long c = c0 + tid; c < c1; c += L3_THREADS) {
        Col<T> cl;
        col_of(c, cl);
        const int f = S.flags[cl.slot];
        if (!(f & F_INNER)) continue;
        const size_t ub = (size_t)cl.u * a.nv + cl.kx + (size_t)W * cl.ky;
        const size_t mb = (size_t)cl.pt * a.nv + cl.kx + (size_t)W * cl.ky;
        p2_column<T>(a.d + ub, a.r + ub, a.p + ub, a.q + ub, a.minvT + mb,
                     a.labels + (size_t)cl.pt * n * n * n, vecT(cl.slot), n, cl.kx, cl.ky, cl.bxy,
                     m, P * P, nq, a.N - 1, (T)S.alpha[cl.slot], (T)S.beta[cl.slot],
                     (f & 8) != 0);
      }
      __syncthreads();
      if (tid == 0) {
        for (int s = 0; s < K; ++s) {
          if (!(S.flags[s] & F_INNER)) continue;
          if (S.flags[s] & 8) {
            S.flags[s] &= ~(F_INNER | 8);
          } else if (leader(u0 + s)) {
            atomicAdd(&a.cnt[ph % 3], 1);
          }
        }
      }
      __syncthreads();
      sync();
      if (*(volatile int *)&a.cnt[(ph + 2) % 3] == 0) break;
    }
  }

  // per-unit records from the leader CTA
  __syncthreads();
  if (tid == 0) {
    for (int s = 0; s < K; ++s) {
      const int u = u0 + s;
      if (!leader(u)) continue;
      a.iters[u] = S.iters[s];
      a.sweeps[u] = S.sweeps[s];
      a.ratio[u] = S.ratio[s];
      a.status[u] = (S.flags[s] & F_BREAK) ? 1 : 0;
    }
  }
}

template <typename T>
cudaError_t launch3(const Level3Args<T> &a0, cudaStream_t st) {
  Level3Args<T> a = a0;
  const long long cpu = (long long)(a.n - 1) * (a.n - 1);
  const long long total = (long long)a.npts * a.R * cpu;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // slots per CTA: a range of C columns touches at most ceil(C / cpu) + 1 units
  auto smem_for = [&](int kmax) {
    return (size_t)kmax * (sizeof(double) * (8 + 3 * a.nc + 6) + sizeof(int) * 3) + 64;
  };
  int occ = 0;
  int grid = 0;
  for (int kmax = 2; kmax <= 64; kmax *= 2) {
    const size_t smem = smem_for(kmax);
    e = cudaFuncSetAttribute(k_level3d<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_level3d<T>, L3_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    grid = occ * sms;
    long long per = (total + grid - 1) / grid;
    per = ((per + L3_THREADS - 1) / L3_THREADS) * L3_THREADS;
    const long long need = (per + cpu - 1) / cpu + 1;
    if (need <= kmax) {
      a.kmax = kmax;
      a.cols_per_cta = per;
      grid = (int)((total + per - 1) / per);
      void *args[] = {&a};
      return cudaLaunchCooperativeKernel((const void *)k_level3d<T>, dim3(grid),
                                         dim3(L3_THREADS), args, smem, st);
    }
  }
  return cudaErrorInvalidConfiguration;
}

}  // namespace

template <typename T>
cudaError_t launch_level3d(const Level3Args<T> &a, cudaStream_t st) {
  if (a.nc > MCH_MAX_NC3 || a.n < 2 || a.n % a.P || a.m != a.n / a.P) return cudaErrorInvalidValue;
  return launch3<T>(a, st);
}

template cudaError_t launch_level3d<float>(const Level3Args<float> &, cudaStream_t);
template cudaError_t launch_level3d<double>(const Level3Args<double> &, cudaStream_t);

}  // namespace mch
