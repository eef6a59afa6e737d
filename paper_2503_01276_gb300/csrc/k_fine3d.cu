// 3D level-1-grid (fine) work of a child level, the level-grid apply for the effective
// coefficients, and the 3D backward kernels; all FP64.
//
// Sec. 3.3, Eqs. (PhiXiI), (phiXiI_all): I = sum_t c_t Phi_t on the level-1 grid.
// Eqs. (phi_avar_corrector), (phi_grad_corrector): b = -P^T A_1 I and g = G - C_1 I, with A_1
// the level-1 stiffness of the child's medium (prolonged piecewise constantly from its
// level-n grid); Eq. (Bs_defi): E starts from K_I = I^T A_1 I (Gram of I and A_1 I).
// Phi = I + P Xi after the correction solve (trilinear nested prolongation P).
//
// Backward (see k_adjoint.cu for the 2D form and the derivation): Psi' = sum_r What_rs Phi_r
// - P mu_s, Psi = 1/2 sum_r What_rs Phi_r - P mu_s; dL/dkappa_E = sum_{fine e in E}
// h_f Psi_s|e^T Khat Phi_s|e; U_r = V_r + A_1 Psi'_r + rho^-3 Ct_1^T sigma_r pushed to the
// parents. With oversampling (E over R_p, the central (P - 2 o)^3 periods) E is not
// stationary in the cell functions: as in 2D, the level's own term sum_s What_rs A_{1,R}
// Phi_s is an adjoint source of every level (k_adj_own3d), the envelope terms are dropped,
// and the direct term counts only the elements inside R_p.
#include <type_traits>

#include "ff.cuh"
#include "k3d.cuh"
#include "kernels.h"

namespace mch {

namespace {

constexpr int F3_THREADS = 256;

__device__ __forceinline__ size_t cidx(int ex, int ey, int ez, int n) {
  return (size_t)ex + (size_t)n * (ey + (size_t)n * ez);
}

// conductivity of the fine element (ex, ey, ez) from the (nf >> lgr)-grid
__device__ __forceinline__ double kc_of(const double *kc, int ex, int ey, int ez, int lgr,
                                        int ncg) {
  return kc[cidx(ex >> lgr, ey >> lgr, ez >> lgr, ncg)];
}

// y = h A(kappa) x + cb b; one thread per lattice entry (boundary and padding written as 0).
__global__ void __launch_bounds__(F3_THREADS) k_apply3d(ApplyArgs a, double h) {
  const int unit = blockIdx.y, pt = unit / a.R;
  const int n = a.n, W = n + 1, lgr = __ffs(a.rho) - 1, ncg = n / a.rho;
  const int k = blockIdx.x * F3_THREADS + threadIdx.x;
  if (k >= a.nv) return;
  double *y = a.y + (size_t)unit * a.nv;
  const int kx = k % W, ky = (k / W) % W, kz = k / (W * W);
  if (k >= W * W * W || kx == 0 || ky == 0 || kz == 0 || kx == n || ky == n || kz == n) {
    y[k] = 0.0;
    return;
  }
  const double *x = a.x + (size_t)unit * a.nv;
  const double *kc = a.kappa + (size_t)pt * ncg * ncg * ncg;
  double v[3][3][3], kk[2][2][2];
#pragma unroll
  for (int dz = 0; dz < 3; ++dz)
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx)
        v[dz][dy][dx] = x[k + (dx - 1) + W * (dy - 1) + W * W * (dz - 1)];
#pragma unroll
  for (int sz = 0; sz < 2; ++sz)
#pragma unroll
    for (int sy = 0; sy < 2; ++sy)
#pragma unroll
      for (int sx = 0; sx < 2; ++sx)
        kk[sz][sy][sx] = kc_of(kc, kx - 1 + sx, ky - 1 + sy, kz - 1 + sz, lgr, ncg);
  double r = h * q1_apply3d<double>(v, kk);
  if (a.b) r += a.cb * a.b[(size_t)unit * a.nv + k];
  y[k] = r;
}

// The 3D stencil of k3d.cuh for any value type (FP64 or float-float): up to the factor h.
template <typename V>
__device__ __forceinline__ V q1_apply3d_v(const V (&v)[3][3][3], const V (&k)[2][2][2], V third,
                                          V twelfth) {
  const V ksum = ((k[0][0][0] + k[0][0][1]) + (k[0][1][0] + k[0][1][1])) +
                 ((k[1][0][0] + k[1][0][1]) + (k[1][1][0] + k[1][1][1]));
  V acc = k[0][0][0] * v[0][0][0];
#pragma unroll
  for (int c = 1; c < 8; ++c) {
    const int oz = c >> 2, oy = (c >> 1) & 1, ox = c & 1;
    acc += k[oz][oy][ox] * v[2 * oz][2 * oy][2 * ox];
  }
#pragma unroll
  for (int oy = 0; oy < 2; ++oy)
#pragma unroll
    for (int ox = 0; ox < 2; ++ox) acc += (k[0][oy][ox] + k[1][oy][ox]) * v[1][2 * oy][2 * ox];
#pragma unroll
  for (int oz = 0; oz < 2; ++oz)
#pragma unroll
    for (int ox = 0; ox < 2; ++ox) acc += (k[oz][0][ox] + k[oz][1][ox]) * v[2 * oz][1][2 * ox];
#pragma unroll
  for (int oz = 0; oz < 2; ++oz)
#pragma unroll
    for (int oy = 0; oy < 2; ++oy) acc += (k[oz][oy][0] + k[oz][oy][1]) * v[2 * oz][2 * oy][1];
  return ksum * v[1][1][1] * third - acc * twelfth;
}

template <class S>
__global__ void __launch_bounds__(F3_THREADS) k_interp3d(ChildArgs a) {
  using V = typename S::V;
  const int unit = blockIdx.y, pt = unit / a.R, r = unit % a.R;
  // the point's parents with a cell function, packed to the front, and their weights,
  // converted once per block
  __shared__ typename S::P pp[8];
  __shared__ V pw[8];
  __shared__ int nslot;
  if (threadIdx.x == 0) {
    int ns = 0;
    for (int s = 0; s < a.slots && s < 8; ++s) {
      const double *b = a.par_ptr[pt * a.slots + s];
      if (!b) continue;
      pp[ns] = S::vec(b, r, a.nvf);
      pw[ns] = S::from(a.par_w[pt * a.slots + s]);
      ++ns;
    }
    nslot = ns;
  }
  __syncthreads();
  const int k = blockIdx.x * F3_THREADS + threadIdx.x;
  if (k >= a.nvf) return;
  const int ns = nslot;
  // every parent's load is issued before the sum of products
  V pv[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) pv[s] = s < ns ? S::ldv(pp[s], a.nvf, k) : S::zero();
  typename S::D acc = S::dzero();
#pragma unroll
  for (int s = 0; s < 8; ++s)
    if (s < ns) S::dadd(acc, pw[s], pv[s]);
  S::st(a.phi, unit, a.nvf, k, S::dget(acc));
}

// y = h_f A_1 phi and g -= s C_1 phi: one thread per interior node column of the level-1
// lattice, walking z with sliding windows; the constraint functionals go per (element
// column, label) into registers, per CTA into shared memory, then into g. OVS: also the
// stencil restricted to R_p (oversampling); a separate instantiation, so that the common
// case keeps its registers (two resident CTAs per SM).
template <class S, bool OVS>
__global__ void __launch_bounds__(F3_THREADS, 2) k_fine_apply3d(ChildArgs a, double hf) {
  using V = typename S::V;
  const int unit = blockIdx.y, pt = unit / a.R, r = unit % a.R;
  const int nf = a.nf, W = nf + 1, ni = nf - 1, lgr = a.lgr, ncg = nf >> lgr;
  const int P = a.P, mf = 1 << a.lgmf, nq = P * P * P;
  __shared__ double bins[MCH_MAX_NC3];
  for (int i = threadIdx.x; i < a.nc; i += F3_THREADS) bins[i] = 0.0;
  __syncthreads();
  const int t = blockIdx.x * F3_THREADS + threadIdx.x;
  if (t < ni * ni) {
    const int kx = 1 + t % ni, ky = 1 + t / ni;
    const size_t W2 = (size_t)W * W;
    const double *kc = a.kappa_c + (size_t)pt * ncg * ncg * ncg;
    const uint8_t *lc = a.labels_c + (size_t)pt * ncg * ncg * ncg;
    const size_t base = kx + (size_t)W * ky;
    const V third = S::from(1.0 / 3.0), twelfth = S::from(1.0 / 12.0), hv = S::from(hf);
    // float-float storage reads the prepared kappa planes (no conversion per node)
    auto kval = [&](size_t c) -> V {
      if constexpr (std::is_same<V, ff>::value)
        return ff_load(a.kappa_ff, pt, ncg * ncg * ncg, (int)c);
      else return kc[c];
    };
    V v[3][3][3], kk[2][2][2];
    int lo[2][2], up[2][2];
    auto load_v = [&](V (&pl)[3][3], int z) {
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx)
          pl[dy][dx] = S::ld(a.phi, unit, a.nvf, (int)(base + W2 * z + (dx - 1) + W * (dy - 1)));
    };
    auto load_k = [&](V (&pl)[2][2], int (&lp)[2][2], int ez) {
#pragma unroll
      for (int sy = 0; sy < 2; ++sy)
#pragma unroll
        for (int sx = 0; sx < 2; ++sx) {
          const size_t c = cidx((kx - 1 + sx) >> lgr, (ky - 1 + sy) >> lgr, ez >> lgr, ncg);
          pl[sy][sx] = kval(c);
          lp[sy][sx] = lc[c];
        }
    };
    load_v(v[0], 0);
    load_v(v[1], 1);
    load_k(kk[0], lo, 0);
    // kappa pair sums of the element plane below the node (carried over from the step
    // before): along x per element row oy, along y per element column ox, and the plane's sum
    V px0[2], py0[2], ps0;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      px0[i] = kk[0][i][0] + kk[0][i][1];
      py0[i] = kk[0][0][i] + kk[0][1][i];
    }
    ps0 = px0[0] + px0[1];
    const V hv12 = S::from(hf / 12.0);
    // C_1 phi: each of the four element columns c = 2 sy + sx around the node column sums,
    // per (label, z-block), the node pairs (kz, kz+1) of its elements; all four share one
    // running prefix Q of the column's node values, and a run of elements with one label and
    // z-block adds (Q_e + Q_(e-1)) - (Q_(s-1) + Q_(s-2)) to its bin when it ends (labels and
    // z-blocks change rarely along a column), instead of per-node adds into every label slot.
    int bxy[4];
#pragma unroll
    for (int c = 0; c < 4; ++c)
      bxy[c] = ((ky - 1 + (c >> 1)) >> a.lgmf) * P + ((kx - 1 + (c & 1)) >> a.lgmf);
    V q1 = S::zero(), q2 = S::zero(), rs[4];
    int rl[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      rs[c] = S::zero();
      rl[c] = lo[c >> 1][c & 1];
    }
    int zoff = 0;  // z-block of the current element plane * P^2
    auto close = [&](int c) {
      const double d = S::to((q1 + q2) - rs[c]);
      if (rl[c] < a.N && d != 0.0) atomicAdd(&bins[rl[c] * nq + zoff + bxy[c]], d);
      rs[c] = q1 + q2;
    };
    // element plane i = kz - 1 (labels lp) gets the next node value through v_next
    auto elem_plane = [&](int i, const int (&lp)[2][2], V v_next) {
      if (i > 0 && (i & (mf - 1)) == 0) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          close(c);
          rl[c] = lp[c >> 1][c & 1];
        }
        zoff = (i >> a.lgmf) * P * P;
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (lp[c >> 1][c & 1] != rl[c]) {
            close(c);
            rl[c] = lp[c >> 1][c & 1];
          }
      }
      q2 = q1;
      q1 = q1 + v_next;
    };
    // oversampling: the same stencil with kappa zero outside R_p (period index of each
    // adjacent fine element)
    const int o = a.overs;
    auto in_r = [&](int ex, int ey, int ez) {
      const int px = ex >> a.lgmf, py = ey >> a.lgmf, pz = ez >> a.lgmf;
      return px >= o && px < P - o && py >= o && py < P - o && pz >= o && pz < P - o;
    };
    for (int kz = 1; kz < nf; ++kz) {
      load_v(v[2], kz + 1);
      load_k(kk[1], up, kz);
      // the 21-point stencil (k3d.cuh) as one sum of products: 4 ksum x0 minus every
      // coupling kappa (sum) times its neighbour, over 12
      V px1[2], py1[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        px1[i] = kk[1][i][0] + kk[1][i][1];
        py1[i] = kk[1][0][i] + kk[1][1][i];
      }
      const V ps1 = px1[0] + px1[1];
      typename S::D t = S::dzero();
      S::dadd(t, S::scale2(ps0 + ps1, 4.f), v[1][1][1]);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int oz = c >> 2, oy = (c >> 1) & 1, ox = c & 1;
        S::dadd(t, -kk[oz][oy][ox], v[2 * oz][2 * oy][2 * ox]);
      }
#pragma unroll
      for (int oy = 0; oy < 2; ++oy)
#pragma unroll
        for (int ox = 0; ox < 2; ++ox)
          S::dadd(t, -(kk[0][oy][ox] + kk[1][oy][ox]), v[1][2 * oy][2 * ox]);
#pragma unroll
      for (int ox = 0; ox < 2; ++ox) {
        S::dadd(t, -py0[ox], v[0][1][2 * ox]);
        S::dadd(t, -py1[ox], v[2][1][2 * ox]);
      }
#pragma unroll
      for (int oy = 0; oy < 2; ++oy) {
        S::dadd(t, -px0[oy], v[0][2 * oy][1]);
        S::dadd(t, -px1[oy], v[2][2 * oy][1]);
      }
      S::st(a.y, unit, a.nvf, (int)(base + W2 * kz), S::dget(t) * hv12);
      if constexpr (OVS) {
        V kr[2][2][2];
#pragma unroll
        for (int sz = 0; sz < 2; ++sz)
#pragma unroll
          for (int sy = 0; sy < 2; ++sy)
#pragma unroll
            for (int sx = 0; sx < 2; ++sx)
              kr[sz][sy][sx] = in_r(kx - 1 + sx, ky - 1 + sy, kz - 1 + sz) ? kk[sz][sy][sx]
                                                                           : S::zero();
        S::st(a.yR, unit, a.nvf, (int)(base + W2 * kz),
              hv * q1_apply3d_v<V>(v, kr, third, twelfth));
      }
      elem_plane(kz - 1, lo, v[1][1][1]);
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
          kk[0][i][j] = kk[1][i][j];
          lo[i][j] = up[i][j];
        }
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        px0[i] = px1[i];
        py0[i] = py1[i];
      }
      ps0 = ps1;
    }
    // the top element plane nf - 1 (its upper nodes are boundary nodes, value 0)
    elem_plane(nf - 1, lo, S::zero());
#pragma unroll
    for (int c = 0; c < 4; ++c) close(c);
  }
  __syncthreads();
  double *g = a.g + (size_t)pt * a.nc * a.R + r;
  for (int i = threadIdx.x; i < a.nc; i += F3_THREADS)
    if (bins[i] != 0.0) atomicAdd(&g[(size_t)i * a.R], -a.s * bins[i]);
}

// out = scale P^T y on the coarse lattice (one thread per coarse lattice entry; out FP64).
template <class S>
__global__ void __launch_bounds__(F3_THREADS) k_restrict3d(int nf, int lgr, const double *yf,
                                                           int nvf, double scale, double *outc,
                                                           int nvc) {
  using V = typename S::V;
  const int unit = blockIdx.y;
  const int rho = 1 << lgr, ncg = nf >> lgr, Wc = ncg + 1, Wf = nf + 1;
  const int k = blockIdx.x * F3_THREADS + threadIdx.x;
  if (k >= nvc) return;
  double *o = outc + (size_t)unit * nvc;
  const int Kx = k % Wc, Ky = (k / Wc) % Wc, Kz = k / (Wc * Wc);
  if (k >= Wc * Wc * Wc || Kx == 0 || Ky == 0 || Kz == 0 || Kx == ncg || Ky == ncg ||
      Kz == ncg) {
    o[k] = 0.0;
    return;
  }
  const float ir = 1.0f / rho;  // exact: rho is a power of two
  V s = S::zero();
  for (int dz = 1 - rho; dz < rho; ++dz) {
    const float wz = 1.0f - fabsf((float)dz) * ir;
    V sy = S::zero();
    for (int dy = 1 - rho; dy < rho; ++dy) {
      const float wy = 1.0f - fabsf((float)dy) * ir;
      const int row = Wf * ((Kz * rho + dz) * Wf + Ky * rho + dy);
      V sx = S::zero();
      for (int dx = 1 - rho; dx < rho; ++dx)
        sx += S::ld(yf, unit, nvf, row + Kx * rho + dx) * (1.0f - fabsf((float)dx) * ir);
      sy += sx * wy;
    }
    s += sy * wz;
  }
  o[k] = scale * S::to(s);
}

// phi += P x_c: one thread per coarse cell; the cell's rho^3 fine nodes (lower corners
// included) get the trilinear interpolant of its eight coarse values (x FP64).
template <class S>
__global__ void __launch_bounds__(F3_THREADS) k_prolong_add3d(int nf, int lgr, const double *xc,
                                                              int nvc, double *phif, int nvf) {
  using V = typename S::V;
  const int unit = blockIdx.y;
  const int rho = 1 << lgr, ncg = nf >> lgr, Wc = ncg + 1, Wf = nf + 1;
  const int cell = blockIdx.x * F3_THREADS + threadIdx.x;
  if (cell >= ncg * ncg * ncg) return;
  const int bx = cell % ncg, by = (cell / ncg) % ncg, bz = cell / (ncg * ncg);
  const double *x = xc + (size_t)unit * nvc + bx + (size_t)Wc * (by + (size_t)Wc * bz);
  const size_t sy = Wc, sz = (size_t)Wc * Wc;
  const V x000 = S::from(x[0]), x100 = S::from(x[1]), x010 = S::from(x[sy]),
          x110 = S::from(x[sy + 1]), x001 = S::from(x[sz]), x101 = S::from(x[sz + 1]),
          x011 = S::from(x[sz + sy]), x111 = S::from(x[sz + sy + 1]);
  const float ir = 1.0f / rho;
  for (int kz = 0; kz < rho; ++kz) {
    const float tz = kz * ir;
    for (int jy = 0; jy < rho; ++jy) {
      const float ty = jy * ir;
      const V a0 = x000 + (x010 - x000) * ty, a1 = x100 + (x110 - x100) * ty;
      const V b0 = x001 + (x011 - x001) * ty, b1 = x101 + (x111 - x101) * ty;
      const V c0 = a0 + (b0 - a0) * tz, c1 = a1 + (b1 - a1) * tz;
      const V dc = c1 - c0;
      const int row = (bx * rho) + Wf * ((by * rho + jy) + Wf * (bz * rho + kz));
      for (int ix = 0; ix < rho; ++ix) {
        const int k = row + ix;
        S::st(phif, unit, nvf, k, S::ld(phif, unit, nvf, k) + (c0 + dc * (ix * ir)));
      }
    }
  }
}

// ---- backward

__device__ __forceinline__ double phi3(const AdjArgs &a, size_t v, size_t k) {
  return a.ffs ? ff_to(ff_load(a.phi, v, a.nvf, (int)k)) : a.phi[v * a.nvf + k];
}

template <int R>
__global__ void __launch_bounds__(F3_THREADS) k_adj_combine3d(AdjArgs a) {
  const int pt = blockIdx.y;
  const int nf = a.nf, Wf = nf + 1, lgr = a.lgr, ncg = nf >> lgr, Wc = ncg + 1;
  const int k = blockIdx.x * F3_THREADS + threadIdx.x;
  if (k >= Wf * Wf * Wf) return;
  const int fx = k % Wf, fy = (k / Wf) % Wf, fz = k / (Wf * Wf);
  double wh[R * R];
  const double *Wp = a.W + (size_t)pt * R * R;
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int s = 0; s < R; ++s) wh[r * R + s] = (Wp[r * R + s] + Wp[s * R + r]) * a.inv_vol;
  double phi[R];
#pragma unroll
  for (int r = 0; r < R; ++r) phi[r] = phi3(a, (size_t)pt * R + r, k);
  const int bx = min(fx >> lgr, ncg - 1), by = min(fy >> lgr, ncg - 1), bz = min(fz >> lgr, ncg - 1);
  const double ir = 1.0 / (1 << lgr);
  const double tx = (fx - (bx << lgr)) * ir, ty = (fy - (by << lgr)) * ir,
               tz = (fz - (bz << lgr)) * ir;
  const size_t c0 = bx + (size_t)Wc * (by + (size_t)Wc * bz), sy = Wc, sz = (size_t)Wc * Wc;
#pragma unroll
  for (int s = 0; s < R; ++s) {
    double x = 0.0;
    if (!a.overs)
#pragma unroll
      for (int r = 0; r < R; ++r) x += wh[r * R + s] * phi[r];
    double pm = 0.0;
    if (a.mu) {
      const double *m = a.mu + ((size_t)pt * R + s) * a.nvc + c0;
      const double e00 = (1 - tx) * m[0] + tx * m[1], e10 = (1 - tx) * m[sy] + tx * m[sy + 1];
      const double e01 = (1 - tx) * m[sz] + tx * m[sz + 1];
      const double e11 = (1 - tx) * m[sz + sy] + tx * m[sz + sy + 1];
      pm = (1 - tz) * ((1 - ty) * e00 + ty * e10) + tz * ((1 - ty) * e01 + ty * e11);
    }
    const size_t o = ((size_t)pt * R + s) * a.nvf + k;
    a.psi1[o] = x - pm;
    a.psi2[o] = 0.5 * x - pm;
  }
}

// dL/dkappa per coarse element: one thread per (point, coarse element).
template <int R>
__global__ void __launch_bounds__(F3_THREADS) k_adj_grad3d(AdjArgs a, double hf) {
  const int pt = blockIdx.y;
  const int nf = a.nf, Wf = nf + 1, lgr = a.lgr, rho = 1 << lgr, ncg = nf >> lgr;
  const int E = blockIdx.x * F3_THREADS + threadIdx.x;
  if (E >= ncg * ncg * ncg) return;
  const int Ex = E % ncg, Ey = (E / ncg) % ncg, Ez = E / (ncg * ncg);
  const size_t sy = Wf, sz = (size_t)Wf * Wf;
  double g = 0.0;
  if (a.overs) {
    // direct term sum_rs W_rs Phi_r^T Khat Phi_s / |R_p| on the elements inside R_p (R_p is a
    // union of level-n elements: test one fine element's period)
    const int P = a.P, o = a.overs;
    const int px = (Ex * rho) >> a.lgmf, py = (Ey * rho) >> a.lgmf, pz = (Ez * rho) >> a.lgmf;
    if (px >= o && px < P - o && py >= o && py < P - o && pz >= o && pz < P - o) {
      const double *Wp = a.W + (size_t)pt * R * R;
      const size_t off[8] = {0, 1, sy, sy + 1, sz, sz + 1, sz + sy, sz + sy + 1};
      for (int kz = 0; kz < rho; ++kz)
        for (int jy = 0; jy < rho; ++jy)
          for (int ix = 0; ix < rho; ++ix) {
            const size_t k0 = (Ex * rho + ix) + sy * (Ey * rho + jy) + sz * (Ez * rho + kz);
            for (int s = 0; s < R; ++s) {
              double kp[8];
              {
                double p[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) p[c] = phi3(a, (size_t)pt * R + s, k0 + off[c]);
#pragma unroll
                for (int c = 0; c < 8; ++c)
                  kp[c] = p[c] * (1.0 / 3.0) -
                          (p[c ^ 3] + p[c ^ 5] + p[c ^ 6] + p[c ^ 7]) * (1.0 / 12.0);
              }
              for (int r = 0; r < R; ++r) {
                const double w = Wp[r * R + s];
                if (w == 0.0) continue;
                double e = 0.0;
#pragma unroll
                for (int c = 0; c < 8; ++c) e += phi3(a, (size_t)pt * R + r, k0 + off[c]) * kp[c];
                g += w * a.inv_vol * e;
              }
            }
          }
    }
  }
  for (int kz = 0; kz < rho; ++kz)
    for (int jy = 0; jy < rho; ++jy)
      for (int ix = 0; ix < rho; ++ix) {
        const size_t k0 = (Ex * rho + ix) + sy * (Ey * rho + jy) + sz * (Ez * rho + kz);
        const size_t off[8] = {0, 1, sy, sy + 1, sz, sz + 1, sz + sy, sz + sy + 1};
#pragma unroll
        for (int s = 0; s < R; ++s) {
          const size_t o = ((size_t)pt * R + s) * a.nvf + k0;
          double p[8], q[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            p[c] = phi3(a, (size_t)pt * R + s, k0 + off[c]);
            q[c] = a.psi2[o + off[c]];
          }
          // Khat p at corner c: 1/3 p_c - 1/12 (sum of the 3 face-diagonal corners c^3, c^5,
          // c^6 and the opposite corner c^7); axis neighbours do not couple
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const double kp = p[c] * (1.0 / 3.0) -
                              (p[c ^ 3] + p[c ^ 5] + p[c ^ 6] + p[c ^ 7]) * (1.0 / 12.0);
            g += q[c] * kp;
          }
        }
      }
  a.dkappa[(size_t)pt * ncg * ncg * ncg + E] = g * hf;
}

template <int NCN>
__global__ void __launch_bounds__(F3_THREADS) k_adj_seed3d(AdjArgs a, double hf) {
  const int unit = blockIdx.y;
  const int R = a.R, pt = unit / R, r = unit % R;
  const int nf = a.nf, Wf = nf + 1, lgr = a.lgr, ncg = nf >> lgr, nc = a.nc;
  const int lgmf = a.lgmf, P = a.P, nq3 = P * P * P;
  __shared__ double sig[MCH_MAX_NC3];
  for (int b = threadIdx.x; b < nc; b += F3_THREADS) {
    double sgm = 0.0;
    const double *Wp = a.W + (size_t)pt * R * R;
    if (!a.overs)
      for (int s = 0; s < R; ++s)
        sgm += (Wp[r * R + s] + Wp[s * R + r]) * a.inv_vol * a.lam[((size_t)pt * R + s) * nc + b];
    if (a.lamadj) sgm -= a.lamadj[((size_t)pt * R + r) * nc + b];
    sig[b] = sgm * a.inv_rho2;
  }
  __syncthreads();
  const int k = blockIdx.x * F3_THREADS + threadIdx.x;
  if (k >= Wf * Wf * Wf) return;
  const int fx = k % Wf, fy = (k / Wf) % Wf, fz = k / (Wf * Wf);
  if (fx == 0 || fy == 0 || fz == 0 || fx == nf || fy == nf || fz == nf) return;
  const double *kc = a.kappa_c + (size_t)pt * ncg * ncg * ncg;
  const uint8_t *lc = a.labels_c + (size_t)pt * ncg * ncg * ncg;
  const double *ps = a.psi1 + ((size_t)pt * R + r) * a.nvf;
  double v[3][3][3], kk[2][2][2];
  double u = 0.0;
  const size_t W2 = (size_t)Wf * Wf;
#pragma unroll
  for (int dz = 0; dz < 3; ++dz)
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) v[dz][dy][dx] = ps[k + (dx - 1) + Wf * (dy - 1) + W2 * (dz - 1)];
#pragma unroll
  for (int sz = 0; sz < 2; ++sz)
#pragma unroll
    for (int sy = 0; sy < 2; ++sy)
#pragma unroll
      for (int sx = 0; sx < 2; ++sx) {
        const int ex = fx - 1 + sx, ey = fy - 1 + sy, ez = fz - 1 + sz;
        const size_t c = cidx(ex >> lgr, ey >> lgr, ez >> lgr, ncg);
        kk[sz][sy][sx] = kc[c];
        const int l = min((int)lc[c], nc / nq3 - 1);
        const int bin = l * nq3 + ((ez >> lgmf) * P + (ey >> lgmf)) * P + (ex >> lgmf);
        u += sig[bin];
      }
  u += hf * q1_apply3d<double>(v, kk);
  if (a.V) u += a.V[((size_t)pt * R + r) * a.nvf + k];
  for (int t = 0; t < a.slots; ++t) {
    const double w = a.par_w[pt * a.slots + t];
    if (w != 0.0) atomicAdd(&a.par_V[pt * a.slots + t][(size_t)r * a.nvf + k], w * u);
  }
}

// Oversampling: V_r += sum_s What_rs A_{1,R} Phi_s at the interior fine nodes, with kappa
// zero on the fine elements outside R_p.
template <int R>
__global__ void __launch_bounds__(F3_THREADS) k_adj_own3d(AdjArgs a, double hf) {
  const int pt = blockIdx.y;
  const int nf = a.nf, Wf = nf + 1, lgr = a.lgr, ncg = nf >> lgr;
  const int k = blockIdx.x * F3_THREADS + threadIdx.x;
  if (k >= Wf * Wf * Wf) return;
  const int fx = k % Wf, fy = (k / Wf) % Wf, fz = k / (Wf * Wf);
  if (fx == 0 || fy == 0 || fz == 0 || fx == nf || fy == nf || fz == nf) return;
  const int P = a.P, o = a.overs;
  const double *kc = a.kappa_c + (size_t)pt * ncg * ncg * ncg;
  double kk[2][2][2];
#pragma unroll
  for (int sz = 0; sz < 2; ++sz)
#pragma unroll
    for (int sy = 0; sy < 2; ++sy)
#pragma unroll
      for (int sx = 0; sx < 2; ++sx) {
        const int ex = fx - 1 + sx, ey = fy - 1 + sy, ez = fz - 1 + sz;
        const int px = ex >> a.lgmf, py = ey >> a.lgmf, pz = ez >> a.lgmf;
        const bool in = px >= o && px < P - o && py >= o && py < P - o && pz >= o && pz < P - o;
        kk[sz][sy][sx] = in ? kc[cidx(ex >> lgr, ey >> lgr, ez >> lgr, ncg)] : 0.0;
      }
  const size_t W2 = (size_t)Wf * Wf;
  double y[R];
#pragma unroll
  for (int s = 0; s < R; ++s) {
    double v[3][3][3];
    const size_t vs = (size_t)pt * R + s;
#pragma unroll
    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx)
          v[dz][dy][dx] = phi3(a, vs, k + (dx - 1) + Wf * (dy - 1) + W2 * (dz - 1));
    y[s] = hf * q1_apply3d<double>(v, kk);
  }
  const double *Wp = a.W + (size_t)pt * R * R;
  double *V = const_cast<double *>(a.V);
#pragma unroll
  for (int r = 0; r < R; ++r) {
    double u = 0.0;
#pragma unroll
    for (int s = 0; s < R; ++s) u += (Wp[r * R + s] + Wp[s * R + r]) * a.inv_vol * y[s];
    V[((size_t)pt * R + r) * a.nvf + k] += u;
  }
}

}  // namespace

cudaError_t launch_adj_own3d(const AdjArgs &a, double hf, cudaStream_t st) {
  const int Wf = a.nf + 1;
  dim3 grid((Wf * Wf * Wf + F3_THREADS - 1) / F3_THREADS, a.npts);
  switch (a.R) {
    case 4: k_adj_own3d<4><<<grid, F3_THREADS, 0, st>>>(a, hf); break;
    case 8: k_adj_own3d<8><<<grid, F3_THREADS, 0, st>>>(a, hf); break;
    case 12: k_adj_own3d<12><<<grid, F3_THREADS, 0, st>>>(a, hf); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_apply3d(const ApplyArgs &a, double h, cudaStream_t st) {
  dim3 grid((a.nv + F3_THREADS - 1) / F3_THREADS, a.npts * a.R);
  k_apply3d<<<grid, F3_THREADS, 0, st>>>(a, h);
  return cudaGetLastError();
}

cudaError_t launch_interp3d(const ChildArgs &a, cudaStream_t st, bool ffs) {
  if (a.slots > 8) return cudaErrorInvalidValue;
  dim3 grid((a.nvf + F3_THREADS - 1) / F3_THREADS, a.npts * a.R);
  if (ffs) k_interp3d<FFS><<<grid, F3_THREADS, 0, st>>>(a);
  else k_interp3d<F64S><<<grid, F3_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fine_apply3d(const ChildArgs &a, double hf, cudaStream_t st, bool ffs) {
  if (a.nc > MCH_MAX_NC3 || (ffs && !a.kappa_ff)) return cudaErrorInvalidValue;
  const int ni = a.nf - 1;
  dim3 grid((ni * ni + F3_THREADS - 1) / F3_THREADS, a.npts * a.R);
  auto go = [&](auto kern) { kern<<<grid, F3_THREADS, 0, st>>>(a, hf); };
  const bool ovs = a.yR != nullptr;
  if (ffs) ovs ? go(k_fine_apply3d<FFS, true>) : go(k_fine_apply3d<FFS, false>);
  else ovs ? go(k_fine_apply3d<F64S, true>) : go(k_fine_apply3d<F64S, false>);
  return cudaGetLastError();
}

cudaError_t launch_restrict3d(int npts, int R, int nf, int rho, const double *yf, int nvf,
                              double scale, double *outc, int nvc, cudaStream_t st, bool ffs) {
  dim3 grid((nvc + F3_THREADS - 1) / F3_THREADS, npts * R);
  if (ffs) k_restrict3d<FFS><<<grid, F3_THREADS, 0, st>>>(nf, __builtin_ctz(rho), yf, nvf, scale, outc, nvc);
  else k_restrict3d<F64S><<<grid, F3_THREADS, 0, st>>>(nf, __builtin_ctz(rho), yf, nvf, scale, outc, nvc);
  return cudaGetLastError();
}

cudaError_t launch_prolong_add3d(int npts, int R, int nf, int rho, const double *xc, int nvc,
                                 double *phif, int nvf, cudaStream_t st, bool ffs) {
  const int ncg = nf / rho;
  dim3 grid((ncg * ncg * ncg + F3_THREADS - 1) / F3_THREADS, npts * R);
  if (ffs) k_prolong_add3d<FFS><<<grid, F3_THREADS, 0, st>>>(nf, __builtin_ctz(rho), xc, nvc, phif, nvf);
  else k_prolong_add3d<F64S><<<grid, F3_THREADS, 0, st>>>(nf, __builtin_ctz(rho), xc, nvc, phif, nvf);
  return cudaGetLastError();
}

cudaError_t launch_adj_combine3d(const AdjArgs &a, cudaStream_t st) {
  const int Wf = a.nf + 1;
  dim3 grid((Wf * Wf * Wf + F3_THREADS - 1) / F3_THREADS, a.npts);
  switch (a.R) {
    case 4: k_adj_combine3d<4><<<grid, F3_THREADS, 0, st>>>(a); break;
    case 8: k_adj_combine3d<8><<<grid, F3_THREADS, 0, st>>>(a); break;
    case 12: k_adj_combine3d<12><<<grid, F3_THREADS, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_adj_grad3d(const AdjArgs &a, double hf, cudaStream_t st) {
  const int ncg = a.nf >> a.lgr;
  dim3 grid((ncg * ncg * ncg + F3_THREADS - 1) / F3_THREADS, a.npts);
  switch (a.R) {
    case 4: k_adj_grad3d<4><<<grid, F3_THREADS, 0, st>>>(a, hf); break;
    case 8: k_adj_grad3d<8><<<grid, F3_THREADS, 0, st>>>(a, hf); break;
    case 12: k_adj_grad3d<12><<<grid, F3_THREADS, 0, st>>>(a, hf); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_adj_seed3d(const AdjArgs &a, double hf, cudaStream_t st) {
  if (a.nc > MCH_MAX_NC3) return cudaErrorInvalidValue;
  const int Wf = a.nf + 1;
  dim3 grid((Wf * Wf * Wf + F3_THREADS - 1) / F3_THREADS, a.npts * a.R);
  k_adj_seed3d<2><<<grid, F3_THREADS, 0, st>>>(a, hf);
  return cudaGetLastError();
}

}  // namespace mch
