// Backward pass: gradient of L = sum_levels sum_points sum_rs W_p[r,s] E_p[r,s] with respect to
// kappa of every element of every level (FP64).
//
// Derived from the energy form of Sec. 3, Eq. (phi_abstract) and the correction problems of
// Sec. 3.3 (Eqs. phi_avar_corrector, phi_grad_corrector). For a point p of level n with
// cell functions Phi (level-1 grid), forward multipliers lambda (A_n Xi + Ct^T lambda = b at
// convergence), What = (W + W^T) / |R_p|, and seeds V_r = dL/dPhi_r from its children:
//   adjoint solve  A_n mu_r + Ct^T lambda'_r = P^T V_r,  Ct mu_r = 0   (same level kernel)
//   Psi'_s = sum_r What_rs Phi_r - P mu_s,   Psi_s = 1/2 sum_r What_rs Phi_r - P mu_s
//   dL/dkappa_E = sum_{fine e in E} sum_s Psi_s|e^T Khat Phi_s|e            (k_adj_grad2d)
//   U_r = V_r + A_1 Psi'_r + rho^-2 Ct_1^T (sum_s What_rs lambda_s - lambda'_r)
//   V_t,r += c_t U_r for the parents t                                      (k_adj_seed2d)
// (Ct_1 is the fine-grid constraint operator in the library's scaling; rho^-2 converts the
// level-n multipliers to it.)
#include "common.cuh"
#include "ff.cuh"
#include "kernels.h"

namespace mch {

namespace {

// cell function entry k of vector v (FP64 or float-float storage)
__device__ __forceinline__ double phi_at(const AdjArgs &a, size_t v, int k) {
  return a.ffs ? ff_to(ff_load(a.phi, v, a.nvf, k)) : a.phi[v * a.nvf + k];
}

// Psi' and Psi at every fine node of every point.
template <int R>
__global__ void k_adj_combine2d(AdjArgs a) {
  const int pt = blockIdx.y;
  const int nf = a.nf, Wf = nf + 1, lgr = a.lgr, rho = 1 << lgr, ncg = nf >> lgr, Wc = ncg + 1;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Wf * Wf) return;
  const int fx = k % Wf, fy = k / Wf;
  double wh[R * R];
  const double *Wp = a.W + (size_t)pt * R * R;
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int s = 0; s < R; ++s) wh[r * R + s] = (Wp[r * R + s] + Wp[s * R + r]) * a.inv_vol;
  double phi[R];
#pragma unroll
  for (int r = 0; r < R; ++r) phi[r] = phi_at(a, (size_t)pt * R + r, k);
  // bilinear weights of P mu at this fine node
  const int bx = min(fx >> lgr, ncg - 1), by = min(fy >> lgr, ncg - 1);
  const double ir = 1.0 / rho;  // exact: rho is a power of two
  const double tx = double(fx - (bx << lgr)) * ir, ty = double(fy - (by << lgr)) * ir;
  const double w00 = (1 - tx) * (1 - ty), w10 = tx * (1 - ty), w01 = (1 - tx) * ty, w11 = tx * ty;
  const int c0 = bx + Wc * by;
#pragma unroll
  for (int s = 0; s < R; ++s) {
    double x = 0.0;
    if (!a.overs)
#pragma unroll
      for (int r = 0; r < R; ++r) x += wh[r * R + s] * phi[r];
    double pm = 0.0;
    if (a.mu) {
      const double *m = a.mu + ((size_t)pt * R + s) * a.nvc + c0;
      pm = w00 * m[0] + w10 * m[1] + w01 * m[Wc] + w11 * m[Wc + 1];
    }
    const size_t o = ((size_t)pt * R + s) * a.nvf + k;
    a.psi1[o] = x - pm;
    a.psi2[o] = 0.5 * x - pm;
  }
}

// dL/dkappa of each level-n element: one thread per (point, coarse element) sums its rho^2
// fine elements.
template <int R>
__global__ void k_adj_grad2d(AdjArgs a) {
  const int pt = blockIdx.y;
  const int nf = a.nf, Wf = nf + 1, lgr = a.lgr, rho = 1 << lgr, ncg = nf >> lgr;
  const int E = blockIdx.x * blockDim.x + threadIdx.x;
  if (E >= ncg * ncg) return;
  const int Ex = E % ncg, Ey = E / ncg;
  double g = 0.0;
  if (a.overs) {
    // direct term sum_rs W_rs Phi_r^T Khat Phi_s / |R_p| on elements inside R_p (R_p is a
    // union of level-n elements: test one fine element's period)
    const int P = a.P, o = a.overs;
    const int px = (Ex * rho) >> a.lgmf, py = (Ey * rho) >> a.lgmf;
    if (px >= o && px < P - o && py >= o && py < P - o) {
      const double *Wp = a.W + (size_t)pt * R * R;
      for (int j = 0; j < rho; ++j)
        for (int i = 0; i < rho; ++i) {
          const int k = (Ex * rho + i) + Wf * (Ey * rho + j);
          double p0[R], p1[R], p2[R], p3[R];
#pragma unroll
          for (int s = 0; s < R; ++s) {
            const size_t v = (size_t)pt * R + s;
            p0[s] = phi_at(a, v, k);
            p1[s] = phi_at(a, v, k + 1);
            p2[s] = phi_at(a, v, k + Wf);
            p3[s] = phi_at(a, v, k + Wf + 1);
          }
#pragma unroll
          for (int s = 0; s < R; ++s) {
            const double k0 = (4 * p0[s] - p1[s] - p2[s] - 2 * p3[s]) * (1.0 / 6.0);
            const double k1 = (4 * p1[s] - p0[s] - p3[s] - 2 * p2[s]) * (1.0 / 6.0);
            const double k2 = (4 * p2[s] - p0[s] - p3[s] - 2 * p1[s]) * (1.0 / 6.0);
            const double k3 = (4 * p3[s] - p1[s] - p2[s] - 2 * p0[s]) * (1.0 / 6.0);
#pragma unroll
            for (int r = 0; r < R; ++r)
              g += Wp[r * R + s] * a.inv_vol *
                   (p0[r] * k0 + p1[r] * k1 + p2[r] * k2 + p3[r] * k3);
          }
        }
    }
  }
  for (int j = 0; j < rho; ++j)
    for (int i = 0; i < rho; ++i) {
      const int k = (Ex * rho + i) + Wf * (Ey * rho + j);
#pragma unroll
      for (int s = 0; s < R; ++s) {
        const size_t o = ((size_t)pt * R + s) * a.nvf + k;
        const size_t v = (size_t)pt * R + s;
        const double p0 = phi_at(a, v, k), p1 = phi_at(a, v, k + 1), p2 = phi_at(a, v, k + Wf),
                     p3 = phi_at(a, v, k + Wf + 1);
        const double q0 = a.psi2[o], q1 = a.psi2[o + 1], q2 = a.psi2[o + Wf], q3 = a.psi2[o + Wf + 1];
        // unit-square Q1 element matrix times the corner values (corners 0 1 / 2 3, 0 and
        // 3 opposite): 1/6 (4 v_a - v_edge - v_edge - 2 v_opposite)
        const double k0 = 4 * p0 - p1 - p2 - 2 * p3, k1 = 4 * p1 - p0 - p3 - 2 * p2;
        const double k2 = 4 * p2 - p0 - p3 - 2 * p1, k3 = 4 * p3 - p1 - p2 - 2 * p0;
        g += (q0 * k0 + q1 * k1 + q2 * k2 + q3 * k3) * (1.0 / 6.0);
      }
    }
  a.dkappa[(size_t)pt * ncg * ncg + E] = g;
}

// U_r at every interior fine node of every (point, function), pushed to the parents' seeds.
__global__ void k_adj_seed2d(AdjArgs a) {
  const int unit = blockIdx.y;
  const int R = a.R, pt = unit / R, r = unit % R;
  const int nf = a.nf, Wf = nf + 1, lgr = a.lgr, ncg = nf >> lgr, nc = a.nc;
  const int lgmf = a.lgmf, P = a.P, nq = a.P * a.P;
  __shared__ double sig[MCH_MAX_NC];
  // sigma = sum_s What_rs lambda_s - lambda'_r, scaled by rho^-2
  for (int b = threadIdx.x; b < nc; b += blockDim.x) {
    double sgm = 0.0;
    const double *Wp = a.W + (size_t)pt * R * R;
    if (!a.overs)
      for (int s = 0; s < R; ++s)
        sgm += (Wp[r * R + s] + Wp[s * R + r]) * a.inv_vol * a.lam[((size_t)pt * R + s) * nc + b];
    if (a.lamadj) sgm -= a.lamadj[((size_t)pt * R + r) * nc + b];
    sig[b] = sgm * a.inv_rho2;
  }
  __syncthreads();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Wf * Wf) return;
  const int fx = k % Wf, fy = k / Wf;
  if (fx == 0 || fy == 0 || fx == nf || fy == nf) return;
  const double *kc = a.kappa_c + (size_t)pt * ncg * ncg;
  const uint8_t *lc = a.labels_c + (size_t)pt * ncg * ncg;
  const double *ps = a.psi1 + ((size_t)pt * R + r) * a.nvf + k;
  auto K = [&](int ex, int ey) { return kc[(ex >> lgr) + ncg * (ey >> lgr)]; };
  const int Nm1 = nc / nq - 1;
  auto bin = [&](int ex, int ey) {
    const int l = min((int)lc[(ex >> lgr) + ncg * (ey >> lgr)], Nm1);
    return l * nq + (ey >> lgmf) * P + (ex >> lgmf);
  };
  double u = q1_apply(K(fx - 1, fy - 1), K(fx, fy - 1), K(fx - 1, fy), K(fx, fy), ps[-Wf - 1],
                      ps[-Wf], ps[-Wf + 1], ps[-1], ps[0], ps[1], ps[Wf - 1], ps[Wf], ps[Wf + 1]);
  u += sig[bin(fx - 1, fy - 1)] + sig[bin(fx, fy - 1)] + sig[bin(fx - 1, fy)] + sig[bin(fx, fy)];
  if (a.V) u += a.V[((size_t)pt * R + r) * a.nvf + k];
  for (int t = 0; t < a.slots; ++t) {
    const double w = a.par_w[pt * a.slots + t];
    if (w != 0.0) atomicAdd(&a.par_V[pt * a.slots + t][(size_t)r * a.nvf + k], w * u);
  }
}

// Oversampling: V_r += sum_s What_rs A_{1,R} Phi_s at the interior fine nodes, with kappa
// zero on the fine elements outside R_p.
template <int R>
__global__ void k_adj_own2d(AdjArgs a) {
  const int pt = blockIdx.y;
  const int nf = a.nf, Wf = nf + 1, lgr = a.lgr, ncg = nf >> lgr;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Wf * Wf) return;
  const int fx = k % Wf, fy = k / Wf;
  if (fx == 0 || fy == 0 || fx == nf || fy == nf) return;
  const int P = a.P, o = a.overs;
  const double *kc = a.kappa_c + (size_t)pt * ncg * ncg;
  auto K = [&](int ex, int ey) {
    const int px = ex >> a.lgmf, py = ey >> a.lgmf;
    const bool in = px >= o && px < P - o && py >= o && py < P - o;
    return in ? kc[(ex >> lgr) + ncg * (ey >> lgr)] : 0.0;
  };
  const double kSW = K(fx - 1, fy - 1), kSE = K(fx, fy - 1), kNW = K(fx - 1, fy), kNE = K(fx, fy);
  double y[R];
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const size_t v = (size_t)pt * R + s;
    y[s] = q1_apply(kSW, kSE, kNW, kNE, phi_at(a, v, k - Wf - 1), phi_at(a, v, k - Wf),
                    phi_at(a, v, k - Wf + 1), phi_at(a, v, k - 1), phi_at(a, v, k),
                    phi_at(a, v, k + 1), phi_at(a, v, k + Wf - 1), phi_at(a, v, k + Wf),
                    phi_at(a, v, k + Wf + 1));
  }
  const double *Wp = a.W + (size_t)pt * R * R;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    double u = 0.0;
#pragma unroll
    for (int s = 0; s < R; ++s) u += (Wp[r * R + s] + Wp[s * R + r]) * a.inv_vol * y[s];
    double *V = const_cast<double *>(a.V);
    V[((size_t)pt * R + r) * a.nvf + k] += u;
  }
}

}  // namespace

cudaError_t launch_adj_own2d(const AdjArgs &a, cudaStream_t st) {
  const int Wf = a.nf + 1;
  dim3 grid((Wf * Wf + 127) / 128, a.npts);
  switch (a.R) {
    case 3: k_adj_own2d<3><<<grid, 128, 0, st>>>(a); break;
    case 6: k_adj_own2d<6><<<grid, 128, 0, st>>>(a); break;
    case 9: k_adj_own2d<9><<<grid, 128, 0, st>>>(a); break;
    case 12: k_adj_own2d<12><<<grid, 128, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_adj_combine2d(const AdjArgs &a, cudaStream_t st) {
  const int Wf = a.nf + 1;
  dim3 grid((Wf * Wf + 127) / 128, a.npts);
  switch (a.R) {
    case 3: k_adj_combine2d<3><<<grid, 128, 0, st>>>(a); break;
    case 6: k_adj_combine2d<6><<<grid, 128, 0, st>>>(a); break;
    case 9: k_adj_combine2d<9><<<grid, 128, 0, st>>>(a); break;
    case 12: k_adj_combine2d<12><<<grid, 128, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_adj_grad2d(const AdjArgs &a, cudaStream_t st) {
  const int ncg = a.nf >> a.lgr;
  dim3 grid((ncg * ncg + 127) / 128, a.npts);
  switch (a.R) {
    case 3: k_adj_grad2d<3><<<grid, 128, 0, st>>>(a); break;
    case 6: k_adj_grad2d<6><<<grid, 128, 0, st>>>(a); break;
    case 9: k_adj_grad2d<9><<<grid, 128, 0, st>>>(a); break;
    case 12: k_adj_grad2d<12><<<grid, 128, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_adj_seed2d(const AdjArgs &a, cudaStream_t st) {
  const int Wf = a.nf + 1;
  dim3 grid((Wf * Wf + 255) / 256, a.npts * a.R);
  k_adj_seed2d<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace mch
