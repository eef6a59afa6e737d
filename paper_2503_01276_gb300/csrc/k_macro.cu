// Macroscopic multicontinuum problem (Sec. 2, Eq. macro_eq) from the effective coefficients.
//
// Source (Eq. Bs_defi, b_j, with the Gaussian source of the numerical examples of Sec. 5):
// fbar_j(p) = (1/|R_p|) int_{R_p} f phi_j for the N constant cell functions of a point, with
// f = w_j exp(-alpha |x - c|^2) in continuum j sampled at the centroids of the level-1-grid
// elements (x = x_p + y; the element's continuum is that of the level-n element containing
// it). For this piecewise-constant f and the Q1 phi_j the integral is exact:
// sum_e f_e (h^d / 2^d) sum_{corners b} phi_j(b).
//
// Solve: the coarse blocks K_p = x_p + [-H/2, H/2]^d of all macropoints are the elements of
// the macro mesh; U_j is Q1 on their (M+1)^d vertices with zero Dirichlet data on the outer
// boundary, and
//   sum_p int_{K_p} w(V)^T E_p w(U) = sum_p int_{K_p} sum_j fbar_j(p) V_j,
// w(U) = (U_i, d_m U_i) in the order of the cell functions (r = i, r = N + i d + m), E_p and
// fbar_p constant on K_p, integrated exactly with 2 Gauss points per axis. The system is
// symmetric positive definite when every E_p is; one CTA runs matrix-free Jacobi-PCG in FP64
// (the macro system has at most a few thousand unknowns), bounded by max_iter.
#include "ff.cuh"
#include "kernels.h"

namespace mch {

namespace {

constexpr int MS_THREADS = 256;
constexpr int MC_THREADS = 256;

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

template <class S, int D>
__global__ void __launch_bounds__(MS_THREADS) k_macro_source(MacroSourceArgs a) {
  const int pt = blockIdx.x, tid = threadIdx.x;
  const int nf = a.nf, W = nf + 1, N = a.N, ncg = nf >> a.lgr;
  const double h = a.rve_len / nf;
  const int mper = nf / a.P;
  const int lo = a.overs * mper, hi = (a.P - a.overs) * mper;
  const uint8_t *lab = a.labels + (size_t)pt * (D == 3 ? ncg * ncg * ncg : ncg * ncg);
  const double *xp = a.xp + (size_t)pt * D;
  const int nel = D == 3 ? nf * nf * nf : nf * nf;
  double acc[MCH_MACRO_MAXN];
#pragma unroll
  for (int j = 0; j < MCH_MACRO_MAXN; ++j) acc[j] = 0.0;
  for (int e = tid; e < nel; e += MS_THREADS) {
    int ec[3] = {e % nf, (e / nf) % nf, D == 3 ? e / (nf * nf) : 0};
    bool inside = true;
    double r2 = 0.0;
    int li = 0, stride = 1;
#pragma unroll
    for (int m = 0; m < D; ++m) {
      inside = inside && ec[m] >= lo && ec[m] < hi;
      const double x = xp[m] - 0.5 * a.rve_len + (ec[m] + 0.5) * h - a.c[m];
      r2 += x * x;
      li += (ec[m] >> a.lgr) * stride;
      stride *= ncg;
    }
    if (!inside) continue;
    const int l = min((int)lab[li], N - 1);
    const double f = a.w[l] * exp(-a.alpha * r2);
    const int base = ec[0] + W * (ec[1] + W * ec[2]);
#pragma unroll
    for (int j = 0; j < MCH_MACRO_MAXN; ++j) {
      if (j >= N) break;
      const typename S::P pj = S::vec(a.phi, (size_t)pt * a.R + j, a.nvf);
      double s = 0.0;
#pragma unroll
      for (int b = 0; b < (1 << D); ++b)
        s += S::to(S::ldv(pj, a.nvf, base + (b & 1) + W * ((b >> 1) & 1) + W * W * (b >> 2)));
      acc[j] += f * s;
    }
  }
  __shared__ double red[MS_THREADS / 32][MCH_MACRO_MAXN];
  const int lane = tid & 31, w = tid >> 5;
#pragma unroll
  for (int j = 0; j < MCH_MACRO_MAXN; ++j) {
    double v = acc[j];
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[w][j] = v;
  }
  __syncthreads();
  if (tid < N) {
    double s = 0.0;
    for (int ww = 0; ww < MS_THREADS / 32; ++ww) s += red[ww][tid];
    double hd = 1.0, side = (hi - lo) * h, vol = 1.0;
    for (int m = 0; m < D; ++m) {
      hd *= h;
      vol *= side;
    }
    a.fbar[(size_t)pt * N + tid] = s * hd / (1 << D) / vol;
  }
}

__global__ void k_macro_gather(int npts, int R, int N, const int *elem, const double *E,
                               const double *fbar, double *Eg, double *fg) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int per = R * R + N;
  if (t >= npts * per) return;
  const int p = t / per, k = t % per;
  const size_t e = (size_t)elem[p];
  if (k < R * R) Eg[e * R * R + k] = E[(size_t)p * R * R + k];
  else fg[e * N + (k - R * R)] = fbar[(size_t)p * N + (k - R * R)];
}

// block-wide sum of one double per thread (all threads of the CTA call it)
__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < MC_THREADS / 32; ++i) s += red[i];
  return s;
}

template <int D, int N>
__global__ void __launch_bounds__(MC_THREADS) k_macro_cg(MacroSolveArgs a) {
  constexpr int NB = 1 << D, R = N * (1 + D);
  const int M = a.M, Wn = M + 1;
  const int nn = D == 3 ? Wn * Wn * Wn : Wn * Wn;
  const int nu = N * nn, nel = D == 3 ? M * M * M : M * M;
  const int tid = threadIdx.x;
  const double H = a.H;
  double vol = 1.0;
  for (int m = 0; m < D; ++m) vol *= H;
  __shared__ double val[NB][NB], grad[NB][NB][D];  // [Gauss point][corner]
  __shared__ double red[MC_THREADS / 32];
  if (tid < NB * NB) {
    const int g = tid / NB, b = tid % NB;
    const double gp[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
    double f1[D];
#pragma unroll
    for (int m = 0; m < D; ++m) {
      const double xi = gp[(g >> m) & 1];
      f1[m] = ((b >> m) & 1) ? xi : 1.0 - xi;
    }
    double v = 1.0;
#pragma unroll
    for (int m = 0; m < D; ++m) v *= f1[m];
    val[g][b] = v;
#pragma unroll
    for (int m = 0; m < D; ++m) {
      double gr = ((b >> m) & 1) ? 1.0 / H : -1.0 / H;
#pragma unroll
      for (int o = 0; o < D; ++o)
        if (o != m) gr *= f1[o];
      grad[g][b][m] = gr;
    }
  }
  auto boundary = [&](int node) {
    int q = node;
#pragma unroll
    for (int m = 0; m < D; ++m) {
      const int c = q % Wn;
      if (c == 0 || c == M) return true;
      q /= Wn;
    }
    return false;
  };
  auto corner = [&](int e, int b) {
    const int ex = e % M, ey = (e / M) % M, ez = D == 3 ? e / (M * M) : 0;
    return (ex + (b & 1)) + Wn * ((ey + ((b >> 1) & 1)) + Wn * (ez + (b >> 2)));
  };
  // out += A v (element by element, atomics; boundary rows skipped)
  auto apply = [&](const double *v, double *out) {
    for (int e = tid; e < nel; e += MC_THREADS) {
      const double *Ee = a.E + (size_t)e * R * R;
      double pl[NB][N], yl[NB][N];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int node = corner(e, b);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          pl[b][i] = v[i * nn + node];
          yl[b][i] = 0.0;
        }
      }
#pragma unroll
      for (int g = 0; g < NB; ++g) {
        double w[R], y[R];
#pragma unroll
        for (int i = 0; i < N; ++i) {
          double s = 0.0;
#pragma unroll
          for (int b = 0; b < NB; ++b) s += val[g][b] * pl[b][i];
          w[i] = s;
#pragma unroll
          for (int m = 0; m < D; ++m) {
            double t = 0.0;
#pragma unroll
            for (int b = 0; b < NB; ++b) t += grad[g][b][m] * pl[b][i];
            w[N + i * D + m] = t;
          }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
          double s = 0.0;
#pragma unroll
          for (int c = 0; c < R; ++c) s += Ee[r * R + c] * w[c];
          y[r] = s * (vol / NB);
        }
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
          for (int j = 0; j < N; ++j) {
            double s = val[g][b] * y[j];
#pragma unroll
            for (int m = 0; m < D; ++m) s += grad[g][b][m] * y[N + j * D + m];
            yl[b][j] += s;
          }
      }
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int node = corner(e, b);
        if (boundary(node)) continue;
#pragma unroll
        for (int j = 0; j < N; ++j) atomicAdd(&out[j * nn + node], yl[b][j]);
      }
    }
  };

  // ---- load vector (into r) and Jacobi diagonal
  for (int k = tid; k < nu; k += MC_THREADS) {
    a.U[k] = 0.0;
    a.r[k] = 0.0;
    a.diag[k] = 0.0;
  }
  __syncthreads();
  for (int e = tid; e < nel; e += MC_THREADS) {
    const double *Ee = a.E + (size_t)e * R * R;
    for (int b = 0; b < NB; ++b) {
      const int node = corner(e, b);
      if (boundary(node)) continue;
      for (int j = 0; j < N; ++j) {
        atomicAdd(&a.r[j * nn + node], a.f[(size_t)e * N + j] * vol / NB);
        double dsum = 0.0;
        for (int g = 0; g < NB; ++g) {
          double wv[1 + D];
          int idx[1 + D];
          wv[0] = val[g][b];
          idx[0] = j;
          for (int m = 0; m < D; ++m) {
            wv[1 + m] = grad[g][b][m];
            idx[1 + m] = N + j * D + m;
          }
          double s = 0.0;
          for (int r = 0; r < 1 + D; ++r)
            for (int c = 0; c < 1 + D; ++c) s += wv[r] * Ee[idx[r] * R + idx[c]] * wv[c];
          dsum += s * (vol / NB);
        }
        atomicAdd(&a.diag[j * nn + node], dsum);
      }
    }
  }
  __syncthreads();
  double bb = 0.0, rz = 0.0;
  for (int k = tid; k < nu; k += MC_THREADS) {
    const bool bnd = boundary(k % nn);
    const double dg = bnd || !(a.diag[k] > 0.0) ? 1.0 : a.diag[k];
    a.diag[k] = dg;
    const double r = bnd ? 0.0 : a.r[k];
    a.r[k] = r;
    const double z = r / dg;
    a.p[k] = z;
    bb += r * r;
    rz += r * z;
  }
  bb = block_sum(bb, red);
  rz = block_sum(rz, red);
  const double bnorm = sqrt(bb);
  int it = 0;
  double rn = bnorm;
  if (bnorm > 0.0) {
    for (; it < a.max_iter; ++it) {
      for (int k = tid; k < nu; k += MC_THREADS) a.q[k] = 0.0;
      __syncthreads();
      apply(a.p, a.q);
      __syncthreads();
      double pq = 0.0;
      for (int k = tid; k < nu; k += MC_THREADS) pq += a.p[k] * a.q[k];
      pq = block_sum(pq, red);
      if (!(pq > 0.0)) break;
      const double alpha = rz / pq;
      double rr = 0.0, rz2 = 0.0;
      for (int k = tid; k < nu; k += MC_THREADS) {
        a.U[k] += alpha * a.p[k];
        const double r = a.r[k] - alpha * a.q[k];
        a.r[k] = r;
        rr += r * r;
        rz2 += r * r / a.diag[k];
      }
      rr = block_sum(rr, red);
      rz2 = block_sum(rz2, red);
      rn = sqrt(rr);
      if (rn <= a.tol * bnorm) {
        ++it;
        break;
      }
      const double beta = rz2 / rz;
      rz = rz2;
      for (int k = tid; k < nu; k += MC_THREADS) a.p[k] = a.r[k] / a.diag[k] + beta * a.p[k];
      __syncthreads();
    }
  }
  if (tid == 0) {
    *a.iters = it;
    *a.relres = bnorm > 0.0 ? rn / bnorm : 0.0;
  }
}

template <int D>
cudaError_t cg_dispatch(const MacroSolveArgs &a, cudaStream_t st) {
  switch (a.N) {
    case 1: k_macro_cg<D, 1><<<1, MC_THREADS, 0, st>>>(a); break;
    case 2: k_macro_cg<D, 2><<<1, MC_THREADS, 0, st>>>(a); break;
    case 3: k_macro_cg<D, 3><<<1, MC_THREADS, 0, st>>>(a); break;
    case 4: k_macro_cg<D, 4><<<1, MC_THREADS, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_macro_source(const MacroSourceArgs &a, bool ffs, cudaStream_t st) {
  if (a.N < 1 || a.N > MCH_MACRO_MAXN || a.npts <= 0 || (a.dim != 2 && a.dim != 3))
    return cudaErrorInvalidValue;
  if (a.dim == 2) {
    if (ffs) k_macro_source<FFS, 2><<<a.npts, MS_THREADS, 0, st>>>(a);
    else k_macro_source<F64S, 2><<<a.npts, MS_THREADS, 0, st>>>(a);
  } else {
    if (ffs) k_macro_source<FFS, 3><<<a.npts, MS_THREADS, 0, st>>>(a);
    else k_macro_source<F64S, 3><<<a.npts, MS_THREADS, 0, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_macro_gather(int npts, int R, int N, const int *elem, const double *E,
                                const double *fbar, double *Eg, double *fg, cudaStream_t st) {
  const int total = npts * (R * R + N);
  if (total <= 0) return cudaSuccess;
  k_macro_gather<<<(total + 255) / 256, 256, 0, st>>>(npts, R, N, elem, E, fbar, Eg, fg);
  return cudaGetLastError();
}

cudaError_t launch_macro_cg(const MacroSolveArgs &a, cudaStream_t st) {
  if (a.M < 2 || a.max_iter < 0) return cudaErrorInvalidValue;
  if (a.dim == 2) return cg_dispatch<2>(a, st);
  if (a.dim == 3) return cg_dispatch<3>(a, st);
  return cudaErrorInvalidValue;
}

}  // namespace mch
