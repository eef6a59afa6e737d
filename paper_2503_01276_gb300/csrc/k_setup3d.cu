// Per-point constraint data for the 3D cell problems (the 3D counterpart of k_setup.cu).
//
// Sec. 2, Eqs. (phi_avar), (phi_grad): row (j, q) = continuum j on period q; targets
// delta_ij int_{R_q} psi_j (phi_i) and delta_ij int_{R_q} (y_m - c_mj) psi_j (phi_i^m), with
// c_mj the centroid of continuum j over the RVE. Everything is scaled by 8 / h^3: the target
// of row (j, q) is 8 * #elements for phi_j and 8 * sum over its elements of
// (centroid_m - c_mj) for phi_j^m.
//
// S = Ct M^-1 Ct^T with M = diag(A) (Jacobi), inverted in FP64 (Cholesky, then
// L^-T L^-1); rows of empty (continuum, period) pairs get a unit diagonal (zero multiplier).
//
// k_setup3d_nodes runs on (point, slab of z-planes): validates kappa and the labels, adds the
// slab's element counts and centroid sums per row, writes M^-1 (FP64 and FP32) and the FP32
// copy of kappa, and adds the slab's part of S. A thread walks one node line along x; its
// node's eight adjacent elements give eight rows, and runs of nodes with the same eight rows
// are summed before they are added to every ordered pair of those rows.
// k_setup3d_point (one CTA per point) forms the targets and S^-1; S is in shared memory, the
// inverse factor in the (then free) global accumulator of S.
#include "k3d.cuh"
#include "kernels.h"

namespace mch {

namespace {

constexpr int S3N_THREADS = 256;
constexpr int S3P_THREADS = 512;

__device__ __forceinline__ double fast_rcp3(double d) {
  double y = (double)(1.0f / (float)d);
  y = y * (2.0 - d * y);
  y = y * (2.0 - d * y);
  return y;
}

__global__ void __launch_bounds__(S3N_THREADS) k_setup3d_nodes(SetupArgs a, int slices) {
  const int pt = blockIdx.x, slice = blockIdx.y;
  const int n = a.n, P = a.P, N = a.N, nc = a.nc;
  const int m = n / P, nq = P * P * P;
  const int W = n + 1;
  const int tid = threadIdx.x;
  const size_t ne = (size_t)n * n * n;
  const double *kap = a.kappa + (size_t)pt * ne;
  const uint8_t *lab = a.labels + (size_t)pt * ne;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *S = reinterpret_cast<double *>(smem_raw);  // [nc][nc]
  double *bs = S + nc * nc;                          // [nc][4]
  __shared__ int flags;
  if (tid == 0) flags = 0;
  for (int i = tid; i < nc * nc; i += S3N_THREADS) S[i] = 0.0;
  for (int i = tid; i < nc * 4; i += S3N_THREADS) bs[i] = 0.0;
  __syncthreads();

  // node planes [z0, z1) of the lattice; element planes [z0, min(z1, n))
  const int per = (W + slices - 1) / slices;
  const int z0 = slice * per, z1 = min(W, z0 + per);
  const size_t e0 = (size_t)z0 * n * n, e1 = (size_t)min(z1, n) * n * n;
  float *k32 = a.kap32 ? a.kap32 + (size_t)pt * ne : nullptr;
  for (size_t e = e0 + tid; e < e1; e += S3N_THREADS) {
    const double k = kap[e];
    const int l = lab[e];
    if (k32) k32[e] = (float)k;
    if (!(k > 0.0) || !(k < 1e300)) atomicOr(&flags, 1);
    if (l >= N) {
      atomicOr(&flags, 2);
      continue;
    }
    const int ex = (int)(e % n), ey = (int)((e / n) % n), ez = (int)(e / ((size_t)n * n));
    const int b = l * nq + ((ez / m) * P + ey / m) * P + ex / m;
    atomicAdd(&bs[4 * b + 0], 1.0);
    atomicAdd(&bs[4 * b + 1], -0.5 * a.len + (ex + 0.5) * a.h);
    atomicAdd(&bs[4 * b + 2], -0.5 * a.len + (ey + 0.5) * a.h);
    atomicAdd(&bs[4 * b + 3], -0.5 * a.len + (ez + 0.5) * a.h);
  }
  __syncthreads();
  if (flags) {
    if (tid == 0) atomicOr(&a.status[pt], flags);
    return;
  }

  double *mv = a.minv + (size_t)pt * a.nv;
  float *mv32 = a.minv32 ? a.minv32 + (size_t)pt * a.nv : nullptr;
  const int nlines = W * (z1 - z0);
  auto eidx = [&](int ex, int ey, int ez) { return (size_t)ex + (size_t)n * (ey + (size_t)n * ez); };
  for (int t = tid; t < nlines; t += S3N_THREADS) {
    const int ky = t % W, kz = z0 + t / W;
    const size_t base = (size_t)W * (ky + (size_t)W * kz);
    const bool bnd = ky == 0 || kz == 0 || ky == n || kz == n;
    unsigned long long sig = ~0ull;
    double acc = 0.0;
    auto flush = [&]() {
      if (sig == ~0ull) return;
      int bb[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) bb[i] = (int)((sig >> (7 * i)) & 127ull);
      for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) atomicAdd(&S[bb[i] * nc + bb[j]], acc);
    };
    for (int kx = 0; kx < W; ++kx) {
      if (bnd || kx == 0 || kx == n) {
        mv[base + kx] = 0.0;
        if (mv32) mv32[base + kx] = 0.f;
        continue;
      }
      double ks = 0.0;
      unsigned long long key = 0ull;
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int ex = kx - 1 + (s & 1), ey = ky - 1 + ((s >> 1) & 1), ez = kz - 1 + (s >> 2);
        const size_t e = eidx(ex, ey, ez);
        ks += kap[e];
        // labels of the neighbouring slab are validated there: clamp them here
        const int b = min((int)lab[e], N - 1) * nq + ((ez / m) * P + ey / m) * P + ex / m;
        key |= (unsigned long long)b << (7 * s);
      }
      const double dinv = fast_rcp3(ks * a.h * (1.0 / 3.0));
      mv[base + kx] = dinv;
      if (mv32) mv32[base + kx] = (float)dinv;
      if (key != sig) {
        flush();
        sig = key;
        acc = 0.0;
      }
      acc += dinv;
    }
    flush();
  }
  __syncthreads();
  double *Sg = a.Sacc + (size_t)pt * nc * nc;
  for (int i = tid; i < nc * nc; i += S3N_THREADS)
    if (S[i] != 0.0) atomicAdd(&Sg[i], S[i]);
  double *bg = a.bacc + (size_t)pt * nc * 4;
  for (int i = tid; i < nc * 4; i += S3N_THREADS)
    if (bs[i] != 0.0) atomicAdd(&bg[i], bs[i]);
}

__global__ void __launch_bounds__(S3P_THREADS) k_setup3d_point(SetupArgs a) {
  const int pt = blockIdx.x;
  const int P = a.P, N = a.N, R = a.R, nc = a.nc;
  const int nq = P * P * P;
  const int tid = threadIdx.x;
  if (a.status[pt] & 3) return;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *S = reinterpret_cast<double *>(smem_raw);  // [nc][nc]
  double *bs = S + nc * nc;                          // [nc][4]
  double *cen = bs + 4 * nc;                         // [MCH_MAX_CONT][3]
  double *dorig = cen + 3 * MCH_MAX_CONT;            // [nc]
  __shared__ int flags;
  if (tid == 0) flags = 0;
  double *Sg = a.Sacc + (size_t)pt * nc * nc;
  for (int i = tid; i < nc * nc; i += S3P_THREADS) S[i] = Sg[i];
  for (int i = tid; i < 4 * nc; i += S3P_THREADS) bs[i] = a.bacc[(size_t)pt * nc * 4 + i];
  __syncthreads();

  // centroids c_mj over the integration region R_p (the central (P - 2 overs)^3 periods;
  // the whole RVE when the continuum is absent there, or when overs = 0)
  if (tid < N) {
    double c = 0, x = 0, y = 0, z = 0, ca = 0, xa = 0, ya = 0, za = 0;
    const int o = a.overs;
    for (int q = 0; q < nq; ++q) {
      const int b = tid * nq + q;
      const int qx = q % P, qy = (q / P) % P, qz = q / (P * P);
      ca += bs[4 * b];
      xa += bs[4 * b + 1];
      ya += bs[4 * b + 2];
      za += bs[4 * b + 3];
      if (qx >= o && qx < P - o && qy >= o && qy < P - o && qz >= o && qz < P - o) {
        c += bs[4 * b];
        x += bs[4 * b + 1];
        y += bs[4 * b + 2];
        z += bs[4 * b + 3];
      }
    }
    if (ca == 0.0) atomicOr(&flags, 8);
    if (c == 0.0) {
      c = ca;
      x = xa;
      y = ya;
      z = za;
    }
    cen[3 * tid] = c > 0 ? x / c : 0.0;
    cen[3 * tid + 1] = c > 0 ? y / c : 0.0;
    cen[3 * tid + 2] = c > 0 ? z / c : 0.0;
  }
  __syncthreads();

  double *G = a.G + (size_t)pt * nc * R;
  for (int t = tid; t < nc * R; t += S3P_THREADS) {
    const int b = t / R, r = t % R;
    const int j = b / nq;
    double v = 0.0;
    if (r < N) {
      if (r == j) v = 8.0 * bs[4 * b];
    } else {
      const int i = (r - N) / 3, mm = (r - N) % 3;
      if (i == j) v = 8.0 * (bs[4 * b + 1 + mm] - bs[4 * b] * cen[3 * j + mm]);
    }
    G[t] = v;
  }
  if (tid < nc) {
    if (bs[4 * tid] == 0.0) S[tid * nc + tid] = 1.0;
    dorig[tid] = S[tid * nc + tid];
  }
  __syncthreads();

  for (int k = 0; k < nc; ++k) {
    if (tid == 0) {
      double v = S[k * nc + k];
      if (!(v > 1e-13 * dorig[k])) {
        flags |= 4;
        v = dorig[k] > 0 ? dorig[k] : 1.0;
      }
      S[k * nc + k] = sqrt(v);
    }
    __syncthreads();
    for (int i = k + 1 + tid; i < nc; i += S3P_THREADS) S[i * nc + k] /= S[k * nc + k];
    __syncthreads();
    const int rem = nc - k - 1;
    for (int t = tid; t < rem * rem; t += S3P_THREADS) {
      const int i = k + 1 + t / rem, j = k + 1 + t % rem;
      if (j <= i) S[i * nc + j] -= S[i * nc + k] * S[j * nc + k];
    }
    __syncthreads();
  }

  // Z = L^-1 into the global scratch (column j by forward substitution)
  double *Z = Sg;
  for (int j = tid; j < nc; j += S3P_THREADS) {
    for (int i = 0; i < nc; ++i) {
      double v = (i == j) ? 1.0 : 0.0;
      if (i > j)
        for (int k = j; k < i; ++k) v -= S[i * nc + k] * Z[k * nc + j];
      Z[i * nc + j] = (i < j) ? 0.0 : v / S[i * nc + i];
    }
  }
  __syncthreads();
  double *Si64 = a.Sinv64 + (size_t)pt * nc * nc;
  float *Si32 = a.Sinv32 ? a.Sinv32 + (size_t)pt * nc * nc : nullptr;
  for (int t = tid; t < nc * nc; t += S3P_THREADS) {
    const int i = t / nc, j = t % nc;
    double v = 0.0;
    for (int k = max(i, j); k < nc; ++k) v += Z[k * nc + i] * Z[k * nc + j];
    Si64[t] = v;
    if (Si32) Si32[t] = (float)v;
  }
  if (tid == 0) {
    int nd = 0;
    for (int b = 0; b < nc; ++b) nd += (bs[4 * b] == 0.0);
    a.dropped[pt] = nd;
    a.status[pt] |= flags;
  }
}

}  // namespace

cudaError_t launch_setup3d(const SetupArgs &a, cudaStream_t st) {
  if (a.nc > MCH_MAX_NC3 || a.N > MCH_MAX_CONT) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(a.Sacc, 0, sizeof(double) * a.npts * a.nc * a.nc, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.bacc, 0, sizeof(double) * a.npts * a.nc * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.status, 0, sizeof(int) * a.npts, st);
  if (e != cudaSuccess) return e;
  int slices = (4 * device_sm_count() + a.npts - 1) / a.npts;
  slices = slices < 1 ? 1 : (slices > (a.n + 1) / 2 ? (a.n + 1) / 2 : slices);
  const size_t smem_n = sizeof(double) * ((size_t)a.nc * a.nc + 4 * a.nc);
  e = cudaFuncSetAttribute(k_setup3d_nodes, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem_n);
  if (e != cudaSuccess) return e;
  k_setup3d_nodes<<<dim3(a.npts, slices), S3N_THREADS, smem_n, st>>>(a, slices);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem_p =
      sizeof(double) * ((size_t)a.nc * a.nc + 5 * a.nc + 3 * MCH_MAX_CONT);
  e = cudaFuncSetAttribute(k_setup3d_point, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem_p);
  if (e != cudaSuccess) return e;
  k_setup3d_point<<<a.npts, S3P_THREADS, smem_p, st>>>(a);
  return cudaGetLastError();
}

}  // namespace mch
