// Shared device helpers for the 2D cell-problem kernels.
//
// Grid conventions (identical on every level): an RVE of n x n Q1 elements; element
// (ex, ey) has flat index ex + n*ey; node vectors live on the padded (n+1) x (n+1)
// lattice (node (kx, ky) at kx + (n+1)*ky), boundary entries are kept at zero, and each
// vector of a batch starts at a multiple of `nv` = round_up((n+1)^2, 32) elements.
//
// Constraint rows (Sec. 2, Eqs. phi_avar and phi_grad): row b = j * P^2 + qy * P + qx for
// continuum j and sub-block R_q = period (qx, qy). The library works with the row-scaled
// operator Ct = (4 / h^2) C, whose entry for (row, node) is the number of elements of the
// row's (continuum, sub-block) pair adjacent to the node; targets are scaled the same way.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define MCH_MAX_CONT 4
#define MCH_MAX_NC 64

namespace mch {

__host__ __device__ __forceinline__ int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Streaming multiprocessors of the current device (grid sizing); 1 if the query fails.
inline int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1) {
    cudaGetLastError();
    return 1;
  }
  return sms;
}
__host__ __device__ __forceinline__ int nv_of(int n) { return round_up((n + 1) * (n + 1), 32); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over aligned groups of `seg` lanes (seg a power of two <= 32).
template <typename T>
__device__ __forceinline__ T seg_sum(T v, int seg) {
  for (int o = seg >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ void add_by_label(T (&acc)[MCH_MAX_CONT], int lab, T v) {
#pragma unroll
  for (int j = 0; j < MCH_MAX_CONT; ++j) acc[j] += (lab == j) ? v : T(0);
}

// acc[lab] += v for a label held in a register (predicated adds into static slots; labels
// >= NC add nothing)
template <int NC, typename V>
__device__ __forceinline__ void add_lab(V (&acc)[NC], int lab, V v) {
#pragma unroll
  for (int j = 0; j < NC; ++j) acc[j] += (lab == j) ? v : V(0);
}

template <typename T>
__device__ __forceinline__ T q1_apply(T a, T b, T c, T d, T xSW, T xS, T xSE, T xW, T x0, T xE,
                                      T xNW, T xN, T xNE) {
  const T t = T(4) * (a + b + c + d) * x0 - (b + d) * xE - (a + c) * xW - (c + d) * xN -
              (a + b) * xS - T(2) * (d * xNE + c * xNW + b * xSE + a * xSW);
  return t * T(1.0 / 6.0);
}

template <typename T>
__device__ __forceinline__ T q1_diag(T a, T b, T c, T d) {
  return (a + b + c + d) * T(2.0 / 3.0);
}

}  // namespace mch
