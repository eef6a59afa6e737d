// Shared device helpers for the 3D cell-problem kernels.
//
// Grid conventions: an RVE of n^3 Q1 hexahedra; element (ex, ey, ez) has flat index
// ex + n*(ey + n*ez); node vectors live on the (n+1)^3 lattice (node (kx, ky, kz) at
// kx + W*(ky + W*kz), W = n+1) with zero boundary entries, each vector of a batch starting
// at a multiple of nv3 = round_up((n+1)^3, 32).
//
// Constraint rows (Sec. 2, Eqs. phi_avar, phi_grad): row b = j * P^3 + (qz * P + qy) * P + qx
// for continuum j and period (qx, qy, qz). As in 2D the library uses the row-scaled operator
// Ct = (8 / h^3) C: entry (row, node) = number of the row's elements adjacent to the node.
//
// Q1 stiffness (Sec. 2, Eq. weak_galerkin) of an element of side h and conductivity kappa:
// kappa * h * Khat with the unit-cube matrix Khat = Kx(x)My(x)Mz + Mx(x)Ky(x)Mz + Mx(x)My(x)Kz
// (1D stiffness [[1,-1],[-1,1]], 1D mass [[1/3,1/6],[1/6,1/3]]). Its entries depend only on
// how many coordinates two corners differ in: 0 -> 1/3, 1 -> 0, 2 -> -1/12, 3 -> -1/12. At a
// node the assembled operator is therefore a 21-point stencil: the 6 axis neighbours do not
// couple, each of the 12 face-diagonal neighbours couples through the 2 elements sharing
// that face diagonal, each of the 8 body-diagonal neighbours through 1 element.
#pragma once

#include "common.cuh"

#define MCH_MAX_NC3 128

namespace mch {

__host__ __device__ __forceinline__ int nv3_of(int n) {
  return round_up((n + 1) * (n + 1) * (n + 1), 32);
}

// A x at a node, up to the factor h. v[dz][dy][dx]: values at offsets -1..1 (index 0..2);
// k[sz][sy][sx]: conductivity of the adjacent element whose lowest corner is at offset
// (sx-1, sy-1, sz-1).
template <typename V>
__device__ __forceinline__ V q1_apply3d(const V (&v)[3][3][3], const V (&k)[2][2][2]) {
  const V ksum = ((k[0][0][0] + k[0][0][1]) + (k[0][1][0] + k[0][1][1])) +
                 ((k[1][0][0] + k[1][0][1]) + (k[1][1][0] + k[1][1][1]));
  V acc = V(0);
  // body diagonals: offset (ox, oy, oz), each +-1, one element: s = (o == 1 ? 1 : 0)
#pragma unroll
  for (int oz = 0; oz < 2; ++oz)
#pragma unroll
    for (int oy = 0; oy < 2; ++oy)
#pragma unroll
      for (int ox = 0; ox < 2; ++ox) acc += k[oz][oy][ox] * v[2 * oz][2 * oy][2 * ox];
  // face diagonals in the xy plane (oz = 0): elements s = (sx, sy, 0) and (sx, sy, 1)
#pragma unroll
  for (int oy = 0; oy < 2; ++oy)
#pragma unroll
    for (int ox = 0; ox < 2; ++ox)
      acc += (k[0][oy][ox] + k[1][oy][ox]) * v[1][2 * oy][2 * ox];
  // xz plane (oy = 0)
#pragma unroll
  for (int oz = 0; oz < 2; ++oz)
#pragma unroll
    for (int ox = 0; ox < 2; ++ox)
      acc += (k[oz][0][ox] + k[oz][1][ox]) * v[2 * oz][1][2 * ox];
  // yz plane (ox = 0)
#pragma unroll
  for (int oz = 0; oz < 2; ++oz)
#pragma unroll
    for (int oy = 0; oy < 2; ++oy)
      acc += (k[oz][oy][0] + k[oz][oy][1]) * v[2 * oz][2 * oy][1];
  return ksum * v[1][1][1] * V(1.0 / 3.0) - acc * V(1.0 / 12.0);
}

}  // namespace mch
