// FP32-inner instantiations of the persistent level kernel (mixed-precision mode): the
// default launch shape (index 0 of k_level_shapes.h) of every grid size. Per grid size n the
// shape is NEL = n lanes per row, RG row groups of RPT rows each, a cluster of CL CTAs when
// one CTA's slab of RG*RPT rows does not cover the n-1 node rows, MINB resident CTAs per SM
// requested from the register allocator, and NCH Chebyshev steps in the preconditioner
// (1 = Jacobi).
#include "k_level.cuh"
#include "k_level_shapes.h"

namespace mch {

template <>
cudaError_t launch_level2d<float>(const LevelArgs<float> &a, cudaStream_t st) {
  if (a.variant != 0) return launch_level2d_alt(a, st);
  switch (a.n) {
#define MCH_DEFAULT(N_)                                                                     \
  case N_: {                                                                                \
    constexpr LevelShape s = *find_level_shape(N_, 0);                                      \
    return launch_level_nc<float, N_, s.rg, s.rpt, s.cl, s.minb, s.nch>(a, st);             \
  }
    MCH_DEFAULT(16)
    MCH_DEFAULT(32)
    MCH_DEFAULT(64)
    MCH_DEFAULT(128)
    MCH_DEFAULT(256)
    MCH_DEFAULT(24)
    MCH_DEFAULT(48)
    MCH_DEFAULT(96)
#undef MCH_DEFAULT
  }
  return cudaErrorInvalidValue;
}

}  // namespace mch
