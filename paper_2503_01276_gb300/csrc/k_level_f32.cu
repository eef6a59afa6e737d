// FP32-inner instantiations of the persistent level kernel (mixed-precision mode). Per grid
// size n the launch shape is NEL = n lanes per row, RG row groups of RPT rows each, a
// cluster of CL CTAs when one CTA's slab of RG*RPT rows does not cover the n-1 node rows,
// and MINB resident CTAs per SM requested from the register allocator.
#include "k_level.cuh"

namespace mch {

template <>
cudaError_t launch_level2d<float>(const LevelArgs<float> &a, cudaStream_t st) {
  if (a.variant != 0) return launch_level2d_alt(a, st);
  switch (a.n) {
    case 16: return launch_level_nc<float, 16, 16, 1, 1, 4>(a, st);
    case 32: return launch_level_nc<float, 32, 8, 4, 1, 3>(a, st);
    case 64: return launch_level_nc<float, 64, 8, 8, 1, 1>(a, st);
    case 128: return launch_level_nc<float, 128, 4, 16, 2, 1>(a, st);
    case 256: return launch_level_nc<float, 256, 2, 16, 8, 1>(a, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mch
