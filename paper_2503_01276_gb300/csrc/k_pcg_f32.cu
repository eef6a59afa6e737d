// FP32 instantiations of the shared-memory PCG sweep (mixed-precision mode). Per grid size
// n the launch shape is NEL = n lanes per row, RG row groups of RPT rows each, and a
// cluster of CL CTAs when one CTA's slab of RG*RPT rows does not cover the n-1 node rows.
#include "k_pcg.cuh"

namespace mch {

template <>
cudaError_t launch_pcg2d<float>(const PcgArgs<float> &a, cudaStream_t st, int *launches) {
  if (launches) ++*launches;
  switch (a.n) {
    case 16: return launch_pcg_nc<float, 16, 16, 1, 1>(a, st);
    case 32: return launch_pcg_nc<float, 32, 8, 4, 1>(a, st);
    case 64: return launch_pcg_nc<float, 64, 16, 4, 1>(a, st);
    case 128: return launch_pcg_nc<float, 128, 8, 8, 2>(a, st);
    case 256: return launch_pcg_nc<float, 256, 2, 16, 8>(a, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mch
