// Alternative launch shapes of the FP32-inner level kernel for grids 128 and 256 (the shape
// table is k_level_shapes.h); a separate translation unit so that the shapes compile in
// parallel.
#include "k_level.cuh"
#include "k_level_shapes.h"

namespace mch {

#define MCH_SHAPE(N_, V_)                                                                   \
  case N_ * 16 + V_: {                                                                      \
    constexpr LevelShape s = *find_level_shape(N_, V_);                                     \
    return launch_level_nc<float, N_, s.rg, s.rpt, s.cl, s.minb, s.nch>(a, st);             \
  }

cudaError_t launch_level2d_alt_big(const LevelArgs<float> &a, cudaStream_t st) {
  switch (a.n * 16 + a.variant) {
    MCH_SHAPE(128, 1)
    MCH_SHAPE(128, 2)
    MCH_SHAPE(128, 3)
    MCH_SHAPE(128, 4)
    MCH_SHAPE(128, 5)
    MCH_SHAPE(128, 6)
    MCH_SHAPE(128, 7)
    MCH_SHAPE(128, 8)
    MCH_SHAPE(256, 1)
    MCH_SHAPE(256, 2)
    MCH_SHAPE(256, 3)
    MCH_SHAPE(256, 4)
    MCH_SHAPE(256, 5)
  }
  return cudaErrorInvalidValue;
}

}  // namespace mch
