// FP64-inner instantiations of the persistent level kernel (the plain FP64 mode): every
// shape of the FP64 table in k_level_shapes.h.
#include "k_level.cuh"
#include "k_level_shapes.h"

namespace mch {

bool level2d_supported(int n, int P, bool fp64) {
  // P need not be a power of two; the sub-block size m = n / P must be (segment sums)
  if (P < 1 || n % P) return false;
  const int m = n / P;
  if (m < 2 || (m & (m - 1))) return false;
  int rpt;  // rows per thread of the launch shape used for this n
  switch (n) {
    case 16: rpt = 1; break;
    case 32: rpt = 4; break;
    case 64: rpt = fp64 ? 4 : 8; break;
    case 128: rpt = fp64 ? 8 : 16; break;
    case 256: if (fp64) return false; rpt = 16; break;
    case 24: rpt = 2; break;
    case 48: rpt = 8; break;
    case 96: rpt = 8; break;
    default: return false;
  }
  return m % rpt == 0;
}

#define MCH_SHAPE64(N_, V_)                                                                 \
  case N_ * 16 + V_: {                                                                      \
    constexpr LevelShape s = *find_level_shape(N_, V_, true);                               \
    return launch_level_nc<double, N_, s.rg, s.rpt, s.cl, s.minb, s.nch>(a, st);            \
  }

template <>
cudaError_t launch_level2d<double>(const LevelArgs<double> &a, cudaStream_t st) {
  switch (a.n * 16 + a.variant) {
    MCH_SHAPE64(16, 0)
    MCH_SHAPE64(16, 1)
    MCH_SHAPE64(32, 0)
    MCH_SHAPE64(32, 1)
    MCH_SHAPE64(32, 2)
    MCH_SHAPE64(64, 0)
    MCH_SHAPE64(64, 1)
    MCH_SHAPE64(64, 2)
    MCH_SHAPE64(128, 0)
    MCH_SHAPE64(128, 1)
    MCH_SHAPE64(128, 2)
    MCH_SHAPE64(24, 0)
    MCH_SHAPE64(48, 0)
    MCH_SHAPE64(96, 0)
  }
  return cudaErrorInvalidValue;
}

}  // namespace mch
