// FP64-inner instantiations of the persistent level kernel (the plain FP64 mode).
#include "k_level.cuh"

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

template <>
cudaError_t launch_level2d<double>(const LevelArgs<double> &a, cudaStream_t st) {
  switch (a.n) {
    case 16: return launch_level_nc<double, 16, 16, 1, 1, 2>(a, st);
    case 32: return launch_level_nc<double, 32, 8, 4, 1, 2>(a, st);
    case 64: return launch_level_nc<double, 64, 8, 4, 2, 1>(a, st);
    case 128: return launch_level_nc<double, 128, 4, 8, 4, 1>(a, st);
    case 24: return launch_level_nc<double, 24, 12, 2, 1, 2>(a, st);
    case 48: return launch_level_nc<double, 48, 6, 8, 1, 1>(a, st);
    case 96: return launch_level_nc<double, 96, 4, 8, 3, 1>(a, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mch
