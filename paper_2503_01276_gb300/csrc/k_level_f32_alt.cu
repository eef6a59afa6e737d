// Alternative launch shapes of the FP32-inner level kernel for grids 16, 32 and 64 (the
// shape table is k_level_shapes.h), the variant queries, and the dispatcher of every
// alternative shape.
#include "k_level.cuh"
#include "k_level_shapes.h"

namespace mch {

cudaError_t launch_level2d_alt_big(const LevelArgs<float> &a, cudaStream_t st);

int level2d_variant_count(int n, bool fp64) {
  int c = 0;
  if (fp64) {
    for (const LevelShape &s : kLevelShapes64) c += s.n == n;
  } else {
    for (const LevelShape &s : kLevelShapes) c += s.n == n;
  }
  return c > 0 ? c : 1;
}

bool level2d_variant_ok(int n, int P, bool fp64, int v) {
  if (v == 0) return level2d_supported(n, P, fp64);
  if (!level2d_supported(n, P, fp64)) return false;
  const LevelShape *s = find_level_shape(n, v, fp64);
  return s && (n / P) % s->rpt == 0;
}

int level2d_cheb_steps(int n, bool fp64, int v) {
  const LevelShape *s = find_level_shape(n, v, fp64);
  return s ? s->nch : 1;
}

#define MCH_SHAPE(N_, V_)                                                                   \
  case N_ * 16 + V_: {                                                                      \
    constexpr LevelShape s = *find_level_shape(N_, V_);                                     \
    return launch_level_nc<float, N_, s.rg, s.rpt, s.cl, s.minb, s.nch>(a, st);             \
  }

cudaError_t launch_level2d_alt(const LevelArgs<float> &a, cudaStream_t st) {
  switch (a.n * 16 + a.variant) {
    MCH_SHAPE(16, 1)
    MCH_SHAPE(16, 2)
    MCH_SHAPE(16, 3)
    MCH_SHAPE(32, 1)
    MCH_SHAPE(32, 2)
    MCH_SHAPE(32, 3)
    MCH_SHAPE(32, 4)
    MCH_SHAPE(32, 5)
    MCH_SHAPE(32, 6)
    MCH_SHAPE(64, 1)
    MCH_SHAPE(64, 2)
    MCH_SHAPE(64, 3)
    MCH_SHAPE(64, 4)
    MCH_SHAPE(64, 5)
    MCH_SHAPE(64, 6)
    MCH_SHAPE(64, 7)
    MCH_SHAPE(64, 8)
    MCH_SHAPE(64, 9)
  }
  return launch_level2d_alt_big(a, st);
}

}  // namespace mch
