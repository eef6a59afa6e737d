// Alternative launch shapes of the FP32-inner level kernel, searched by the autotuner
// (mch_autotune_level). Shape v of grid n: RG row groups of RPT rows (NEL = n lanes per row),
// clusters of CL CTAs, MINB resident CTAs per SM requested from the register allocator.
// (1024-thread shapes spill at 64 registers and are not offered.)
// Fewer, longer strips per thread amortise the per-iteration reductions, the per-warp
// multiplier evaluation and the barriers over more nodes; more CTAs per SM hide latency.
// A shape is valid when its rows per thread divide the sub-block size m = n / P.
#include "k_level.cuh"

namespace mch {

namespace {

struct Shape {
  int n, v, rg, rpt, cl, minb;
};

// index 0 of each n is the default shape of k_level_f32.cu
constexpr Shape kShapes[] = {
    {16, 0, 16, 1, 1, 4}, {16, 1, 8, 2, 1, 6}, {16, 2, 4, 4, 1, 8},
    {32, 0, 8, 4, 1, 3},  {32, 1, 4, 8, 1, 5}, {32, 2, 16, 2, 1, 2}, {32, 3, 4, 4, 2, 6},
    {64, 0, 8, 8, 1, 1},  {64, 1, 4, 16, 1, 2}, {64, 2, 4, 8, 2, 2}, {64, 3, 8, 4, 2, 1},
    {64, 4, 2, 8, 4, 4},  {64, 5, 4, 4, 4, 3},
    {128, 0, 4, 16, 2, 1}, {128, 1, 4, 8, 4, 1}, {128, 2, 2, 8, 8, 3}, {128, 3, 4, 4, 8, 2},
    {256, 0, 2, 16, 8, 1},
};

const Shape *find(int n, int v) {
  for (const Shape &s : kShapes)
    if (s.n == n && s.v == v) return &s;
  return nullptr;
}

}  // namespace

int level2d_variant_count(int n, bool fp64) {
  if (fp64) return 1;
  int c = 0;
  for (const Shape &s : kShapes) c += s.n == n;
  return c;
}

bool level2d_variant_ok(int n, int P, bool fp64, int v) {
  if (v == 0) return level2d_supported(n, P, fp64);
  if (fp64 || !level2d_supported(n, P, fp64)) return false;
  const Shape *s = find(n, v);
  return s && (n / P) % s->rpt == 0;
}

cudaError_t launch_level2d_alt(const LevelArgs<float> &a, cudaStream_t st) {
  switch (a.n * 16 + a.variant) {
    case 16 * 16 + 1: return launch_level_nc<float, 16, 8, 2, 1, 6>(a, st);
    case 16 * 16 + 2: return launch_level_nc<float, 16, 4, 4, 1, 8>(a, st);
    case 32 * 16 + 1: return launch_level_nc<float, 32, 4, 8, 1, 5>(a, st);
    case 32 * 16 + 2: return launch_level_nc<float, 32, 16, 2, 1, 2>(a, st);
    case 64 * 16 + 1: return launch_level_nc<float, 64, 4, 16, 1, 2>(a, st);
    case 64 * 16 + 2: return launch_level_nc<float, 64, 4, 8, 2, 2>(a, st);
    case 64 * 16 + 3: return launch_level_nc<float, 64, 8, 4, 2, 1>(a, st);
    case 32 * 16 + 3: return launch_level_nc<float, 32, 4, 4, 2, 6>(a, st);
    case 64 * 16 + 4: return launch_level_nc<float, 64, 2, 8, 4, 4>(a, st);
    case 64 * 16 + 5: return launch_level_nc<float, 64, 4, 4, 4, 3>(a, st);
    case 128 * 16 + 1: return launch_level_nc<float, 128, 4, 8, 4, 1>(a, st);
    case 128 * 16 + 2: return launch_level_nc<float, 128, 2, 8, 8, 3>(a, st);
    case 128 * 16 + 3: return launch_level_nc<float, 128, 4, 4, 8, 2>(a, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mch
