// Launch shapes of the FP32-inner 2D level kernel, searched by the autotuner
// (mch_autotune_level). Shape v of grid n: RG row groups of RPT rows (NEL = n lanes per row),
// clusters of CL CTAs, MINB resident CTAs per SM requested from the register allocator, NCH
// Chebyshev steps in the preconditioner (1 = the Jacobi-weighted projection). Index 0 of each
// n is the default shape (k_level_f32.cu); the others are instantiated in
// k_level_f32_alt.cu and k_level_f32_alt2.cu. A shape is valid when its rows per thread
// divide the sub-block size m = n / P. (1024-thread shapes spill at 64 registers and are not
// offered.) Fewer, longer strips per thread amortise the per-iteration reductions, the
// per-warp multiplier evaluation and the barriers over more nodes; more CTAs per SM hide
// latency; more Chebyshev steps trade reductions and barriers for stencil applications.
#pragma once

namespace mch {

struct LevelShape {
  int n, v, rg, rpt, cl, minb, nch;
};

constexpr LevelShape kLevelShapes[] = {
    {16, 0, 16, 1, 1, 4, 1},  {16, 1, 8, 2, 1, 6, 1},   {16, 2, 4, 4, 1, 8, 1},
    {16, 3, 16, 1, 1, 4, 2},
    {32, 0, 8, 4, 1, 3, 2},   {32, 1, 4, 8, 1, 5, 1},   {32, 2, 16, 2, 1, 2, 1},
    {32, 3, 4, 4, 2, 6, 1},   {32, 4, 8, 4, 1, 3, 1},   {32, 5, 4, 8, 1, 5, 2},
    {32, 6, 8, 4, 1, 3, 4},
    {64, 0, 8, 8, 1, 1, 4},   {64, 1, 4, 16, 1, 2, 1},  {64, 2, 4, 8, 2, 2, 1},
    {64, 3, 8, 4, 2, 1, 1},   {64, 4, 2, 8, 4, 4, 1},   {64, 5, 4, 4, 4, 3, 1},
    {64, 6, 8, 8, 1, 1, 1},   {64, 7, 4, 16, 1, 2, 4},  {64, 8, 8, 8, 1, 1, 2},
    {64, 9, 8, 8, 1, 1, 6},
    {128, 0, 4, 16, 2, 1, 4}, {128, 1, 4, 8, 4, 1, 1},  {128, 2, 2, 8, 8, 3, 1},
    {128, 3, 4, 4, 8, 2, 1},  {128, 4, 4, 16, 2, 1, 1}, {128, 5, 4, 16, 2, 1, 6},
    {128, 6, 4, 8, 4, 1, 4},  {128, 7, 4, 16, 2, 1, 8},  {128, 8, 4, 16, 2, 1, 12},
    {256, 0, 2, 16, 8, 1, 4}, {256, 1, 2, 16, 8, 1, 1}, {256, 2, 2, 16, 8, 1, 6},
    {256, 3, 2, 16, 8, 1, 3}, {256, 4, 2, 16, 8, 1, 8},  {256, 5, 2, 16, 8, 1, 12},
    // grids with an odd number of sub-blocks per side (P = 3: m = 8, 16, 32)
    {24, 0, 12, 2, 1, 3, 2},  {48, 0, 6, 8, 1, 2, 2},   {96, 0, 4, 8, 3, 1, 4},
};

// Shapes of the FP64-inner kernel (the plain FP64 mode): index 0 is the default of
// k_level_f64.cu; the others (k_level_f64.cu) add Chebyshev steps to the same tiles.
constexpr LevelShape kLevelShapes64[] = {
    {16, 0, 16, 1, 1, 2, 1},  {16, 1, 16, 1, 1, 2, 2},
    {32, 0, 8, 4, 1, 2, 1},   {32, 1, 8, 4, 1, 2, 2},  {32, 2, 8, 4, 1, 2, 4},
    {64, 0, 8, 4, 2, 1, 1},   {64, 1, 8, 4, 2, 1, 4},  {64, 2, 8, 4, 2, 1, 6},
    {128, 0, 4, 8, 4, 1, 1},  {128, 1, 4, 8, 4, 1, 4}, {128, 2, 4, 8, 4, 1, 8},
    {24, 0, 12, 2, 1, 2, 1},  {48, 0, 6, 8, 1, 1, 1},  {96, 0, 4, 8, 3, 1, 1},
};

constexpr const LevelShape *find_level_shape(int n, int v, bool fp64 = false) {
  if (fp64) {
    for (const LevelShape &s : kLevelShapes64)
      if (s.n == n && s.v == v) return &s;
    return nullptr;
  }
  for (const LevelShape &s : kLevelShapes)
    if (s.n == n && s.v == v) return &s;
  return nullptr;
}

}  // namespace mch
