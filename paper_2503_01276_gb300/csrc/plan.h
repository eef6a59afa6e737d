// Host-side level plan of the hierarchical macrogrid.
#pragma once
#include <string>
#include <vector>

namespace mch {

struct LevelPlan {
  int n_elem = 0;                    // elements per RVE side on this level
  std::vector<int> points;           // [npts][dim] macro indices, x fastest order
  std::vector<int> par_level;        // [npts][2^dim] 1-based level, 0 = unused slot
  std::vector<int> par_pos;          // [npts][2^dim]
  std::vector<double> par_w;         // [npts][2^dim]
  int npts() const { return n_elem > 0 ? (int)points.size() : 0; }
};

// Sec. 3.1, Eq. (defi_Sn): T_n = indices that are multiples of stride_n on every axis,
// S_1 = T_1, S_n = T_n \ T_{n-1}. Sec. 3.3: parents of a point of S_n are the vertices of the
// T_{n-1} cell containing it (only the grid-line vertex along axes where it lies on a
// T_{n-1} line), with multilinear weights that sum to one (interp = 0). With interp = 1 the
// single parent is the nearest point of S_1 with weight one (the choice of the paper's
// experiments, Sec. 3.3: I_p = Phi_t with x_t in S_1); ties go to the lower index. Returns
// false and sets err on an invalid stride set.
bool build_plan(int dim, int macro_n, const std::vector<int> &strides, int n_fine, int eta,
                std::vector<LevelPlan> &levels, std::string &err, int interp = 0);

}  // namespace mch
