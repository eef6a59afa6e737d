// Host-side level plan; see plan.h.
#include "plan.h"

#include <map>

namespace mch {

bool build_plan(int dim, int macro_n, const std::vector<int> &strides, int n_fine, int eta,
                std::vector<LevelPlan> &levels, std::string &err, int interp) {
  if (interp != 0 && interp != 1) { err = "interp must be 0 or 1"; return false; }
  const int L = (int)strides.size();
  if (L < 1 || strides.back() != 1) { err = "the last level stride must be 1"; return false; }
  for (int i = 0; i + 1 < L; ++i)
    if (strides[i] <= strides[i + 1] || strides[i] % strides[i + 1]) {
      err = "level strides must strictly decrease and divide each other";
      return false;
    }
  if ((macro_n - 1) % strides[0]) { err = "stride of level 1 must divide macro_n - 1"; return false; }
  if (dim < 1 || dim > 3) { err = "dim must be 1..3"; return false; }
  long long total = 1;
  for (int a = 0; a < dim; ++a) total *= macro_n;
  if (total > (1LL << 26)) { err = "macrogrid too large"; return false; }

  levels.assign(L, LevelPlan());
  std::map<long long, std::pair<int, int>> where;  // flat index -> (level, pos)
  std::vector<int> idx(dim);
  const int slots = 1 << dim;
  int scale = 1;
  for (int n = 0; n < L; ++n) {
    LevelPlan &lp = levels[n];
    lp.n_elem = n_fine / scale;
    scale *= eta;
    const int s = strides[n];
    const int sp = n > 0 ? strides[n - 1] : 0;
    for (long long f = 0; f < total; ++f) {
      long long r = f;
      bool inT = true, inPrev = (n > 0);
      for (int a = 0; a < dim; ++a) {
        idx[a] = (int)(r % macro_n);
        r /= macro_n;
        if (idx[a] % s) inT = false;
        if (n > 0 && idx[a] % sp) inPrev = false;
      }
      if (!inT || inPrev) continue;
      const int pos = (int)(lp.points.size() / dim);
      for (int a = 0; a < dim; ++a) lp.points.push_back(idx[a]);
      where[f] = {n + 1, pos};
      if (n == 0) {
        for (int t = 0; t < slots; ++t) {
          lp.par_level.push_back(0);
          lp.par_pos.push_back(0);
          lp.par_w.push_back(0.0);
        }
        continue;
      }
      if (interp == 1) {
        // nearest point of S_1 = T_1 (per axis: round to the stride, ties down)
        const int s1 = strides[0];
        long long pf = 0, mul = 1;
        for (int a = 0; a < dim; ++a) {
          const int lo = (idx[a] / s1) * s1, rem = idx[a] - lo;
          pf += (long long)(2 * rem > s1 ? lo + s1 : lo) * mul;
          mul *= macro_n;
        }
        auto it = where.find(pf);
        if (it == where.end() || it->second.first != 1) { err = "internal: S_1 parent"; return false; }
        for (int t = 0; t < slots; ++t) {
          lp.par_level.push_back(t == 0 ? 1 : 0);
          lp.par_pos.push_back(t == 0 ? it->second.second : 0);
          lp.par_w.push_back(t == 0 ? 1.0 : 0.0);
        }
        continue;
      }
      // parents: tensor product over axes of {lo} (on a T_{n-1} line) or {lo, lo+sp}
      int used = 0;
      for (int t = 0; t < slots; ++t) {
        long long pf = 0, mul = 1;
        double w = 1.0;
        bool valid = true;
        for (int a = 0; a < dim; ++a) {
          const int i = idx[a];
          const int lo = (i / sp) * sp;
          const int bit = (t >> a) & 1;
          int q;
          if (i % sp == 0) {
            if (bit) { valid = false; break; }
            q = i;
          } else {
            const double fr = double(i - lo) / double(sp);
            q = lo + bit * sp;
            w *= bit ? fr : 1.0 - fr;
          }
          pf += (long long)q * mul;
          mul *= macro_n;
        }
        if (!valid) continue;
        auto it = where.find(pf);
        if (it == where.end()) { err = "internal: parent not planned"; return false; }
        lp.par_level.push_back(it->second.first);
        lp.par_pos.push_back(it->second.second);
        lp.par_w.push_back(w);
        ++used;
      }
      for (int t = used; t < slots; ++t) {
        lp.par_level.push_back(0);
        lp.par_pos.push_back(0);
        lp.par_w.push_back(0.0);
      }
    }
  }
  return true;
}

}  // namespace mch
