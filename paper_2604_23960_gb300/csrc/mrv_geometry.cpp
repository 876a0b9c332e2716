// Host-side geometry preprocessing of robot models.
#include "mrv_geometry.h"

#include <algorithm>

namespace mrv {

std::vector<int32_t> self_pair_rectangles(int m, const std::vector<std::pair<int32_t, int32_t>> &pairs,
                                          int max_rects) {
  std::vector<std::vector<int32_t>> partners(m);
  for (auto &p : pairs) partners[p.first].push_back(p.second);
  for (auto &v : partners) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
  }
  std::vector<int32_t> out;
  for (int a0 = 0; a0 < m;) {
    int a1 = a0 + 1;
    while (a1 < m && partners[a1] == partners[a0]) ++a1;
    const auto &v = partners[a0];
    for (size_t k = 0; k < v.size();) {
      size_t e = k + 1;
      while (e < v.size() && v[e] == v[e - 1] + 1) ++e;
      out.insert(out.end(), {a0, a1, v[k], v[e - 1] + 1});
      if ((int)(out.size() / 4) > max_rects) return {};
      k = e;
    }
    a0 = a1;
  }
  return out;
}

}  // namespace mrv
