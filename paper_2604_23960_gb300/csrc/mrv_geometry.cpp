// Host-side geometry preprocessing of robot models.
#include "mrv_geometry.h"

#include <algorithm>
#include <cmath>
#include <numeric>

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

PreparedModel prepare_model(int n_links, int m, const int32_t *link, const float *xyzr, int n_self,
                            const int32_t *pairs) {
  PreparedModel P;
  P.n_links = n_links;
  P.perm.resize(m);
  std::iota(P.perm.begin(), P.perm.end(), 0);
  std::stable_sort(P.perm.begin(), P.perm.end(), [&](int a, int b) { return link[a] < link[b]; });
  std::vector<int32_t> inv(m);
  P.spheres.resize(4 * (size_t)m);
  P.links.resize(m);
  for (int i = 0; i < m; ++i) {
    const int o = P.perm[i];
    inv[o] = i;
    for (int k = 0; k < 4; ++k) P.spheres[4 * i + k] = xyzr[4 * o + k];
    P.links[i] = link[o];
  }
  P.link_start.assign(n_links + 1, 0);
  for (int i = 0; i < m; ++i) P.link_start[P.links[i] + 1]++;
  for (int l = 0; l < n_links; ++l) P.link_start[l + 1] += P.link_start[l];
  P.link_bs.assign(4 * (size_t)n_links, 0.f);
  for (int l = 0; l < n_links; ++l) {
    const int a0 = P.link_start[l], a1 = P.link_start[l + 1];
    if (a0 == a1) {
      P.link_bs[4 * l + 3] = -1.f;
      continue;
    }
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = a0; i < a1; ++i)
      for (int k = 0; k < 3; ++k) {
        lo[k] = std::min(lo[k], (double)P.spheres[4 * i + k]);
        hi[k] = std::max(hi[k], (double)P.spheres[4 * i + k]);
      }
    double c[3], R = 0.0;
    for (int k = 0; k < 3; ++k) c[k] = 0.5 * (lo[k] + hi[k]);
    for (int i = a0; i < a1; ++i) {
      double d2 = 0.0;
      for (int k = 0; k < 3; ++k) d2 += ((double)P.spheres[4 * i + k] - c[k]) * ((double)P.spheres[4 * i + k] - c[k]);
      R = std::max(R, std::sqrt(d2) + (double)P.spheres[4 * i + 3]);
    }
    for (int k = 0; k < 3; ++k) P.link_bs[4 * l + k] = (float)c[k];
    // the float center moved by at most half an ulp per axis: absorbed below
    P.link_bs[4 * l + 3] = (float)(R * (1.0 + 1e-6) + 1e-4);
  }
  P.self.resize(n_self);
  for (int p = 0; p < n_self; ++p) P.self[p] = std::minmax(inv[pairs[2 * p]], inv[pairs[2 * p + 1]]);
  std::sort(P.self.begin(), P.self.end(), [&](const std::pair<int32_t, int32_t> &a, const std::pair<int32_t, int32_t> &b) {
    const int la = P.links[a.first], lb = P.links[b.first], ma = P.links[a.second], mb = P.links[b.second];
    if (la != lb) return la < lb;
    if (ma != mb) return ma < mb;
    return a < b;
  });
  for (size_t p = 0; p < P.self.size();) {
    size_t e = p + 1;
    const int u = P.links[P.self[p].first], v = P.links[P.self[p].second];
    while (e < P.self.size() && P.links[P.self[e].first] == u && P.links[P.self[e].second] == v) ++e;
    P.self_groups.insert(P.self_groups.end(), {u, v, (int32_t)p, (int32_t)(e - p)});
    p = e;
  }
  return P;
}

}  // namespace mrv
