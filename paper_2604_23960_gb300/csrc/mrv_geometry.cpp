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
  // blocks: rows = the larger frame, columns = the smaller (<= 32 spheres)
  bool ok = true;
  for (size_t g = 0; g < P.self_groups.size() / 4 && ok; ++g) {
    const int u = P.self_groups[4 * g], v = P.self_groups[4 * g + 1];
    const int nu = P.link_start[u + 1] - P.link_start[u], nv = P.link_start[v + 1] - P.link_start[v];
    const bool rows_u = nu >= nv;
    const int rf = rows_u ? u : v, cf = rows_u ? v : u;
    const int nr = rows_u ? nu : nv, nc = rows_u ? nv : nu;
    if (nc > 32) {
      ok = false;
      break;
    }
    const int first_mask = (int)P.self_masks.size();
    P.self_masks.resize(P.self_masks.size() + nr, 0u);
    const int p0 = P.self_groups[4 * g + 2], pc = P.self_groups[4 * g + 3];
    for (int q = p0; q < p0 + pc; ++q) {
      int x = P.self[q].first, y = P.self[q].second;   // x in frame u, y in frame v
      if (!rows_u) std::swap(x, y);                      // x: row sphere, y: column sphere
      if (u == v && x > y) std::swap(x, y);
      P.self_masks[first_mask + (x - P.link_start[rf])] |= 1u << (y - P.link_start[cf]);
    }
    P.self_blocks.insert(P.self_blocks.end(),
                         {P.link_start[rf], P.link_start[cf], nr | (nc << 16) | (cf << 24) | (rf << 28), first_mask});
  }
  if (!ok) {
    P.self_blocks.clear();
    P.self_masks.clear();
  }
  return P;
}

// distance from a point to a box (0 inside), double
static double point_box(const double *x, const double *lo, const double *hi) {
  double d2 = 0;
  for (int a = 0; a < 3; ++a) {
    const double e = x[a] < lo[a] ? lo[a] - x[a] : (x[a] > hi[a] ? x[a] - hi[a] : 0.0);
    d2 += e * e;
  }
  return std::sqrt(d2);
}

// distance between two boxes (0 when they overlap), double
static double box_box(const double *alo, const double *ahi, const double *blo, const double *bhi) {
  double d2 = 0;
  for (int a = 0; a < 3; ++a) {
    const double e = blo[a] > ahi[a] ? blo[a] - ahi[a] : (alo[a] > bhi[a] ? alo[a] - bhi[a] : 0.0);
    d2 += e * e;
  }
  return std::sqrt(d2);
}

ObstacleGrid build_obstacle_grid(int n_spheres, const float *xyzr, int n_boxes, const float *lohi, int n_cyl,
                                 const float *cyl, double R, int64_t max_items) {
  ObstacleGrid G;
  if (!(R > 0) || n_spheres + n_boxes + n_cyl == 0 || n_spheres > 65535 || n_boxes > 65535 || n_cyl > 65535)
    return G;
  // a cylinder's bounding box: axis ends +- radius on every axis
  std::vector<double> cbox(6 * (size_t)n_cyl);
  for (int i = 0; i < n_cyl; ++i)
    for (int a = 0; a < 3; ++a) {
      const double p = cyl[7 * i + a], q = cyl[7 * i + 3 + a], rr = cyl[7 * i + 6];
      cbox[6 * i + a] = std::min(p, q) - rr;
      cbox[6 * i + 3 + a] = std::max(p, q) + rr;
    }
  // bounding box of the obstacles
  double blo[3] = {INFINITY, INFINITY, INFINITY}, bhi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int i = 0; i < n_spheres; ++i)
    for (int a = 0; a < 3; ++a) {
      blo[a] = std::min(blo[a], (double)xyzr[4 * i + a] - xyzr[4 * i + 3]);
      bhi[a] = std::max(bhi[a], (double)xyzr[4 * i + a] + xyzr[4 * i + 3]);
    }
  for (int i = 0; i < n_boxes; ++i)
    for (int a = 0; a < 3; ++a) {
      blo[a] = std::min(blo[a], (double)lohi[6 * i + a]);
      bhi[a] = std::max(bhi[a], (double)lohi[6 * i + 3 + a]);
    }
  for (int i = 0; i < n_cyl; ++i)
    for (int a = 0; a < 3; ++a) {
      blo[a] = std::min(blo[a], cbox[6 * i + a]);
      bhi[a] = std::max(bhi[a], cbox[6 * i + 3 + a]);
    }
  double scale = 1.0;
  for (int a = 0; a < 3; ++a) scale = std::max(scale, std::max(std::fabs(blo[a]), std::fabs(bhi[a])));
  // cell size first guess: R / 2, at most 64 cells per axis
  double ext[3], h = R / 2;
  for (int a = 0; a < 3; ++a) {
    ext[a] = bhi[a] - blo[a] + 2 * (R * (1 + 1e-3) + 1e-6 * scale) + 1e-6 * scale;
    h = std::max(h, ext[a] / 64);
  }
  const double slack = 1e-3 * h + 1e-6 * scale;
  // grow the margin by the slack of the final cell size
  for (int a = 0; a < 3; ++a) {
    const double m = R + 2 * slack;
    G.lo[a] = blo[a] - m;
    ext[a] = bhi[a] - blo[a] + 2 * m;
    G.dims[a] = std::max(1, std::min(64, (int)std::ceil(ext[a] / h)));
    h = std::max(h, ext[a] / G.dims[a]);
  }
  G.h = h;
  const int nx = G.dims[0], ny = G.dims[1], nz = G.dims[2];
  const int64_t ncells = (int64_t)nx * ny * nz;
  auto cell_range = [&](const double *lo, const double *hi, int *i0, int *i1) {
    for (int a = 0; a < 3; ++a) {
      i0[a] = std::max(0, (int)std::floor((lo[a] - G.lo[a]) / h) - 1);
      i1[a] = std::min(G.dims[a] - 1, (int)std::floor((hi[a] - G.lo[a]) / h) + 1);
    }
  };
  // visit(c, kind, id) for every (cell, obstacle) within reach
  auto each = [&](auto &&visit) {
    for (int i = 0; i < n_spheres; ++i) {
      const double c[3] = {xyzr[4 * i], xyzr[4 * i + 1], xyzr[4 * i + 2]};
      const double reach = R + xyzr[4 * i + 3] + slack;
      const double lo[3] = {c[0] - reach, c[1] - reach, c[2] - reach}, hi[3] = {c[0] + reach, c[1] + reach, c[2] + reach};
      int i0[3], i1[3];
      cell_range(lo, hi, i0, i1);
      for (int z = i0[2]; z <= i1[2]; ++z)
        for (int y = i0[1]; y <= i1[1]; ++y)
          for (int x = i0[0]; x <= i1[0]; ++x) {
            const double clo[3] = {G.lo[0] + x * h, G.lo[1] + y * h, G.lo[2] + z * h};
            const double chi[3] = {clo[0] + h, clo[1] + h, clo[2] + h};
            if (point_box(c, clo, chi) < reach) visit(((int64_t)z * ny + y) * nx + x, 0, i);
          }
    }
    for (int i = 0; i < n_boxes; ++i) {
      const double reach = R + slack;
      const double olo[3] = {lohi[6 * i], lohi[6 * i + 1], lohi[6 * i + 2]};
      const double ohi[3] = {lohi[6 * i + 3], lohi[6 * i + 4], lohi[6 * i + 5]};
      const double lo[3] = {olo[0] - reach, olo[1] - reach, olo[2] - reach};
      const double hi[3] = {ohi[0] + reach, ohi[1] + reach, ohi[2] + reach};
      int i0[3], i1[3];
      cell_range(lo, hi, i0, i1);
      for (int z = i0[2]; z <= i1[2]; ++z)
        for (int y = i0[1]; y <= i1[1]; ++y)
          for (int x = i0[0]; x <= i1[0]; ++x) {
            const double clo[3] = {G.lo[0] + x * h, G.lo[1] + y * h, G.lo[2] + z * h};
            const double chi[3] = {clo[0] + h, clo[1] + h, clo[2] + h};
            if (box_box(clo, chi, olo, ohi) < reach) visit(((int64_t)z * ny + y) * nx + x, 1, i);
          }
    }
    for (int i = 0; i < n_cyl; ++i) {
      const double reach = R + slack;
      const double *olo = &cbox[6 * i], *ohi = &cbox[6 * i + 3];
      const double lo[3] = {olo[0] - reach, olo[1] - reach, olo[2] - reach};
      const double hi[3] = {ohi[0] + reach, ohi[1] + reach, ohi[2] + reach};
      int i0[3], i1[3];
      cell_range(lo, hi, i0, i1);
      for (int z = i0[2]; z <= i1[2]; ++z)
        for (int y = i0[1]; y <= i1[1]; ++y)
          for (int x = i0[0]; x <= i1[0]; ++x) {
            const double clo[3] = {G.lo[0] + x * h, G.lo[1] + y * h, G.lo[2] + z * h};
            const double chi[3] = {clo[0] + h, clo[1] + h, clo[2] + h};
            if (box_box(clo, chi, olo, ohi) < reach) visit(((int64_t)z * ny + y) * nx + x, 2, i);
          }
    }
  };
  std::vector<int64_t> cnt[3] = {std::vector<int64_t>(ncells, 0), std::vector<int64_t>(ncells, 0),
                                 std::vector<int64_t>(ncells, 0)};
  int64_t total = 0;
  each([&](int64_t c, int kind, int) {
    cnt[kind][c]++;
    ++total;
  });
  if (total > max_items) return ObstacleGrid{};
  G.off.assign(ncells + 1, 0);
  G.ns.assign(ncells, 0);
  G.nb.assign(ncells, 0);
  for (int64_t c = 0; c < ncells; ++c) {
    if (cnt[0][c] > 65535 || cnt[1][c] > 65535) return ObstacleGrid{};
    G.off[c + 1] = G.off[c] + (int32_t)(cnt[0][c] + cnt[1][c] + cnt[2][c]);
    G.ns[c] = (uint16_t)cnt[0][c];
    G.nb[c] = (uint16_t)cnt[1][c];
  }
  G.items.assign((size_t)total, 0);
  std::vector<int32_t> fill[3] = {std::vector<int32_t>(ncells), std::vector<int32_t>(ncells),
                                  std::vector<int32_t>(ncells)};
  for (int64_t c = 0; c < ncells; ++c) {
    fill[0][c] = G.off[c];
    fill[1][c] = G.off[c] + G.ns[c];
    fill[2][c] = G.off[c] + G.ns[c] + G.nb[c];
  }
  each([&](int64_t c, int kind, int id) { G.items[fill[kind][c]++] = (uint16_t)id; });
  G.R = R;
  return G;
}

}  // namespace mrv
