// Host-side geometry preprocessing of robot models (no CUDA dependency).
#pragma once
#include <stdint.h>

#include <utility>
#include <vector>

namespace mrv {

// Exact cover of a self-pair set by rectangles (rows a0..a1-1 x columns
// c0..c1-1, every a < c), returned as a flat list of (a0, a1, c0, c1):
// consecutive rows with equal partner sets share a row range, and each
// partner set is split into contiguous runs.  Pairs are (smaller, larger)
// sphere indices below m; duplicates are allowed.  Returns an empty list
// when the cover needs more than max_rects rectangles.
std::vector<int32_t> self_pair_rectangles(int m, const std::vector<std::pair<int32_t, int32_t>> &pairs,
                                          int max_rects);

// A robot model rearranged for the kernels: spheres grouped by the frame
// they are attached to, one bounding sphere per frame (for the link-level
// broadphase), self pairs grouped by frame pair.
struct PreparedModel {
  int n_links = 0;                     // frames 0..n_links-1
  std::vector<float> spheres;          // m x 4, sorted by frame (stable)
  std::vector<int32_t> links;          // frame of each sorted sphere
  std::vector<int32_t> perm;           // sorted index -> caller's index
  std::vector<int32_t> link_start;     // n_links + 1: spheres of frame l are [start[l], start[l+1])
  std::vector<float> link_bs;          // n_links x 4: frame-local center, radius (radius < 0: no spheres)
  std::vector<std::pair<int32_t, int32_t>> self;  // (x < y) in sorted indices, by (frame x, frame y, x, y)
  std::vector<int32_t> self_groups;    // n_groups x 4: frame u, frame v, first pair, pair count
  // the same pairs per group as a block: rows = the spheres of the frame with
  // more of them, columns = the other frame's (at most 32), one bit mask of
  // listed partners per row.  n_groups x 4: first row sphere, first column
  // sphere, rows | columns << 16 | column frame << 24 | row frame << 28,
  // first mask.  Empty when a group's smaller frame holds more than 32
  // spheres (frames are below 16: at most MRV_MAX_DOF + 2 of them).
  std::vector<int32_t> self_blocks;
  std::vector<uint32_t> self_masks;
};

// Bounding sphere of a frame: center = middle of the bounding box of the
// frame's sphere centers, radius = max(|c_s - center| + r_s) computed in
// double and enlarged by a relative 1e-6 and an absolute 1e-4 (so an FP32
// separation test of two bounding spheres never hides a sphere overlap).
PreparedModel prepare_model(int n_links, int m, const int32_t *link, const float *xyzr, int n_self,
                            const int32_t *pairs);

// Uniform grid over a static obstacle set for the frame-level broadphase.
// A frame bounding sphere of radius <= R whose center lies in cell c can
// only overlap the obstacles listed for c: cell c lists every obstacle sphere
// within R + r_o (+ slack) of the cell's box, every box within R (+ slack) of
// it, and every cylinder whose bounding box (axis ends +- radius per axis)
// lies within R (+ slack) of it.  The slack (1e-3 cell + 1e-6 relative) covers the FP32
// computation of a center's cell.  Centers outside the grid overlap no
// obstacle.  Cell (ix, iy, iz) = [lo + i h, lo + (i + 1) h) per axis, index
// (iz * dims[1] + iy) * dims[0] + ix.
struct ObstacleGrid {
  double lo[3] = {0, 0, 0};
  double h = 0;
  double R = -1;                       // < 0: no grid (full scan)
  int dims[3] = {0, 0, 0};
  std::vector<int32_t> off;            // ncells + 1: items of cell c are [off[c], off[c+1])
  std::vector<uint16_t> ns;            // obstacle spheres listed first, ns[c] of them
  std::vector<uint16_t> nb;            // then nb[c] boxes, then the cylinders
  std::vector<uint16_t> items;         // obstacle sphere ids, box ids, cylinder ids
};

// Builds the grid for frames of radius <= R (at most 64 cells per axis,
// cells of at least R / 2).  Returns R = -1 (no grid) when R <= 0, there are
// no obstacles, any kind exceeds 65535, or the lists would pass max_items.
// cyl: n_cyl x 7 (axis end a, axis end b, radius).
ObstacleGrid build_obstacle_grid(int n_spheres, const float *xyzr, int n_boxes, const float *lohi, int n_cyl,
                                 const float *cyl, double R, int64_t max_items = int64_t(1) << 24);

}  // namespace mrv
