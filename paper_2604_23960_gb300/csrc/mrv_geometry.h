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

}  // namespace mrv
