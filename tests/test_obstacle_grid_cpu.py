"""Upload-time obstacle grid (host C++, checked on the CPU): for frame bounding
spheres of radius <= R, every obstacle sphere or box that such a sphere
overlaps is listed in the cell of its center, with the cell computed in FP32
the way the kernel computes it, and centers outside the grid overlap nothing.
The grid only narrows the candidate set of the bounding-sphere tests, so this
property is all the broadphase needs to stay exact."""
from __future__ import annotations

import subprocess
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]
CSRC = ROOT / "paper_2604_23960_gb300" / "csrc"

DRIVER = r'''
#include <cstdio>
#include <vector>
#include "mrv_geometry.h"
int main() {
  int ns, nb; double R;
  if (scanf("%d %d %lf", &ns, &nb, &R) != 3) return 2;
  std::vector<float> s(4 * ns), b(6 * nb);
  for (auto &v : s) if (scanf("%f", &v) != 1) return 2;
  for (auto &v : b) if (scanf("%f", &v) != 1) return 2;
  auto G = mrv::build_obstacle_grid(ns, s.data(), nb, b.data(), R);
  printf("R %.17g\n", G.R);
  if (G.R < 0) return 0;
  printf("lo %.9g %.9g %.9g\n", (float)G.lo[0], (float)G.lo[1], (float)G.lo[2]);
  printf("inv_h %.9g\n", (float)(1.0 / G.h));
  printf("h %.17g\n", G.h);
  printf("dims %d %d %d\n", G.dims[0], G.dims[1], G.dims[2]);
  printf("off"); for (int v : G.off) printf(" %d", v); printf("\n");
  printf("ns"); for (int v : G.ns) printf(" %d", v); printf("\n");
  printf("items"); for (int v : G.items) printf(" %d", v); printf("\n");
  return 0;
}
'''


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    d = tmp_path_factory.mktemp("grid")
    (d / "drv.cpp").write_text(DRIVER)
    out = d / "drv"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", str(CSRC), str(d / "drv.cpp"), str(CSRC / "mrv_geometry.cpp"),
                    "-o", str(out)], check=True)
    return out


def build(exe, spheres, boxes, R):
    inp = [f"{len(spheres)} {len(boxes)} {R!r}"]
    inp += [" ".join(f"{v:.9g}" for v in row) for row in spheres]
    inp += [" ".join(f"{v:.9g}" for v in row) for row in boxes]
    out = subprocess.run([str(exe)], input="\n".join(inp) + "\n", capture_output=True, text=True, check=True).stdout
    d = {}
    for line in out.splitlines():
        k, *v = line.split()
        d[k] = v
    return d


def cells_of(g, x):
    """The kernel's cell lookup (FP32) for centers x (N x 3): flat indices, -1 outside."""
    lo = np.asarray(g["lo"], np.float32)
    ih = np.float32(g["inv_h"][0])
    dims = np.asarray([int(v) for v in g["dims"]])
    f = (np.asarray(x, np.float32) - lo) * ih
    inside = np.all((f >= 0) & (f < dims.astype(np.float32)), axis=1)
    i = np.where(inside[:, None], f, 0).astype(np.int64)
    return np.where(inside, (i[:, 2] * dims[1] + i[:, 1]) * dims[0] + i[:, 0], -1)


def overlap_masks(c, r, spheres, boxes):
    """float64 overlap of spheres (c, r) with every obstacle: (N x ns, N x nb)."""
    c = np.asarray(c, np.float64)
    ds = np.linalg.norm(c[:, None, :] - spheres[None, :, :3], axis=2)
    q = np.clip(c[:, None, :], boxes[None, :, :3], boxes[None, :, 3:])
    db = np.linalg.norm(c[:, None, :] - q, axis=2)
    return ds < r[:, None] + spheres[None, :, 3], db < r[:, None]


def listed_masks(g, cells, n_s, n_b):
    """Obstacles listed in each cell (N x ns, N x nb booleans)."""
    off = np.asarray([int(v) for v in g["off"]])
    ns = np.asarray([int(v) for v in g["ns"]])
    items = np.asarray([int(v) for v in g["items"]])
    ms = np.zeros((len(cells), n_s), bool)
    mb = np.zeros((len(cells), n_b), bool)
    for n, c in enumerate(cells):
        if c < 0:
            continue
        a, z = off[c], off[c + 1]
        ms[n, items[a:a + ns[c]]] = True
        mb[n, items[a + ns[c]:z]] = True
    return ms, mb


def check(g, c, r, spheres, boxes):
    os_, ob = overlap_masks(c, r, spheres, boxes)
    cells = cells_of(g, np.asarray(c, np.float32))
    ls, lb = listed_masks(g, cells, len(spheres), len(boxes))
    out = cells < 0
    assert not os_[out].any() and not ob[out].any(), "a center outside the grid overlaps an obstacle"
    assert not (os_ & ~ls).any() and not (ob & ~lb).any(), "an overlapping obstacle is not listed"
    return int(os_.sum() + ob.sum())


def scene(rng, n_s, n_b):
    spheres = np.concatenate([rng.uniform(-1, 1, (n_s, 3)) * [1, 1, 0.8] + [0, 0, 0.8],
                              rng.uniform(0.02, 0.12, (n_s, 1))], axis=1)
    lo = rng.uniform(-1.1, 1.0, (n_b, 3))
    boxes = np.concatenate([lo, lo + rng.uniform(0.02, 0.8, (n_b, 3))], axis=1)
    return spheres, boxes


@pytest.mark.parametrize("seed", range(3))
def test_grid_lists_every_overlap(exe, seed):
    rng = np.random.default_rng(500 + seed)
    spheres, boxes = scene(rng, 40, 12)
    R = float(np.float32(rng.uniform(0.1, 0.35)))
    g = build(exe, spheres, boxes, R)
    assert float(g["R"][0]) == R
    n_cells = int(np.prod([int(v) for v in g["dims"]]))
    assert len(g["off"]) == n_cells + 1 and max(int(v) for v in g["dims"]) <= 64
    assert float(g["h"][0]) >= R / 2 * (1 - 1e-12)
    N = 20000
    c = rng.uniform(-1.6, 1.6, (N, 3)) * [1, 1, 0.9] + [0, 0, 0.8]
    r = rng.uniform(0.0, R, N)
    assert check(g, c, r, spheres, boxes) > 1000   # the draw really exercised overlaps
    # and the lists prune: a cell lists far fewer than all obstacles on average
    off = np.asarray([int(v) for v in g["off"]])
    assert (off[-1] / n_cells) < 0.5 * (len(spheres) + len(boxes))


def test_grid_centers_on_cell_faces(exe):
    """Centers on cell boundaries (where FP32 rounding can move them to the
    neighbour cell), at the full radius bound, still find every overlap."""
    rng = np.random.default_rng(7)
    spheres, boxes = scene(rng, 25, 8)
    R = 0.25
    g = build(exe, spheres, boxes, R)
    lo = np.asarray([float(v) for v in g["lo"]])
    h = float(g["h"][0])
    dims = np.asarray([int(v) for v in g["dims"]])
    N = 20000
    c = lo + rng.integers(0, dims + 1, (N, 3)) * h
    axis = rng.integers(0, 3, N)
    c[np.arange(N), axis] += rng.choice([-1, 1], N) * rng.uniform(0, 1e-6, N)
    assert check(g, c, np.full(N, R), spheres, boxes) > 100


def test_grid_declines(exe):
    rng = np.random.default_rng(3)
    spheres, boxes = scene(rng, 4, 2)
    assert float(build(exe, spheres, boxes, 0.0)["R"][0]) < 0        # no radius bound
    assert float(build(exe, spheres[:0], boxes[:0], 0.2)["R"][0]) < 0  # no obstacles
