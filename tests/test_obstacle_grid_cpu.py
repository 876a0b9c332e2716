"""Upload-time obstacle grid (host C++, checked on the CPU): for frame bounding
spheres of radius <= R, every obstacle sphere, box or cylinder that such a
sphere overlaps is listed in the cell of its center, with the cell computed in FP32
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
  int ns, nb, nc; double R;
  if (scanf("%d %d %d %lf", &ns, &nb, &nc, &R) != 4) return 2;
  std::vector<float> s(4 * ns), b(6 * nb), c(7 * nc);
  for (auto &v : s) if (scanf("%f", &v) != 1) return 2;
  for (auto &v : b) if (scanf("%f", &v) != 1) return 2;
  for (auto &v : c) if (scanf("%f", &v) != 1) return 2;
  auto G = mrv::build_obstacle_grid(ns, s.data(), nb, b.data(), nc, c.data(), R);
  printf("R %.17g\n", G.R);
  if (G.R < 0) return 0;
  printf("lo %.9g %.9g %.9g\n", (float)G.lo[0], (float)G.lo[1], (float)G.lo[2]);
  printf("inv_h %.9g\n", (float)(1.0 / G.h));
  printf("h %.17g\n", G.h);
  printf("dims %d %d %d\n", G.dims[0], G.dims[1], G.dims[2]);
  printf("off"); for (int v : G.off) printf(" %d", v); printf("\n");
  printf("ns"); for (int v : G.ns) printf(" %d", v); printf("\n");
  printf("nb"); for (int v : G.nb) printf(" %d", v); printf("\n");
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


def build(exe, spheres, boxes, R, cyls=None):
    cyls = np.zeros((0, 7)) if cyls is None else cyls
    inp = [f"{len(spheres)} {len(boxes)} {len(cyls)} {R!r}"]
    inp += [" ".join(f"{v:.9g}" for v in row) for row in spheres]
    inp += [" ".join(f"{v:.9g}" for v in row) for row in boxes]
    inp += [" ".join(f"{v:.9g}" for v in row) for row in cyls]
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


def cyl_dist(c, cyls):
    """Distance from points c (N x 3) to solid cylinders (M x 7), float64."""
    a, b, rho = cyls[None, :, :3], cyls[None, :, 3:6], cyls[None, :, 6]
    L = np.linalg.norm(b - a, axis=2)
    u = (b - a) / L[..., None]
    w = c[:, None, :] - a
    s = np.sum(w * u, axis=2)
    d = np.linalg.norm(w - s[..., None] * u, axis=2)
    es = np.maximum(np.maximum(-s, s - L), 0.0)
    ed = np.maximum(d - rho, 0.0)
    return np.hypot(es, ed)


def overlap_masks(c, r, spheres, boxes, cyls):
    """float64 overlap of spheres (c, r) with every obstacle: (N x ns, N x nb, N x nc)."""
    c = np.asarray(c, np.float64)
    ds = np.linalg.norm(c[:, None, :] - spheres[None, :, :3], axis=2)
    q = np.clip(c[:, None, :], boxes[None, :, :3], boxes[None, :, 3:])
    db = np.linalg.norm(c[:, None, :] - q, axis=2)
    dc = cyl_dist(c, cyls) if len(cyls) else np.zeros((len(c), 0))
    return ds < r[:, None] + spheres[None, :, 3], db < r[:, None], dc < r[:, None]


def listed_masks(g, cells, n_s, n_b, n_c):
    """Obstacles listed in each cell (N x ns, N x nb, N x nc booleans)."""
    off = np.asarray([int(v) for v in g["off"]])
    ns = np.asarray([int(v) for v in g["ns"]])
    nb = np.asarray([int(v) for v in g["nb"]])
    items = np.asarray([int(v) for v in g["items"]])
    ms = np.zeros((len(cells), n_s), bool)
    mb = np.zeros((len(cells), n_b), bool)
    mc = np.zeros((len(cells), n_c), bool)
    for n, c in enumerate(cells):
        if c < 0:
            continue
        a, z = off[c], off[c + 1]
        ms[n, items[a:a + ns[c]]] = True
        mb[n, items[a + ns[c]:a + ns[c] + nb[c]]] = True
        mc[n, items[a + ns[c] + nb[c]:z]] = True
    return ms, mb, mc


def check(g, c, r, spheres, boxes, cyls=None):
    cyls = np.zeros((0, 7)) if cyls is None else np.asarray(cyls, np.float32).astype(np.float64)
    os_, ob, oc = overlap_masks(c, r, spheres, boxes, cyls)
    cells = cells_of(g, np.asarray(c, np.float32))
    ls, lb, lc = listed_masks(g, cells, len(spheres), len(boxes), len(cyls))
    out = cells < 0
    assert not os_[out].any() and not ob[out].any() and not oc[out].any(), \
        "a center outside the grid overlaps an obstacle"
    assert not (os_ & ~ls).any() and not (ob & ~lb).any() and not (oc & ~lc).any(), \
        "an overlapping obstacle is not listed"
    return int(os_.sum() + ob.sum() + oc.sum())


def scene(rng, n_s, n_b, n_c=0):
    spheres = np.concatenate([rng.uniform(-1, 1, (n_s, 3)) * [1, 1, 0.8] + [0, 0, 0.8],
                              rng.uniform(0.02, 0.12, (n_s, 1))], axis=1)
    lo = rng.uniform(-1.1, 1.0, (n_b, 3))
    boxes = np.concatenate([lo, lo + rng.uniform(0.02, 0.8, (n_b, 3))], axis=1)
    if not n_c:
        return spheres, boxes
    a = rng.uniform(-1, 1, (n_c, 3)) * [1, 1, 0.8] + [0, 0, 0.8]
    d = rng.normal(size=(n_c, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    cyls = np.concatenate([a, a + d * rng.uniform(0.1, 1.2, (n_c, 1)), rng.uniform(0.01, 0.15, (n_c, 1))], axis=1)
    return spheres, boxes, cyls


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


@pytest.mark.parametrize("seed", range(3))
def test_grid_lists_every_cylinder_overlap(exe, seed):
    rng = np.random.default_rng(600 + seed)
    spheres, boxes, cyls = scene(rng, 20, 6, 16)
    R = float(np.float32(rng.uniform(0.1, 0.35)))
    g = build(exe, spheres, boxes, R, cyls)
    N = 20000
    c = rng.uniform(-1.6, 1.6, (N, 3)) * [1, 1, 0.9] + [0, 0, 0.8]
    r = rng.uniform(0.0, R, N)
    assert check(g, c, r, spheres, boxes, cyls) > 1000


def test_grid_cylinders_only(exe):
    """A cage of cylinders alone (no spheres or boxes) builds a grid."""
    rng = np.random.default_rng(9)
    _, _, cyls = scene(rng, 1, 1, 12)
    g = build(exe, np.zeros((0, 4)), np.zeros((0, 6)), 0.25, cyls)
    assert float(g["R"][0]) > 0
    N = 10000
    c = rng.uniform(-1.6, 1.6, (N, 3)) * [1, 1, 0.9] + [0, 0, 0.8]
    assert check(g, c, np.full(N, 0.25), np.zeros((0, 4)), np.zeros((0, 6)), cyls) > 100
