"""The upload-time rectangle cover of self-collision pairs is exact: every
listed pair (a < b after normalisation) lies in exactly one rectangle and no
rectangle holds an unlisted pair.  Checked through a C++ build of the same
routine on the CPU (no GPU call)."""
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
#include <utility>
#include "mrv_geometry.h"
int main() {
  int m, n; if (scanf("%d %d", &m, &n) != 2) return 2;
  std::vector<std::pair<int,int>> p(n);
  for (auto &e : p) { int a, b; if (scanf("%d %d", &a, &b) != 2) return 2; e = {a < b ? a : b, a < b ? b : a}; }
  auto r = mrv::self_pair_rectangles(m, p, 100000);
  for (size_t k = 0; k < r.size(); k += 4) printf("%d %d %d %d\n", r[k], r[k+1], r[k+2], r[k+3]);
  return 0;
}
'''


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    d = tmp_path_factory.mktemp("rects")
    (d / "drv.cpp").write_text(DRIVER)
    out = d / "drv"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", str(CSRC), str(d / "drv.cpp"), str(CSRC / "mrv_geometry.cpp"),
                    "-o", str(out)], check=True)
    return out


def cover(exe, m, pairs):
    inp = f"{m} {len(pairs)}\n" + "\n".join(f"{a} {b}" for a, b in pairs)
    r = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True)
    return [tuple(map(int, l.split())) for l in r.stdout.splitlines()]


@pytest.mark.parametrize("seed", range(5))
def test_cover_is_exact(exe, seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(2, 70))
    allp = [(a, b) for a in range(m) for b in range(a + 1, m)]
    keep = [allp[i] for i in np.nonzero(rng.uniform(size=len(allp)) < rng.uniform(0.2, 0.95))[0]]
    # duplicates and reversed pairs are allowed in the input
    pairs = keep + [(b, a) for a, b in keep[: len(keep) // 5]]
    got = set()
    for a0, a1, c0, c1 in cover(exe, m, pairs):
        for a in range(a0, a1):
            for c in range(c0, c1):
                assert a < c
                assert (a, c) not in got
                got.add((a, c))
    assert got == set(keep)


def test_cage_fixture_cover(exe):
    from paper_2604_23960_gb300 import workloads as W
    sp = W.load_cage_fixtures()["self_pairs"]
    rects = cover(exe, 64, [tuple(p) for p in sp])
    assert sum((a1 - a0) * (c1 - c0) for a0, a1, c0, c1 in rects) == len({tuple(sorted(p)) for p in sp})
