"""Upload-time model preparation (host C++, checked on the CPU): spheres are
regrouped by frame without losing any, every frame's bounding sphere encloses
its spheres with the stated margin, and the self pairs are regrouped by frame
pair without losing or adding any."""
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
  int L, m, n; if (scanf("%d %d %d", &L, &m, &n) != 3) return 2;
  std::vector<int> link(m); std::vector<float> x(4 * m); std::vector<int> pr(2 * n);
  for (int i = 0; i < m; ++i) if (scanf("%d %f %f %f %f", &link[i], &x[4*i], &x[4*i+1], &x[4*i+2], &x[4*i+3]) != 5) return 2;
  for (int p = 0; p < 2 * n; ++p) if (scanf("%d", &pr[p]) != 1) return 2;
  auto P = mrv::prepare_model(L, m, link.data(), x.data(), n, pr.data());
  printf("perm"); for (int v : P.perm) printf(" %d", v); printf("\n");
  printf("start"); for (int v : P.link_start) printf(" %d", v); printf("\n");
  printf("bs"); for (float v : P.link_bs) printf(" %.9g", v); printf("\n");
  printf("self"); for (auto &e : P.self) printf(" %d %d", e.first, e.second); printf("\n");
  printf("groups"); for (int v : P.self_groups) printf(" %d", v); printf("\n");
  printf("blocks"); for (int v : P.self_blocks) printf(" %d", v); printf("\n");
  printf("masks"); for (unsigned v : P.self_masks) printf(" %u", v); printf("\n");
  return 0;
}
'''


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    d = tmp_path_factory.mktemp("prep")
    (d / "drv.cpp").write_text(DRIVER)
    out = d / "drv"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", str(CSRC), str(d / "drv.cpp"), str(CSRC / "mrv_geometry.cpp"),
                    "-o", str(out)], check=True)
    return out


def run(exe, L, link, xyzr, pairs):
    inp = [f"{L} {len(link)} {len(pairs)}"]
    inp += [f"{l} {a:.9g} {b:.9g} {c:.9g} {r:.9g}" for l, (a, b, c, r) in zip(link, xyzr)]
    inp += [f"{a} {b}" for a, b in pairs]
    out = subprocess.run([str(exe)], input="\n".join(inp), capture_output=True, text=True, check=True).stdout
    d = {}
    for line in out.splitlines():
        k, *v = line.split()
        d[k] = v
    return d


@pytest.mark.parametrize("seed", range(4))
def test_prepare_model(exe, seed):
    rng = np.random.default_rng(seed)
    L = int(rng.integers(2, 10))
    m = int(rng.integers(1, 80))
    link = rng.integers(0, L, m)
    xyzr = np.column_stack([rng.uniform(-0.5, 0.5, (m, 3)), rng.uniform(0.01, 0.2, m)]).astype(np.float32)
    allp = [(a, b) for a in range(m) for b in range(m) if a != b]
    pairs = [allp[i] for i in rng.choice(len(allp), size=min(len(allp), int(rng.integers(0, 200))), replace=False)]
    d = run(exe, L, link, xyzr, pairs)
    perm = np.array(d["perm"], int)
    assert sorted(perm) == list(range(m))
    slink = link[perm]
    assert np.all(np.diff(slink) >= 0)
    start = np.array(d["start"], int)
    assert start[0] == 0 and start[-1] == m
    bs = np.array(d["bs"], float).reshape(L, 4)
    for l in range(L):
        idx = perm[start[l]:start[l + 1]]
        assert np.all(link[idx] == l)
        if len(idx) == 0:
            assert bs[l, 3] < 0
            continue
        dist = np.linalg.norm(xyzr[idx, :3].astype(np.float64) - bs[l, :3], axis=1) + xyzr[idx, 3]
        assert np.all(dist + 1e-4 <= bs[l, 3] + 1e-12)
    inv = np.argsort(perm)
    want = sorted({(min(inv[a], inv[b]), max(inv[a], inv[b])) for a, b in pairs} | set())
    got = [tuple(map(int, d["self"][k:k + 2])) for k in range(0, len(d["self"]), 2)]
    assert sorted(set(got)) == want
    assert len(got) == len(pairs)
    g = np.array(d["groups"], int).reshape(-1, 4)
    covered = 0
    for u, v, s0, cnt in g:
        for a, b in got[s0:s0 + cnt]:
            assert slink[a] == u and slink[b] == v
        covered += cnt
    assert covered == len(got)
    check_blocks(d, g, got, start)


def check_blocks(d, g, got, start):
    """Every group's block (rows = the frame with more spheres, columns = the
    other, at most 32) lists exactly the group's pairs, each once."""
    blocks = np.array(d.get("blocks", []), int).reshape(-1, 4)
    masks = [int(v) for v in d.get("masks", [])]
    counts = np.diff(start)
    if len(blocks) == 0:
        # only when some group's smaller frame has more than 32 spheres
        assert len(g) == 0 or any(min(counts[u], counts[v]) > 32 for u, v, _, _ in g)
        return
    assert len(blocks) == len(g)
    for (u, v, s0, cnt), (r0, c0, rc, m0) in zip(g, blocks):
        rc &= 0xffffffff
        nr, nc, cf, rf = rc & 0xffff, (rc >> 16) & 0xff, (rc >> 24) & 0xf, rc >> 28
        assert nc <= 32 and nr >= nc
        assert {(r0, nr), (c0, nc)} == {(start[u], counts[u]), (start[v], counts[v])}
        assert {rf, cf} == {u, v} and (r0, c0) == (start[rf], start[cf])
        listed = set()
        for row in range(nr):
            for c in range(nc):
                if masks[m0 + row] >> c & 1:
                    listed.add(tuple(sorted((r0 + row, c0 + c))))
        want = {tuple(sorted(p)) for p in got[s0:s0 + cnt]}
        assert listed == want and sum(bin(masks[m0 + row]).count("1") for row in range(nr)) == len(want)


def test_blocks_wide_frames(exe):
    """A model whose frames both exceed 32 spheres keeps the pair list only;
    one with a 32-sphere frame against a large one uses blocks."""
    rng = np.random.default_rng(9)
    for n0, n1, expect in ((40, 40, False), (60, 32, True)):
        link = np.array([0] * n0 + [1] * n1)
        xyzr = np.column_stack([rng.uniform(-0.5, 0.5, (len(link), 3)), np.full(len(link), 0.05)]).astype(np.float32)
        pairs = [(a, n0 + b) for a in range(0, n0, 3) for b in range(0, n1, 2)]
        d = run(exe, 2, link, xyzr, pairs)
        got = [tuple(map(int, d["self"][k:k + 2])) for k in range(0, len(d["self"]), 2)]
        g = np.array(d["groups"], int).reshape(-1, 4)
        assert (len(d.get("blocks", [])) > 0) == expect
        check_blocks(d, g, got, np.array(d["start"], int))
