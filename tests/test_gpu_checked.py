"""The bounds-checked build (libmrv_checked.so, kernels compiled with
MRV_CHECKED): every shared- and global-memory index of the kernels is
checked against its array, and a failure sets the call's error record and
comes back as MRV_ERR_CUDA naming the check.  A child process runs the
tiny, edge-case, cylinder, prioritized, 16-arm and ragged inputs of
tests/checked_child.py through every path with that build, and
benchmark-sized ragged, FFC, 8- and 16-arm batches: no check may fail, and
every output must equal this process's run of the normal build."""
from __future__ import annotations

import os
import subprocess
import sys
from pathlib import Path

import numpy as np
import pytest

from tests import checked_child

pytestmark = pytest.mark.gpu
ROOT = Path(__file__).resolve().parents[1]


def test_checked_build_clean_and_equal(tmp_path):
    from paper_2604_23960_gb300 import mrv
    assert (ROOT / "paper_2604_23960_gb300" / "libmrv_checked.so").exists(), "build() makes the checked library"
    out = tmp_path / "checked.npz"
    r = subprocess.run([sys.executable, "-m", "tests.checked_child", str(out)], cwd=ROOT,
                       env=dict(os.environ, MRV_LIBRARY="checked"), capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    got = np.load(out)
    assert str(got["library"]) == "libmrv_checked.so"
    ctx = mrv.Context(0)
    ref = checked_child.results(ctx)
    ctx.close()
    kind = ref["ragged_kind"]
    assert set(ref) == set(got.files) - {"library"}
    for k, v in ref.items():
        g = got[k]
        if k in ("ragged_v", "ragged_gv"):      # mrv_run writes each query's own output only
            np.testing.assert_array_equal(g[kind == 0], v[kind == 0], err_msg=k)
        elif k in ("ragged_c", "ragged_gc"):
            np.testing.assert_array_equal(g[kind == 1], v[kind == 1], err_msg=k)
        elif k == "big_ragged_v":
            np.testing.assert_array_equal(g[ref["big_ragged_kind"] == 0], v[ref["big_ragged_kind"] == 0], err_msg=k)
        elif k == "big_ragged_c":
            np.testing.assert_array_equal(g[ref["big_ragged_kind"] == 1], v[ref["big_ragged_kind"] == 1], err_msg=k)
        elif k.endswith("_mc") or k.endswith("_clr"):
            fin = np.isfinite(v)
            np.testing.assert_array_equal(np.isfinite(g), fin, err_msg=k)
            np.testing.assert_allclose(g[fin], v[fin], atol=1e-5, rtol=0, err_msg=k)
        else:
            np.testing.assert_array_equal(g, v, err_msg=k)
