"""The comparison rules of tests/parity.py, exercised on the CPU.

Two discs of radius 0.25 on a timed path: a shallow overlap at t = 1
(clearance -5e-5 m, inside the 1e-4 m margin), clear at t = 2, a deep overlap
at t = 3.  The oracle's answer (1, 0, 1) is undecidable, so an FP32 answer
may be (1, 0, 1) or (3, 0, 1), but not one that passes over the deep conflict
and not a state where the pair is clear.  The checked "GPU" answers are
planted here; no device is involved.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2604_23960_gb300 import workloads as W
from tests import parity as PA


def _shallow_then_deep():
    d = W.disc_robot(0.25)
    bb = W.BatchBuilder(2, True)
    path1 = np.array([(3.0, 0.0), (0.49995, 0.0), (3.0, 0.0), (0.3, 0.0), (3.0, 0.0)], np.float32)
    path0 = np.array([(0.0, 0.0), (0.0, 0.0)], np.float32)
    bb.add([0, 0], [path0, path1], [[4], [1, 1, 1, 1]])
    return W.Workload("shallow_deep", [d], [], bb.build(0.05), env=-1, check_env=False)


def test_undecidable_ffc_rules():
    w = _shallow_then_deep()
    o = O.Oracle(w)
    assert tuple(o.ffc()[0]) == (1, 0, 1)
    assert not o.ffc_decidable()[0]
    assert tuple(o.ffc_below(-PA.MARGIN)[0]) == (3, 0, 1)
    for ok in ((1, 0, 1), (3, 0, 1)):
        PA.check_ffc(o, np.array([ok], np.int32))
    for bad in ((-1, -1, -1), (4, 0, 1), (2, 0, 1), (0, 0, 1)):
        with pytest.raises(AssertionError):
            PA.check_ffc(o, np.array([bad], np.int32))


def test_decidable_ffc_must_match():
    w = _shallow_then_deep()
    # move the shallow contact out of the margin band: the answer is decidable
    w.batch.waypoints[w.batch.slot_wp_off[1] + 1, 0] = np.float32(0.6)
    o = O.Oracle(w)
    assert o.ffc_decidable()[0]
    PA.check_ffc(o, o.ffc())
    with pytest.raises(AssertionError):
        PA.check_ffc(o, np.array([(1, 0, 1)], np.int32))
