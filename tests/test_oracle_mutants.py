"""Planted mistakes in the oracle must fail its pins.

Each case copies the oracle's C source, plants one plausible mistake (a sign,
a dropped term, a transposed product, an off-by-one, a wrong padding or tie
order), builds it on the CPU and runs the pin suite against that build in a
child process; the pins must fail.  The unmodified source must pass.
"""
from __future__ import annotations

import os
import subprocess
import sys
from pathlib import Path

import pytest

from oracle import oracle as O

ROOT = Path(__file__).resolve().parents[1]

MUTANTS = {
    "rot_x_sign": ("r.m[1][2] = -sin(a);", "r.m[1][2] = sin(a);"),
    "dh_order": ("mat4 t1 = mat_mul(&rx, &tx);\n  mat4 t2 = mat_mul(&t1, &rz);",
                 "mat4 t1 = mat_mul(&rx, &rz);\n  mat4 t2 = mat_mul(&t1, &tx);"),
    "flange_dropped": ("mat4 fl = r->flange ? mat_from34(r->flange) : mat_identity();",
                       "mat4 fl = mat_identity();"),
    "last_state_dropped": ("for (int64_t t = 0; t <= T && !found; ++t) {",
                           "for (int64_t t = 0; t < T && !found; ++t) {"),
    "mv_last_state_dropped": ("for (int64_t t = 0; t <= T && valid; ++t) {",
                              "for (int64_t t = 0; t < T && valid; ++t) {"),
    "ffc_pair_order": ("for (int i = 0; i < qs.n && !found; ++i)\n      for (int j = i + 1; j < qs.n && !found; ++j)\n        if (pair_min(&qs, i, j) < 0.0) {",
                       "for (int j = 1; j < qs.n && !found; ++j)\n      for (int i = 0; i < j && !found; ++i)\n        if (pair_min(&qs, i, j) < 0.0) {"),
    "pad_first": ("const float *l = W + (size_t)(w1 - 1) * st;", "const float *l = W + (size_t)w0 * st;"),
    "box_sign": ("else if (c[i] > hi) e = c[i] - hi;", "else if (c[i] > hi) e = hi - c[i] - 1.0;"),
    "interp_offbyone": ("double f = (double)(t - tau) / (double)n;", "double f = (double)(t - tau) / (double)(n + 1);"),
    "steps_floor": ("return (int64_t)ceil(dist / res);", "return (int64_t)floor(dist / res);"),
    "self_dropped": ("for (int p = 0; p < r->n_self; ++p) {\n    int a = r->self_pairs[2 * p], c = r->self_pairs[2 * p + 1];\n    double v",
                     "for (int p = 0; p < 0; ++p) {\n    int a = r->self_pairs[2 * p], c = r->self_pairs[2 * p + 1];\n    double v"),
    "obstacle_radius_dropped": ("double v = orc_sphere_sphere(C + 3 * a, ra, co, e->spheres[4 * o + 3]);",
                                "double v = orc_sphere_sphere(C + 3 * a, ra, co, 0.0);"),
    "base_ignored": ("frame[0] = mat_from34(r->base);", "frame[0] = mat_identity();"),
    "theta_offset_dropped": ("(double)row[3] + q[k - 1]", "q[k - 1]"),
    "prio_pairs_chained": ("if (pair_min(&qs, 0, j) < 0.0) valid = 0;", "if (pair_min(&qs, j - 1, j) < 0.0) valid = 0;"),
    "prio_env_other_robot": ("if (check_env && env_self_min(&qs, env, 0) < 0.0) valid = 0;",
                             "if (check_env && env_self_min(&qs, env, qs.n - 1) < 0.0) valid = 0;"),
    "prio_clearance_pairs": ("double v = pair_min(&qs, 0, j);", "double v = pair_min(&qs, j - 1, j);"),
    "cyl_caps_dropped": ("const double es = s < 0.0 ? -s : (s > L ? s - L : 0.0);", "const double es = 0.0;"),
    "cyl_axis_unnormalised": ("for (int k = 0; k < 3; ++k) u[k] /= L;", "for (int k = 0; k < 3; ++k) u[k] /= 1.0;"),
    "cyl_radius_dropped": ("const double ed = d > rho ? d - rho : 0.0;", "const double ed = d;"),
    "cyl_ignored_in_mv": ("      for (int o = 0; o < e->n_cylinders; ++o) {", "      for (int o = 0; o < 0; ++o) {"),
    "ffc_below_bound_ignored": ("if (pair_min(&qs, i, j) < bound) {", "if (pair_min(&qs, i, j) < 0.0) {"),
    "ffc_below_bound_sign": ("if (pair_min(&qs, i, j) < bound) {", "if (pair_min(&qs, i, j) < -bound) {"),
}

PIN_ARGS = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
            str(ROOT / "tests" / "test_oracle_pins.py")]


def _run_pins(lib: Path) -> int:
    env = dict(os.environ, MRV_ORACLE_LIB=str(lib))
    return subprocess.run(PIN_ARGS, cwd=ROOT, env=env, capture_output=True, timeout=600).returncode


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    src = O.SRC.read_text()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site of {name} not unique"
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    lib = O.build(src=mut, out=tmp_path / "libmut.so")
    assert _run_pins(lib) != 0, f"pins did not catch mutant {name}"


def test_unmodified_passes(tmp_path):
    lib = O.build(src=O.SRC, out=tmp_path / "liborig.so")
    assert _run_pins(lib) == 0
