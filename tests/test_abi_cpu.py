"""CPU checks of the C ABI: the library builds, loads, exports every entry
point include/mrv.h declares, and fails cleanly (a status code, no abort)
where no GPU is present.  No compute call is made here."""
from __future__ import annotations

import ctypes as C
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    text = (ROOT / "include" / "mrv.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", text, re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "sizeof")))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_23960_gb300 import build, mrv
    build.build()
    return mrv.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("robot_model_upload", "env_upload", "mv_validate", "ffc_find", "mrv_run", "mrv_clearance",
                     "mrv_create", "mrv_destroy", "mrv_sync", "mrv_release"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in mrv.h but not exported"


def test_binding_covers_the_header():
    from paper_2604_23960_gb300 import mrv
    assert set(declared_functions()) <= set(mrv.SIGNATURES)


def test_struct_layouts_match_header(lib, tmp_path):
    """ctypes mirrors of the ABI structs have the C compiler's sizes and
    field offsets."""
    import subprocess
    from paper_2604_23960_gb300 import mrv
    pairs = {"mrv_batch": mrv.BatchS, "mrv_robot_desc": mrv.RobotDesc, "mrv_env_desc": mrv.EnvDesc,
             "mrv_conflict": mrv.Conflict, "mrv_stats": mrv.Stats, "mrv_tuning": mrv.Tuning,
             "mrv_server_opts": mrv.ServerOpts, "mrv_server_stats": mrv.ServerStats, "mrv_limits": mrv.Limits}
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{ROOT / "include" / "mrv.h"}"', "int main(void){"]
    for cname, py in pairs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines())
    for cname, py in pairs.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, f"{cname}.{f}"


def test_null_arguments_are_rejected(lib):
    from paper_2604_23960_gb300 import mrv
    assert lib.mrv_create(None, 0, None) == -1
    assert lib.mv_validate(None, None, None, None) == -1
    assert lib.ffc_find(None, None, None) == -1
    assert lib.mrv_destroy(None) == 0
    assert b"NULL" in lib.mrv_last_error(None)
    assert mrv.ERR_NAMES[-1] == "MRV_ERR_ARG"


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    rc = lib.mrv_create(C.byref(h), 0, None)
    assert rc == -4   # MRV_ERR_CUDA
    assert not h.value


def test_product_path_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2604_23960_gb300 import mrv
    monkeypatch.setattr(mrv, "LIB_PATH", tmp_path / "missing.so")
    monkeypatch.setattr(mrv, "_lib", None)
    with pytest.raises(ImportError):
        mrv.lib()


def test_checked_library_exports_the_same_boundary(lib):
    """The bounds-checked build (MRV_CHECKED kernels) is a drop-in library:
    it loads, exports every declared entry point and fails cleanly too."""
    from paper_2604_23960_gb300 import build
    assert build.LIB_CHECKED.exists()
    L = C.CDLL(str(build.LIB_CHECKED))
    for name in declared_functions():
        assert hasattr(L, name), f"{name} missing from the checked library"
    L.mrv_last_error.restype = C.c_char_p
    assert L.mv_validate(None, None, None, None) == -1


def test_library_variant_is_selected_loudly(monkeypatch):
    """MRV_LIBRARY picks the library variant; an unknown value is an error,
    never a silent fallback."""
    import importlib
    import sys
    monkeypatch.setenv("MRV_LIBRARY", "nonsense")
    sys.modules.pop("paper_2604_23960_gb300.mrv", None)
    with pytest.raises(ImportError):
        importlib.import_module("paper_2604_23960_gb300.mrv")
    monkeypatch.setenv("MRV_LIBRARY", "checked")
    sys.modules.pop("paper_2604_23960_gb300.mrv", None)
    m = importlib.import_module("paper_2604_23960_gb300.mrv")
    assert m.LIB_PATH.name == "libmrv_checked.so"
    monkeypatch.delenv("MRV_LIBRARY")
    sys.modules.pop("paper_2604_23960_gb300.mrv", None)
    assert importlib.import_module("paper_2604_23960_gb300.mrv").LIB_PATH.name == "libmrv.so"
