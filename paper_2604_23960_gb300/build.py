"""In-tree build of ``libmrv.so`` (CUDA kernels for sm_103a + the C++ host
runtime) and of ``libmrv_checked.so``, the same library with the kernels
compiled with MRV_CHECKED (every shared- and global-memory index checked
against its array; a failure is reported as a status, never a fault).
Translation units of both compile in parallel; the libraries are linked with
the static CUDA runtime so they only need the driver at load time."""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
INCLUDE = PKG.parent / "include"
BUILD = PKG / "_build"
LIB = PKG / "libmrv.so"
LIB_CHECKED = PKG / "libmrv_checked.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["mrv_kernels.cu", "mrv_noalloc.cu"]
CPP_SOURCES = ["mrv_api.cpp", "mrv_tune.cpp", "mrv_server.cpp", "mrv_geometry.cpp"]


def _cuda_home() -> Path:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and Path(c, "bin", "nvcc").exists():
            return Path(c)
    nvcc = shutil.which("nvcc")
    if nvcc:
        return Path(nvcc).resolve().parents[1]
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _headers():
    return list(CSRC.glob("*.h")) + list(INCLUDE.glob("*.h"))


def _stale(obj: Path, src: Path) -> bool:
    if not obj.exists():
        return True
    t = obj.stat().st_mtime
    return any(p.stat().st_mtime > t for p in [src, *_headers()])


def build(force: bool = False, verbose: bool = False, checked: bool = True) -> Path:
    """Builds libmrv.so (and, with checked, libmrv_checked.so); returns the
    path of libmrv.so."""
    cuda = _cuda_home()
    nvcc = str(cuda / "bin" / "nvcc")
    BUILD.mkdir(exist_ok=True)
    (BUILD / "checked").mkdir(exist_ok=True)
    jobs = []
    cpp_objs, cu_objs = [], {False: [], True: []}
    for variant in ((False, True) if checked else (False,)):
        for s in CU_SOURCES:
            src = CSRC / s
            if not src.exists():
                continue
            obj = (BUILD / "checked" if variant else BUILD) / (s + ".o")
            cu_objs[variant].append(obj)
            if force or _stale(obj, src):
                jobs.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                             *(["-DMRV_CHECKED"] if variant else []),
                             "-Xptxas", "-v" if verbose else "-O3", "-I", str(INCLUDE), "-c", str(src), "-o",
                             str(obj)])
    for s in CPP_SOURCES:
        src = CSRC / s
        if not src.exists():
            continue
        obj = BUILD / (s + ".o")
        cpp_objs.append(obj)
        if force or _stale(obj, src):
            jobs.append(["g++", "-std=c++17", "-O2", "-fPIC", "-ffp-contract=off", "-Wall", "-Wno-unused-function",
                         "-I", str(cuda / "include"), "-I", str(INCLUDE), "-c", str(src), "-o", str(obj)])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r.stdout + r.stderr

    with ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        outs = list(ex.map(run, jobs))
    if verbose:
        for o in outs:
            print(o)
    for variant, lib in ((False, LIB), (True, LIB_CHECKED)):
        if variant and not checked:
            continue
        objs = cu_objs[variant] + cpp_objs
        if force or jobs or not lib.exists() or any(o.stat().st_mtime > lib.stat().st_mtime for o in objs):
            tmp = lib.with_suffix(f".so.{os.getpid()}")
            run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", str(tmp), *map(str, objs), "-lpthread", "-ldl",
                 "-lrt"])
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
