"""Build liblbm.so in-tree for sm_103a (GB300) with nvcc.

The translation units compile in parallel (one per lattice plus the host
runtime), then link into ``paper_1710_02065_gb300/_build/liblbm.so`` with the
CUDA runtime linked statically.  ``python -m paper_1710_02065_gb300.build``
rebuilds; ``build(verbose=True)`` prints ptxas register/spill reports.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblbm.so")
CHECKED_LIB = os.path.join(BUILD, "liblbm_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["lbm_api.cu", "step_d2q9.cu", "step_d3q19.cu", "step_d3q27.cu", "stepvec_d2q9.cu", "stepvec_d3q19.cu",
           "stepvec_d3q27.cu", "aa_d2q9.cu", "aa_d3q19.cu", "aa_d3q27.cu",
           "rows_d2q9.cu", "rows_d3q19.cu", "lbm_noalloc.cu", "lbm_serve.cu"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found (set NVCC or put CUDA's bin on PATH)")


def _deps() -> list[str]:
    out = [os.path.join(INCLUDE, "lbm.h")]
    for name in os.listdir(CSRC):
        out.append(os.path.join(CSRC, name))
    return out


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False, checked: bool = False) -> str:
    """Compile the CUDA sources and link liblbm.so; returns its path.
    checked=True builds liblbm_checked.so instead: the same library with every
    index of the update kernels tested before use (-DLBM_BOUNDS_CHECK; a bad
    index skips the cell and is reported by lbm_sync).  The binding loads it
    when the environment variable LBM_CHECKED is 1."""
    build_dir = os.path.join(BUILD, "checked") if checked else BUILD
    lib = CHECKED_LIB if checked else LIB
    os.makedirs(build_dir, exist_ok=True)
    deps = _deps()
    if not force and not _stale(lib, deps):
        return lib
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", INCLUDE, "-I", CSRC]
    if checked:
        common += ["-DLBM_BOUNDS_CHECK"]
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(src: str) -> str:
        obj = os.path.join(build_dir, src.replace(".cu", ".o"))
        cmd = [nvcc, *common, "-c", os.path.join(CSRC, src), "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
        if verbose:
            sys.stderr.write(res.stdout + res.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
