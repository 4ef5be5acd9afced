"""Build libteno7.so (the CUDA kernels + C ABI) in-tree for sm_103a with nvcc.

Each translation unit is compiled in parallel, then linked into one shared
library next to this file.  teno7_f64.cu and teno7_slab2d_f64.cu are compiled
with -fmad=false so that the FP64 path evaluates every expression operation by
operation.  build(checked=True) makes libteno7_checked.so from the same
sources with T7_CHECKED=1: every array index the kernels form is checked (a
stand-in for a memory checker, for tests; see include/teno7.h).
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = PKG / "libteno7.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", str(ROOT / "include"), "-I", str(CSRC)]
UNITS = {
    "teno7_api.cu": [],
    "teno7_f64.cu": ["-fmad=false"],
    "teno7_f32.cu": [],
    "teno7_static.cu": [],
    "teno7_probe.cu": [],
    "teno7_slab2d_f64.cu": ["-fmad=false"],
    "teno7_slab2d_f32.cu": [],
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or Path(cand).exists()):
            return cand
    raise RuntimeError("nvcc not found")


def _sources_newer_than(target: Path) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    deps = list(CSRC.glob("*")) + list((ROOT / "include").glob("*.h")) + [Path(__file__)]
    return any(p.stat().st_mtime > t for p in deps if p.is_file())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None, checked: bool = False) -> Path:
    lib = LIB.with_name("libteno7_checked.so") if checked else LIB
    objdir = BUILD / "checked" if checked else BUILD
    if not force and not _sources_newer_than(lib):
        return lib
    objdir.mkdir(parents=True, exist_ok=True)
    nv = nvcc()
    extra = (extra or []) + (["-DT7_CHECKED=1"] if checked else [])

    def compile_unit(item):
        src, flags = item
        obj = objdir / (Path(src).stem + ".o")
        cmd = [nv, *ARCH, *COMMON, *flags, *extra, "-c", str(CSRC / src), "-o", str(obj)]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, flush=True)
        return obj

    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_unit, UNITS.items()))
    tmp = lib.with_suffix(f".{os.getpid()}.tmp")
    cmd = [nv, *ARCH, "-shared", "-o", str(tmp), *map(str, objs)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None,
                checked="--checked" in sys.argv))
