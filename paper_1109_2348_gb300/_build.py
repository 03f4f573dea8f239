"""In-tree build of the package's native libraries.

Two shared objects are built next to their sources:

* ``datagen/libbwtgen.so`` -- the seeded synthetic block sources (plain C).
* ``csrc/libbwt_gb300.so`` -- the C-ABI BWT library: host C++ plus CUDA
  kernels compiled for sm_103a only.

Translation units are compiled in parallel and linked with nvcc. A library is
rebuilt when any of its sources or headers is newer than the shared object.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
DATAGEN = PKG / "datagen"
INCLUDE = ROOT / "include"

GEN_SO = DATAGEN / "libbwtgen.so"
BWT_SO = CSRC / "libbwt_gb300.so"
# The same library built with -DBWT_DEBUG: bounds checks in the kernels record
# an internal error (BWT_EINTERNAL) instead of clamping silently. Loaded in
# place of the release library when the environment sets BWT_DEBUG=1.
BWT_DEBUG_SO = CSRC / "libbwt_gb300_debug.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbwt_gb300.so")


def _stale(target: Path, deps: list[Path]) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(d.stat().st_mtime > t for d in deps)


def _run(cmd: list[str]) -> None:
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + res.stdout + res.stderr)


def build_datagen(force: bool = False) -> Path:
    src = DATAGEN / "gen.c"
    if force or _stale(GEN_SO, [src]):
        tmp = GEN_SO.with_suffix(f".so.tmp{os.getpid()}")
        _run(["gcc", "-O2", "-std=c99", "-D_GNU_SOURCE", "-Wall", "-shared", "-fPIC", str(src),
              "-o", str(tmp), "-lpthread", "-lm"])
        os.replace(tmp, GEN_SO)
    return GEN_SO


def _cuda_sources() -> list[Path]:
    return sorted(CSRC.glob("*.cu")) + sorted(CSRC.glob("*.cpp"))


def _cuda_headers() -> list[Path]:
    return sorted(CSRC.glob("*.cuh")) + sorted(CSRC.glob("*.h")) + sorted(INCLUDE.glob("*.h"))


def build_bwt(force: bool = False, jobs: int | None = None, debug: bool = False) -> Path:
    srcs = _cuda_sources()
    hdrs = _cuda_headers()
    target = BWT_DEBUG_SO if debug else BWT_SO
    if not (force or _stale(target, srcs + hdrs)):
        return target
    nvcc = _nvcc()
    objdir = ROOT / "_build" / ("bwt_debug" if debug else "bwt")
    objdir.mkdir(parents=True, exist_ok=True)
    common = ["-std=c++17", "-O3", "-Xcompiler", "-fPIC", "-I", str(INCLUDE), "-I", str(CSRC)]
    if debug:
        common.append("-DBWT_DEBUG")

    def compile_one(src: Path) -> Path:
        obj = objdir / (src.name + ".o")
        if src.suffix == ".cu":
            cmd = [nvcc, *common, *ARCH, "-lineinfo", "-Xptxas", "-O3", "-c", str(src), "-o", str(obj)]
        else:
            cmd = [nvcc, *common, "-x", "c++", "-c", str(src), "-o", str(obj)]
        _run(cmd)
        return obj

    workers = jobs or min(len(srcs), max(1, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = target.with_suffix(f".so.tmp{os.getpid()}")
    _run([nvcc, "-shared", *ARCH, "-o", str(tmp), *map(str, objs), "-lcudart", "-lpthread"])
    os.replace(tmp, target)
    return target


def build_all(force: bool = False) -> None:
    build_datagen(force)
    build_bwt(force)
