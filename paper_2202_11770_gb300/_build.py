"""In-tree build of the native libraries of this package.

* ``libhlbgeom.so``  — seeded lattice generator (host C, gcc, OpenMP).
* ``libhemegb.so``   — the D3Q19 solver: sm_103a CUDA kernels behind a C ABI.

Both land in ``paper_2202_11770_gb300/_lib``.  Rebuilds happen only when a
source or header is newer than the library.  Nothing here is imported on the
solver's hot path; it only runs compilers.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
LIB = PKG / "_lib"
INCLUDE = ROOT / "include"

GEOM_SRC = [CSRC / "geometry.c"]
GEOM_LIB = LIB / "libhlbgeom.so"

CUDA_SRC = sorted(CSRC.glob("hlb_*.cu"))
CUDA_HDR = sorted(CSRC.glob("*.cuh")) + sorted(INCLUDE.glob("*.h"))
CUDA_LIB = LIB / "libhemegb.so"

ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhemegb")


def _stale(target: Path, deps) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(Path(d).stat().st_mtime > t for d in deps)


def _run(cmd, cwd=None):
    r = subprocess.run(cmd, cwd=cwd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout)
        raise RuntimeError(f"build step failed ({r.returncode}): {' '.join(map(str, cmd))}")
    return r.stdout


def build_geometry(force: bool = False) -> Path:
    LIB.mkdir(exist_ok=True)
    deps = GEOM_SRC + [INCLUDE / "hlb_geometry.h"]
    if force or _stale(GEOM_LIB, deps):
        tmp = GEOM_LIB.with_suffix(".so.tmp")
        _run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-Wall",
              "-o", str(tmp)] + [str(s) for s in GEOM_SRC] + ["-lm"])
        tmp.replace(GEOM_LIB)
    return GEOM_LIB


def build_cuda(force: bool = False, verbose_ptxas: bool = False) -> Path:
    LIB.mkdir(exist_ok=True)
    objdir = LIB / "obj"
    objdir.mkdir(exist_ok=True)
    deps = CUDA_SRC + CUDA_HDR
    if not (force or _stale(CUDA_LIB, deps)):
        return CUDA_LIB
    nvcc = _nvcc()
    common = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "--expt-relaxed-constexpr", f"-I{INCLUDE}", f"-I{CSRC}"]
    if verbose_ptxas:
        common += ["-Xptxas", "-v"]

    def one(src: Path):
        obj = objdir / (src.stem + ".o")
        if force or _stale(obj, [src] + CUDA_HDR):
            out = _run(common + ["-c", str(src), "-o", str(obj)])
            if verbose_ptxas:
                sys.stdout.write(out)
        return obj

    with ThreadPoolExecutor(max_workers=max(1, min(len(CUDA_SRC), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(one, CUDA_SRC))
    tmp = CUDA_LIB.with_suffix(".so.tmp")
    _run([nvcc, ARCH, "-shared", "-o", str(tmp)] + [str(o) for o in objs] + ["-lcudart"])
    tmp.replace(CUDA_LIB)
    return CUDA_LIB


def build_all(force: bool = False) -> None:
    build_geometry(force)
    build_cuda(force)


if __name__ == "__main__":
    build_all(force="--force" in sys.argv)
