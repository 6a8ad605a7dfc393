"""Build the CUDA library ``libcales.so`` in-tree for sm_103a (no cmake).

Each ``csrc/*.cu`` is compiled to an object in parallel, then linked with
the static CUDA runtime into ``_build/libcales.so``.  Objects are rebuilt only
when a source or header is newer.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
OUT = PKG / "_build"
LIB = OUT / "libcales.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         f"-I{ROOT / 'include'}", f"-I{CSRC}"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found")


def _newest_header() -> float:
    hs = list(CSRC.glob("*.cuh")) + list(CSRC.glob("*.h")) + list((ROOT / "include").glob("*.h"))
    return max(h.stat().st_mtime for h in hs)


def _compile(nvcc: str, src: Path, obj: Path, extra) -> tuple[Path, str]:
    cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", str(src), "-o", str(obj)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src.name}:\n{r.stderr}")
    return obj, r.stderr


def build(verbose: bool = False, extra_flags=()) -> Path:
    """Compile and link; returns the path of the shared library."""
    OUT.mkdir(exist_ok=True)
    nvcc = _nvcc()
    srcs = sorted(CSRC.glob("*.cu"))
    hdr_t = _newest_header()
    jobs = []
    for s in srcs:
        o = OUT / (s.stem + ".o")
        if not o.exists() or o.stat().st_mtime < max(s.stat().st_mtime, hdr_t) or extra_flags:
            jobs.append((s, o))
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for obj, err in ex.map(lambda j: _compile(nvcc, j[0], j[1], list(extra_flags)), jobs):
                if verbose and err.strip():
                    print(err, file=sys.stderr)
    objs = [OUT / (s.stem + ".o") for s in srcs]
    if jobs or not LIB.exists() or LIB.stat().st_mtime < max(o.stat().st_mtime for o in objs):
        tmp = OUT / "libcales.so.tmp"
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", str(tmp), *map(str, objs)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
