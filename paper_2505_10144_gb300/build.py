"""Builds libvrsplat.so in-tree for sm_103a (GB300) with nvcc: one object per
translation unit, compiled in parallel, then linked into a shared library."""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

HERE = Path(__file__).resolve().parent
CSRC = HERE / "csrc"
OUT = HERE / "lib"
LIB = OUT / "libvrsplat.so"
SOURCES = ["api.cu", "preprocess.cu", "sort.cu", "sort_noalloc.cu", "render.cu", "render_bwd.cu", "loss.cu", "net.cu", "net_train.cu", "peaks.cu", "probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _flags(extra=()):
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
            "-I", str(HERE.parent / "include"), *extra]


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> Path:
    OUT.mkdir(parents=True, exist_ok=True)
    srcs = [CSRC / s for s in SOURCES if (CSRC / s).exists()]
    deps = srcs + list(CSRC.glob("*.cuh")) + [HERE.parent / "include" / "vrsplat.h"]
    newest = max(p.stat().st_mtime for p in deps)
    if not force and LIB.exists() and LIB.stat().st_mtime >= newest:
        return LIB
    objs = []

    def compile_one(src: Path):
        obj = OUT / (src.stem + ".o")
        cmd = [nvcc(), "-c", str(src), "-o", str(obj), *_flags(extra_flags)]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src.name}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = OUT / f"libvrsplat.tmp{os.getpid()}.so"
    cmd = [nvcc(), "-shared", *ARCH, "-o", str(tmp), *map(str, objs)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
