"""Build libsph for sm_103a in-tree: every .cu under csrc/ compiled in parallel with nvcc, then linked into
paper_2502_16517_gb300/_build/libsph.so (the checked build, -DSPH_CHECKED: _build_checked/libsph.so).  Rebuilds
only what changed (source or header newer than object)."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libsph.so")
# the checked build (-DSPH_CHECKED: index checks that set SPH_DEV_BOUNDS instead of accessing out of range)
OUT_CHECKED = os.path.join(HERE, "_build_checked")
INCLUDE = os.path.join(ROOT, "include")

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, extra, out=OUT):
    obj = os.path.join(out, os.path.basename(src)[:-3] + ".o")
    if _stale(obj, [src] + _headers()):
        cmd = [NVCC] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if r.stderr.strip():
            sys.stderr.write(r.stderr)
    return obj


def build(verbose_ptxas: bool = False, checked: bool = False) -> str:
    """Compile and link libsph (checked: the -DSPH_CHECKED build into _build_checked/); returns the library path."""
    out = OUT_CHECKED if checked else OUT
    lib_path = os.path.join(out, "libsph.so")
    os.makedirs(out, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    extra = (["-Xptxas", "-v"] if verbose_ptxas else []) + (["-DSPH_CHECKED"] if checked else [])
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, out), srcs))
    if _stale(lib_path, objs):
        tmp = lib_path + f".tmp{os.getpid()}"
        cmd = [NVCC] + ARCH + ["-shared", "-cudart=static", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(verbose_ptxas="-v" in sys.argv, checked="--checked" in sys.argv))
