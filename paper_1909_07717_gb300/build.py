"""Build libpps.so in-tree with nvcc for sm_103a (GB300).

    python -m paper_1909_07717_gb300.build          # rebuild if stale
    python -m paper_1909_07717_gb300.build --force

The library is compiled from csrc/*.cu (one nvcc process per translation
unit, run in parallel, then linked) against include/pps.h.  The CUDA runtime
is linked statically so the library only needs the driver at run time.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libpps.so")
OBJ_DIR = os.path.join(PKG, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
                     "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


# Sources compiled more than once, each time with its own defines: the
# batched-plan kernels, once per opponent-slot count.
VARIANTS = {"pps_batch_inst.cu": [("j%d" % j, ["-DPPS_BATCH_J=%d" % j])
                                  for j in (6, 8, 12, 16)]}


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _units():
    """(source, object name, extra flags) of every compilation."""
    out = []
    for src in _sources():
        base = os.path.basename(src)
        for tag, flags in VARIANTS.get(base, [("", [])]):
            name = base + ("." + tag if tag else "") + ".o"
            out.append((src, name, flags))
    return out


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(INCLUDE, "*.h")))


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit and link libpps.so; returns its path."""
    if not force and not stale():
        return LIB
    os.makedirs(OBJ_DIR, exist_ok=True)
    nvcc = _nvcc()
    units = _units()

    def compile_one(unit):
        src, name, extra = unit
        obj = os.path.join(OBJ_DIR, name)
        cmd = [nvcc] + NVCC_FLAGS + extra + ["-c", src, "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, len(units))) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
