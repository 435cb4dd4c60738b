"""Build libuspg (all CUDA sources, sm_103a) in-tree.

``python -m paper_2208_12964_gb300.build`` compiles each translation unit with
nvcc in parallel and links ``_lib/libuspg.so``.  The generator is compiled
with ``-fmad=false`` so its FP64 crossings are formed with separately rounded
operations; so are the segment store (the same crossings) and the resample,
whose pixel-centre classification follows the same rule.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libuspg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3", "--expt-relaxed-constexpr"]
UNITS = {
    "api.cu": [],
    "generator.cu": ["-fmad=false"],
    "mart.cu": [],
    "resample.cu": ["-fmad=false"],
    "batch.cu": [],
    "server.cu": [],
    "segments.cu": ["-fmad=false"],
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    return [u for u in UNITS if os.path.exists(os.path.join(SRC, u))]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(SRC, f) for f in os.listdir(SRC)] + [os.path.join(HERE, "..", "include", "uspg.h")]
    return any(os.path.getmtime(p) > t for p in deps if os.path.exists(p))


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()
    objs = []

    def compile_one(unit):
        obj = os.path.join(OUT, unit.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *COMMON, *UNITS[unit], "-c", os.path.join(SRC, unit), "-o", obj]
        if ptxas_v:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {unit}:\n{r.stderr}")
        return obj, r.stderr

    units = _sources()
    with cf.ThreadPoolExecutor(max_workers=len(units)) as ex:
        for obj, log in ex.map(compile_one, units):
            objs.append(obj)
            if verbose and log:
                print(log, file=sys.stderr)
    tmp = LIB + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stderr)
    os.replace(tmp, LIB)
    for o in objs:
        os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="-v" in sys.argv))
