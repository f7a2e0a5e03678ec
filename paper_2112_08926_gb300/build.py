"""Builds the CUDA library ``_build/liblbm.so`` for sm_103a.

Translation units: the C-ABI host code, the codec kernels, and the kernel
instantiation unit compiled once per (storage format, arithmetic) pair, all in
parallel.  Floating-point contraction is disabled on device (--fmad=false) and
host (-ffp-contract=off) so that the only fused multiply-adds are the explicit
fma() calls that the paper's operation order asks for.  The build is skipped
when the sources are unchanged (hash stamp).
"""
from __future__ import annotations

import hashlib
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "liblbm.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ARCH + [
    "-O3", "-std=c++17", "-lineinfo", "--fmad=false", "--expt-relaxed-constexpr",
    "-Xcompiler", "-fPIC,-ffp-contract=off", "-I" + INCLUDE, "-I" + CSRC,
]
# (storage id, arithmetic, velocity set) units: FP32 arithmetic for every
# format, FP64 arithmetic for FP64 and FP32 storage; one unit per velocity
# set keeps the units small enough to compile in parallel
UNITS = [(f, 0, v) for f in range(10) for v in range(3)] + [(f, 1, v) for f in (0, 1) for v in range(3)]


def _headers():
    names = sorted(n for n in os.listdir(CSRC) if n.endswith((".cuh", ".h")))
    return [os.path.join(CSRC, n) for n in names] + [os.path.join(INCLUDE, "lbm.h")]


def _hash(paths, extra: str) -> str:
    h = hashlib.sha256(extra.encode())
    for p in paths:
        with open(p, "rb") as fh:
            h.update(p.encode() + b"\0" + fh.read())
    return h.hexdigest()


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """Compile what changed and link; returns the library path."""
    os.makedirs(OUT, exist_ok=True)
    headers = _headers()
    jobs_list = [
        (os.path.join(CSRC, n), os.path.join(OUT, n[:-3] + ".o"), [])
        for n in sorted(os.listdir(CSRC)) if n.endswith(".cu") and n != "lbm_instantiate.cu"
    ]
    for fmt, arith, vs in UNITS:
        jobs_list.append((os.path.join(CSRC, "lbm_instantiate.cu"),
                          os.path.join(OUT, f"lbm_inst_{fmt}_{arith}_{vs}.o"),
                          [f"-DLBM_FMT={fmt}", f"-DLBM_ARITH={arith}", f"-DLBM_VELSET={vs}"]))

    def stamp_of(job):
        src, _, defs = job
        return _hash([src] + headers, " ".join(NVFLAGS + defs))

    def fresh(job):
        obj = job[1]
        if force or not os.path.exists(obj) or not os.path.exists(obj + ".stamp"):
            return False
        with open(obj + ".stamp") as fh:
            return fh.read().strip() == stamp_of(job)

    todo = [j for j in jobs_list if not fresh(j)]
    link_stamp = _hash([j[1] + ".stamp" for j in jobs_list if os.path.exists(j[1] + ".stamp")], "link")
    if not todo and os.path.exists(LIB) and os.path.exists(LIB + ".stamp"):
        with open(LIB + ".stamp") as fh:
            if fh.read().strip() == link_stamp:
                return LIB

    def compile_one(job):
        src, obj, defs = job
        cmd = ["nvcc"] + NVFLAGS + defs + ["-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        _run(cmd)
        with open(obj + ".stamp", "w") as fh:
            fh.write(stamp_of(job))
        return obj

    jobs = jobs or max(1, os.cpu_count() or 1)
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        list(ex.map(compile_one, todo))
    objs = [j[1] for j in jobs_list]
    tmp = LIB + f".tmp{os.getpid()}"
    _run(["nvcc"] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    with open(LIB + ".stamp", "w") as fh:
        fh.write(_hash([j[1] + ".stamp" for j in jobs_list], "link"))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
