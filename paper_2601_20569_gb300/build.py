"""In-tree build of libtpc.so for sm_103a (nvcc, no cmake).

The sector/fit kernels are compiled twice: ``--fmad=false`` into namespace
``tpc::strict`` (bit-identical to a strict CPU evaluation) and with FMA
contraction and hardware reciprocals (``TPC_FAST_ARITH``) into ``tpc::fast``.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libtpc.so")
BUILD_DIR = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + CSRC,
                 "-I" + INCLUDE]
KERNEL_TUS = ["tpc_sector.cu", "tpc_fit.cu", "tpc_removal.cu"]  # compiled when present
HOST_TUS = ["tpc_api.cu", "tpc_noalloc.cu", "tpc_peak.cu"]


def _sources():
    out = []
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".cu", ".cuh", ".h")):
                out.append(os.path.join(d, f))
    return out


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    srcs = _sources()
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= t for s in srcs):
            return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    objs = []
    for tu in KERNEL_TUS:
        if not os.path.exists(os.path.join(CSRC, tu)):
            continue
        base = os.path.splitext(tu)[0]
        for ns, flags in (("strict", ["--fmad=false"]), ("fast", ["--fmad=true", "-DTPC_FAST_ARITH"])):
            obj = os.path.join(BUILD_DIR, f"{base}_{ns}.o")
            cmd = [nvcc] + COMMON + flags + [f"-DTPC_NS={ns}", "-c", os.path.join(CSRC, tu),
                                             "-o", obj]
            jobs.append(cmd)
            objs.append(obj)
    for tu in HOST_TUS:
        obj = os.path.join(BUILD_DIR, os.path.splitext(tu)[0] + ".o")
        jobs.append([nvcc] + COMMON + ["-c", os.path.join(CSRC, tu), "-o", obj])
        objs.append(obj)
    procs = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for cmd in jobs]
    failed = []
    for cmd, p in zip(jobs, procs):
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
