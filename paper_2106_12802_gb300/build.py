"""Compile the CUDA library (libmrs.so) for sm_103a, in-tree.

Each translation unit is compiled by its own nvcc process (in parallel) and
linked into paper_2106_12802_gb300/_build/libmrs.so.  The renderer units are
compiled with --fmad=false (see pt.cu for why).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
SO = os.path.join(OUT, "libmrs.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
# translation unit -> extra flags
UNITS = {
    "bvh.cu": ["--fmad=false"],
    "pt.cu": ["--fmad=false"],
    "conv_tc.cu": [],
    "fuse.cu": [],
    "rdn.cu": [],
}


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmrs")
    return p


# the seeded scene generator shared with the test side (host C, compiled by
# gcc with -ffp-contract=off: the same scenes on every host)
SYNTH = os.path.join(os.path.dirname(HERE), "synth")
HOST_UNITS = {"scenegen.c": ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC"]}


def _sources():
    srcs = [os.path.join(CSRC, u) for u in UNITS]
    srcs += [os.path.join(SYNTH, u) for u in HOST_UNITS] + [os.path.join(SYNTH, "scenegen.h")]
    return srcs + [os.path.join(CSRC, f) for f in os.listdir(CSRC)]


def _stale() -> bool:
    if not os.path.exists(SO):
        return True
    t = os.path.getmtime(SO)
    inc = os.path.join(os.path.dirname(HERE), "include")
    deps = _sources() + [os.path.join(inc, f) for f in os.listdir(inc)]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return SO
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()

    def compile_unit(u):
        obj = os.path.join(OUT, u.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *COMMON, *UNITS[u], "-c", os.path.join(CSRC, u), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {u}:\n{r.stdout}\n{r.stderr}")
        return obj

    def compile_host(u):
        obj = os.path.join(OUT, u.replace(".c", ".host.o"))
        cmd = ["gcc", *HOST_UNITS[u], "-c", os.path.join(SYNTH, u), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"gcc failed on {u}:\n{r.stdout}\n{r.stderr}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS) + len(HOST_UNITS)) as ex:
        host = [ex.submit(compile_host, u) for u in HOST_UNITS]
        objs = list(ex.map(compile_unit, UNITS)) + [f.result() for f in host]
    tmp = SO + f".{os.getpid()}.tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force=True, verbose=True))
