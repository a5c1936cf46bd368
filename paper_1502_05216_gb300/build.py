"""Build libtf.so (the CUDA kernels and C ABI) in-tree for sm_103a.

    python -m paper_1502_05216_gb300.build

Compiles csrc/tf_capi.cu with nvcc for compute_103a/sm_103a into
paper_1502_05216_gb300/_lib/libtf.so.  The constant header csrc/tf_tables.h is
generated by csrc/gen_tables.py; the build refuses a stale header.
"""
from __future__ import annotations

import io
import os
import runpy
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "_lib")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")
LIB = os.path.join(LIBDIR, "libtf.so")
PROBE_LIB = os.path.join(LIBDIR, "libtfprobe.so")
SOURCES = ["tf_capi.cu", "tf_chain.cu"]
PROBE_SOURCES = ["tf_probe.cu"]
HEADERS = ["tf_core.cuh", "tf_core_f.cuh", "tf_eft.cuh", "tf_fixed.cuh", "tf_tables.h", os.path.join(INCLUDE, "tf.h"),
           os.path.join(INCLUDE, "tf_probe.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xptxas", "-O3", "--fmad=true",
           "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtf.so")


def tables_text() -> str:
    mod = runpy.run_path(os.path.join(CSRC, "gen_tables.py"), run_name="gen_tables")
    buf = io.StringIO()
    mod["main"](buf)
    return buf.getvalue()


def check_tables() -> None:
    with open(os.path.join(CSRC, "tf_tables.h")) as f:
        if f.read() != tables_text():
            raise RuntimeError("csrc/tf_tables.h is stale: run python csrc/gen_tables.py > csrc/tf_tables.h")


def _newest_input() -> float:
    paths = [os.path.join(CSRC, s) for s in SOURCES + PROBE_SOURCES] + [
        h if os.path.isabs(h) else os.path.join(CSRC, h) for h in HEADERS]
    return max(os.path.getmtime(p) for p in paths)


def _compile(out: str, sources, verbose: bool) -> subprocess.Popen:
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, *NVFLAGS, "-I", INCLUDE, "-shared", "-o", tmp,
           *[os.path.join(CSRC, s) for s in sources]]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
    p.tmp, p.out = tmp, out
    return p


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libtf.so (and the benchmark's libtfprobe.so) if missing or older
    than their sources; the two compile in parallel.  Returns libtf.so's path."""
    check_tables()
    os.makedirs(LIBDIR, exist_ok=True)
    newest = _newest_input()
    jobs = []
    for out, srcs in ((LIB, SOURCES), (PROBE_LIB, PROBE_SOURCES)):
        if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
            jobs.append(_compile(out, srcs, verbose))
    for p in jobs:
        _, err = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed ({p.returncode}):\n{err}")
        os.replace(p.tmp, p.out)
        if verbose:
            sys.stderr.write(err)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
