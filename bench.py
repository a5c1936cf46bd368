#!/usr/bin/env python
"""Throughput of the double-twofold exp/log kernels on one GB300 (or N, weak scaling).

One step = one pass of the whole path over its synthetic batch: texp, texpm1,
tlog, tlog1p, tadd and tmul, each over n = 2^26 double twofolds (SoA x0, x1 ->
z0, z1; 1 GiB in + 1 GiB out per unary function), every input resident in HBM
before the timed region.  Inputs are 512 MiB per array, larger than L2, so no
flush is needed between iterations.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  ``value`` is the metric, texp/tlog Gelem/s at
n = 2^26: 2n elements (n of texp, n of tlog) per rank over the two kernels'
time, CUDA events on the launching stream inside the timed step, summed over
ranks; the whole six-function step is reported under ``step``.  ``e2e`` is the
same metric through the host-array API (the kernels read and write pinned host
memory, so every byte crosses the host link inside the timed region);
``roofline`` is for the metric's dominant kernel; ``cpu_baseline`` is the CPU
oracle timed on this host's cores on a bounded sample of texp and tlog.

``--impl reference`` times the CPU oracle (binary128, all host cores) as the
reference arm on bounded samples of the same workload.

``--ncu-summary CSV`` prints the per-kernel count table (markdown) of an ncu
``--csv`` metric capture of this benchmark, stamped with the hash of the
kernel sources; the benchmark reads its instruction counts and DRAM traffic
from that table (profiles/pipe_counts_unary_v2_binary_v2_n2p24.txt) and drops
the traffic when the sources have changed since.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FUNCS = ("texp", "texpm1", "tlog", "tlog1p", "tadd", "tmul")
METRIC_FUNCS = ("texp", "tlog")
METRIC = "double-twofold texp/tlog Gelem/s at n=2^26 and % of FP64/HBM roofline"
WORKLOAD = ("texp, texpm1, tlog, tlog1p (+ tadd, tmul) over double twofolds, n=2^26 each: exp/expm1 "
            "args random sign |x0| log-uniform in [2^-40, 708]; log x0 log-uniform in [2^-1020, 2^1020]; "
            "log1p half |x0| log-uniform in [2^-40, 2^-10), half -1+2^-30 .. 2^100; x1 = x0*u*2^-53")

# Per-element instruction counts and DRAM traffic of each kernel on its
# workload come from one ncu metric capture of this benchmark, summarised in
# COUNTS_FILE (written by --ncu-summary): integer-ALU-pipe, FP64-pipe and
# FMA-pipe thread instructions per element (warp instructions x 32 / n; every
# warp of these kernels runs all 32 lanes) and dram__bytes_read + write per
# launch.  The file carries the hash of the kernel sources it was taken on.
COUNTS_FILE = os.path.join(ROOT, "profiles", "pipe_counts_unary_v2_binary_v2_n2p24.txt")
KERNEL_SOURCES = ("tf_capi.cu", "tf_core.cuh", "tf_core_f.cuh", "tf_fixed.cuh", "tf_eft.cuh", "tf_tables.h")
NCU_METRICS = ("gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum,sm__inst_executed_pipe_alu.sum,"
               "sm__inst_executed_pipe_fp64.sum,sm__inst_executed_pipe_fma.sum,smsp__inst_executed.sum,"
               "sm__inst_executed_pipe_alu.avg.pct_of_peak_sustained_active,"
               "sm__inst_executed_pipe_fp64.avg.pct_of_peak_sustained_active")
# HBM bytes per element: SoA doubles in + out.
BYTES_PER_ELEM = {"texp": 32, "texpm1": 32, "tlog": 32, "tlog1p": 32, "tadd": 48, "tmul": 48}
HBM_PEAK_FALLBACK = 6804.4   # GB/s, a measured copy on the GB300s, when MEASURED_PEAKS.json is absent
SM_MAX_MHZ = 2070.0          # used when no clock sample exists


def hbm_peak():
    """(GB/s, source) of the HBM roof: MEASURED_PEAKS.json's measured copy
    bandwidth when the file is present, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured: MEASURED_PEAKS.json hbm_gbs (STREAM-style copy)"
    except (OSError, KeyError, ValueError):
        return HBM_PEAK_FALLBACK, "fallback: an earlier measured copy on a GB300"


def kernel_source_hash() -> str:
    """Hash of the elementwise kernels' sources with comments and blank space
    removed (a comment edit does not stale the counts; a code edit does)."""
    import hashlib
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1502_05216_gb300", "csrc")
    for name in KERNEL_SOURCES:
        text = open(os.path.join(csrc, name)).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(name.encode())
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def load_counts(path: str = COUNTS_FILE):
    """{kernel: {alu, fp64, fma, inst, traffic, n}} and the source hash from the
    count table; ({}, None) when the file is missing."""
    out, stamp = {}, None
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return out, stamp
    for ln in lines:
        if ln.startswith("kernel source hash:"):
            stamp = ln.split(":", 1)[1].strip().strip("`")
        c = [x.strip() for x in ln.strip().strip("|").split("|")]
        if len(c) == 4 and c[0] in FUNCS and c[0] in out:  # the full-size traffic table
            try:
                out[c[0]]["traffic_n"] = int(c[1])
                out[c[0]]["traffic"] = float(c[2])
            except ValueError:
                pass
        if len(c) == 9 and c[0] in FUNCS + tuple(f + "f" for f in FUNCS[:4]):
            try:
                out[c[0]] = {"n": int(c[1]), "alu": float(c[3]), "fp64": float(c[4]), "fma": float(c[5]),
                             "inst": float(c[6]), "traffic_per_elem": float(c[7])}
            except ValueError:
                continue
    return out, stamp


def ncu_summary(csv_path: str) -> str:
    """Markdown count table from an ncu --csv metric capture of this benchmark:
    the first captured launch of each kernel, in launch order."""
    import csv
    import re
    rows, order = {}, []
    with open(csv_path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    names = {"OpExp": "texp", "OpExpm1": "texpm1", "OpLog": "tlog", "OpLog1p": "tlog1p", "OpAdd": "tadd",
             "OpMul": "tmul", "OpExpF": "texpf", "OpExpm1F": "texpm1f", "OpLogF": "tlogf", "OpLog1pF": "tlog1pf"}
    first = {}
    for r in csv.DictReader(lines):
        op = re.search(r"\b(Op[A-Za-z0-9]+)\b", r["Kernel Name"])
        nm = names.get(op.group(1) if op else "")
        if nm is None:
            continue
        if nm not in first:
            first[nm] = r["ID"]
            order.append(nm)
            rows[nm] = {}
        if r["ID"] != first[nm]:
            continue
        v = r["Metric Value"].replace(",", "")
        rows[nm][r["Metric Name"]] = (float(v), r["Metric Unit"])
    n = N_FOR_SUMMARY[0]
    if order and "sm__inst_executed_pipe_alu.sum" not in rows[order[0]]:
        # a DRAM-traffic capture alone (the full-size launches, one pass)
        out = ["| kernel | n | DRAM bytes per launch (read + write) | ms (serialised) |", "|---|---|---|---|"]
        for nm in order:
            m = rows[nm]
            b = sum(m[k][0] * {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}.get(m[k][1], 1.0)
                    for k in ("dram__bytes_read.sum", "dram__bytes_write.sum"))
            t = m["gpu__time_duration.sum"]
            ms = t[0] * {"nsecond": 1e-6, "ns": 1e-6, "usecond": 1e-3, "us": 1e-3, "msecond": 1.0}.get(t[1], 1.0)
            out.append(f"| {nm} | {n} | {b:.0f} | {ms:.4f} |")
        return "\n".join(out)
    out = [f"kernel source hash: `{kernel_source_hash()}`", "",
           "| kernel | n | ms (serialised) | ALU inst/elem | FP64 inst/elem | FMA inst/elem | all inst/elem | "
           "DRAM bytes/elem | ALU %, FP64 % of peak (active) |", "|---|---|---|---|---|---|---|---|---|"]
    scale = {"nsecond": 1e-6, "ns": 1e-6, "usecond": 1e-3, "us": 1e-3, "msecond": 1.0, "ms": 1.0,
             "byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}
    for nm in order:
        m = rows[nm]
        val = lambda k: m[k][0] * scale.get(m[k][1], 1.0)  # noqa: E731
        per = lambda k: m[k][0] * 32 / n  # noqa: E731
        byts = val("dram__bytes_read.sum") + val("dram__bytes_write.sum")
        out.append(f"| {nm} | {n} | {val('gpu__time_duration.sum'):.4f} | {per('sm__inst_executed_pipe_alu.sum'):.1f} | "
                   f"{per('sm__inst_executed_pipe_fp64.sum'):.1f} | {per('sm__inst_executed_pipe_fma.sum'):.1f} | "
                   f"{per('smsp__inst_executed.sum'):.1f} | {byts / n:.2f} | "
                   f"{m['sm__inst_executed_pipe_alu.avg.pct_of_peak_sustained_active'][0]:.1f}, "
                   f"{m['sm__inst_executed_pipe_fp64.avg.pct_of_peak_sustained_active'][0]:.1f} |")
    return "\n".join(out)


N_FOR_SUMMARY = [1 << 24]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--log2n", type=int, default=26)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-chains", action="store_true", help="skip the batched-chains measurement")
    ap.add_argument("--no-tier", action="store_true", help="skip the float/double precision-tier measurement")
    ap.add_argument("--no-coupled", action="store_true",
                    help="skip the variant entry points (pexp ... tlog1pp, texp_tables)")
    ap.add_argument("--no-sweep", action="store_true", help="skip the size sweep")
    ap.add_argument("--no-hard", action="store_true", help="skip the timed hard-case sets")
    ap.add_argument("--tier-log2n", type=int, default=28)
    ap.add_argument("--sweep-max", type=int, default=30, choices=(26, 28, 30),
                    help="largest size of the sweep (2^28 and 2^30 draw their own inputs: 2 / 8 GiB per array)")
    ap.add_argument("--ncu-summary", default=None, metavar="CSV",
                    help="print the count table of an ncu --csv capture of this benchmark and exit")
    ap.add_argument("--ncu-n", type=int, default=1 << 24, help="n of the captured launches (--ncu-summary)")
    ap.add_argument("--funcs", default=",".join(FUNCS),
                    help="comma-separated subset (for profiling a single kernel)")
    return ap.parse_args()


def rank_start(rank: int, n: int) -> int:
    """First element index of a rank's shard: weak scaling, each rank evaluates
    its own n consecutive elements of every workload (elements are independent,
    so no data-path collective is needed)."""
    return rank * n


def reduce_max(value: float, world: int, device) -> float:
    """The maximum of a per-rank value over all ranks (timings: the job takes as
    long as its slowest rank).  One all_reduce on the initialised process group."""
    if world <= 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------

class Clocks:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.p = None
        self.path = os.path.join(tempfile.gettempdir(), f"tf_bench_clocks_{os.getpid()}.csv")
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
            if gpu_id:
                cmd += ["-i", gpu_id]
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.6)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.p.terminate()
        self.p.wait(timeout=10)
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ("active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            c = [x.strip() for x in line.split(",")]
            if len(c) < 10:
                continue
            try:
                sm.append(float(c[2]))
                mx.append(float(c[3]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], c[6:10]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------------

def oracle_rate(budget_s: float, per_func_cap: int = 1 << 26, funcs=METRIC_FUNCS):
    """Time the CPU oracle on a bounded sample of the metric's functions'
    workloads (texp and tlog), sized from a probe to take about budget_s:
    elements/s over all host threads, plus the sample description."""
    import oracle
    from paper_1502_05216_gb300 import inputs as I
    lib = oracle.load()
    probe = 1 << 16
    pargs = {f: I.workload(f, probe) for f in funcs}
    for f in funcs:  # warm-up: library load and thread start
        oracle.evaluate(f, *pargs[f], lib=lib)
    t0 = time.perf_counter()
    for f in funcs:
        oracle.evaluate(f, *pargs[f], lib=lib)
    rate0 = len(funcs) * probe / (time.perf_counter() - t0)
    m = int(min(per_func_cap, max(probe, budget_s * rate0 / len(funcs))))
    args = {f: I.workload(f, m, start=1 << 30) for f in funcs}
    t0 = time.perf_counter()
    for f in funcs:
        oracle.evaluate(f, *args[f], lib=lib)
    dt = time.perf_counter() - t0
    sample = f"{m} elements of each of {', '.join(funcs)}'s workloads (indices from 2^30), {dt:.1f} s"
    return len(funcs) * m / dt, oracle.threads(), sample, m, dt


def oracle_single_core(m: int, funcs=METRIC_FUNCS):
    """The oracle on one host thread: m elements of each function's workload."""
    import oracle
    from paper_1502_05216_gb300 import inputs as I
    lib = oracle.load()
    t = oracle.threads()
    args = {f: I.workload(f, m, start=1 << 32) for f in funcs}
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        for f in funcs:
            oracle.evaluate(f, *args[f], lib=lib)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(t)
    return {"value": len(funcs) * m / dt / 1e9, "unit": "Gelem/s", "cores": 1,
            "sample": f"{m} elements of each of {', '.join(funcs)}'s workloads (indices from 2^32), {dt:.1f} s"}


def reference_arm(a, world, rank):
    if rank != 0:
        return
    import oracle
    from paper_1502_05216_gb300 import inputs as I
    lib = oracle.load()
    budget = max(1.0, min(8.0, 150.0 / (a.steps + a.warmup)))
    _, cores, _, m, _ = oracle_rate(budget * 0.5)
    args = {f: I.workload(f, m, start=1 << 31) for f in METRIC_FUNCS}
    for _ in range(a.warmup):
        for f in METRIC_FUNCS:
            oracle.evaluate(f, *args[f], lib=lib)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        for f in METRIC_FUNCS:
            oracle.evaluate(f, *args[f], lib=lib)
    dt = (time.perf_counter() - t0) / a.steps
    v = len(METRIC_FUNCS) * m / dt / 1e9
    sample = f"each step: {m} elements of each of texp's and tlog's workloads (bounded sample of n=2^26)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "Gelem/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f128", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": 1 << a.log2n, "functions": list(METRIC_FUNCS)},
        "cpu_baseline": {"value": v, "unit": "Gelem/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "Gelem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------

def fp64_peak(dev):
    """Measured FP64 pipe rate (DFMA thread-instructions/s) of this GPU, from the
    calibration kernel; best of 5."""
    import ctypes
    import torch
    from paper_1502_05216_gb300 import build
    lib = ctypes.CDLL(build.PROBE_LIB)
    lib.tfp_dfma.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads, iters = sms * 8, 256, 6000
    out = torch.empty(blocks * threads, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev)
    best = 0.0
    for i in range(7):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        rc = lib.tfp_dfma(out.data_ptr(), blocks, threads, iters, st.cuda_stream)
        e1.record(st)
        e1.synchronize()
        if rc != 0:
            raise RuntimeError(f"tfp_dfma failed ({rc})")
        if i >= 2:
            best = max(best, blocks * threads * iters * 8 / (e0.elapsed_time(e1) * 1e-3))
    return best, sms


def alu_peak(dev, mode=0):
    """Measured integer-ALU pipe rate (thread-instructions/s) of this GPU, from
    the calibration kernel (16 instructions per iteration and thread; mode 0:
    rotates and three-input xors, which only the ALU pipe executes); best of 5."""
    import ctypes
    import torch
    from paper_1502_05216_gb300 import build
    lib = ctypes.CDLL(build.PROBE_LIB)
    lib.tfp_alu.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                            ctypes.c_void_p]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads, iters = sms * 8, 256, 20000
    out = torch.empty(blocks * threads, dtype=torch.int32, device=dev)
    st = torch.cuda.current_stream(dev)
    best = 0.0
    for i in range(7):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        rc = lib.tfp_alu(out.data_ptr(), blocks, threads, iters, mode, st.cuda_stream)
        e1.record(st)
        e1.synchronize()
        if rc != 0:
            raise RuntimeError(f"tfp_alu failed ({rc})")
        if i >= 2:
            best = max(best, blocks * threads * iters * 16 / (e0.elapsed_time(e1) * 1e-3))
    return best


CHAIN_WORKLOAD = ("65,536 independent chains, lengths geometric (mean 256, cap 4096), ops uniform over "
                  "{tadd, tmul, texp, tlog} (infeasible draws redrawn), states in [2^-20, 2^20], double twofolds")


def host_link(dev, nbytes=1 << 30, reps=3):
    """The GPU's host link, measured: copy-engine copies between pinned host
    memory and the device, host to device, device to host, and both at once on
    two streams (GB/s, median of `reps`).  The end-to-end number moves its
    bytes over this link; SM-driven loads and stores of pinned memory (the
    zero-copy path) measured the same rates on GB300."""
    import torch
    h1 = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    h2 = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d1 = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    d2 = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def rate(h2d, d2h):
        ts = []
        for _ in range(reps + 1):
            torch.cuda.synchronize(dev)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(s1)
            s2.wait_event(e0)
            if h2d:
                with torch.cuda.stream(s1):
                    d1.copy_(h1, non_blocking=True)
            if d2h:
                with torch.cuda.stream(s2):
                    h2.copy_(d2, non_blocking=True)
            e2.record(s2)
            s1.wait_event(e2)
            e1.record(s1)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return (h2d + d2h) * nbytes / (statistics.median(ts[1:]) * 1e-3) / 1e9

    out = {"h2d_gbs": rate(1, 0), "d2h_gbs": rate(0, 1), "both_gbs": rate(1, 1)}
    del h1, h2, d1, d2
    return out


def chains_bench(dev, rank=0, world=1):
    """The batched-chains workload: one fused persistent launch (autotuned chains
    per warp, block size and grid) against one launch per step and op kind, each
    captured in a CUDA graph together with the reset of the chain states; median
    of 5 replays.  With N ranks the 65,536 chains are sharded by chain id
    (chains.shard, strong scaling: the batch is fixed) and the times are the
    slowest rank's."""
    from paper_1502_05216_gb300 import chains, inputs as I
    full = I.chains(65536)
    batch = chains.shard(full, rank, world) if world > 1 else full
    cb = chains.ChainBatch(batch, dev)
    cfg, table = cb.tune()
    fused = reduce_max(cb.time_graph(cb.graph("fused", cfg["threads"], cfg["blocks"], cfg["group"]), 5), world, dev)
    per_op = reduce_max(cb.time_graph(cb.graph("per_op"), 5), world, dev)
    ops = int(full["step_base"][-1])
    best = sorted(table, key=lambda r: r["ms"])
    # the headline figures last, so that the end of the JSON line carries them
    return {"workload": CHAIN_WORKLOAD, "ops": ops, "mix": dict(zip(("tadd", "tmul", "texp", "tlog"),
                                                                    full["mix"].tolist())),
            "max_len": int(full["max_len"]), "per_op_launches": cb.per_op_launches, "ranks": world,
            "scaling": "strong (chains sharded by chain id)" if world > 1 else None,
            "tuning": {"tried": len(table), "cols": ["group", "threads", "blocks", "ms"],
                       "fastest": [[r["group"], r["threads"], r["blocks"], round(r["ms"], 3)] for r in best[:4]],
                       "slowest_ms": round(best[-1]["ms"], 3)},
            "fused_config": cfg, "fused_gops_s": ops / (fused * 1e-3) / 1e9,
            "fused_ms": fused, "per_op_ms": per_op, "speedup": per_op / fused}


def _time_launches(fn, reps=5, warm=3):
    """Median ms of one call of fn() (CUDA events on the current stream)."""
    import torch
    st = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def coupled_variants(dev, dargs, n, reps=5):
    """Kernel time of the coupled-result (pexp, pexpm1, plog, plog1p) and
    coupled-argument (texpp, texpm1p, tlogp, tlog1pp) entry points, and of
    texp through the paper's own table reduction (texp_tables), on the same
    inputs as their twofold functions, CUDA events, mean of ``reps`` launches
    after one warm-up."""
    import torch
    from paper_1502_05216_gb300 import tf
    st = torch.cuda.current_stream(dev)
    z0 = torch.empty(n, dtype=torch.float64, device=dev)
    z1 = torch.empty_like(z0)
    out = {}
    for name, fn in tf.FUNCS_C.items():
        base = tf.BASE_OF[name]
        res = {}
        for key, f in ((name, fn), (base, tf.FUNCS[base])):
            f(*dargs[base], out=(z0, z1), stream=st)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                f(*dargs[base], out=(z0, z1), stream=st)
            e1.record(st)
            e1.synchronize()
            res[key] = e0.elapsed_time(e1) / reps
        out[name] = {"ms": res[name], "gelem_s": n / (res[name] * 1e-3) / 1e9, "twofold": base,
                     "twofold_ms": res[base], "time_ratio": res[name] / res[base]}
    # A/B variants: texp through the paper's own table reduction, the logs with
    # their Newton step in binary64 (same inputs as the default kernels)
    what = {"texp_tables": "the paper's own reduction x = 2m + n/256 + y (K = 8, L = 1), tables e^(2m), e^(n/256)",
            "tlog_newton_fp64": "tlog with the Newton step u = t + S + tS in binary64 (S = e^-R - 1 as a pair)",
            "tlog1p_newton_fp64": "tlog1p with the Newton step u = t + S + tS in binary64"}
    for var, (fv, base) in tf.VARIANT_FUNCS.items():
        res = {}
        for key, f in ((var, fv), (base, tf.FUNCS[base])):
            f(*dargs[base], out=(z0, z1), stream=st)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(reps):
                f(*dargs[base], out=(z0, z1), stream=st)
            e1.record(st)
            e1.synchronize()
            res[key] = e0.elapsed_time(e1) / reps
        out[var] = {"ms": res[var], "gelem_s": n / (res[var] * 1e-3) / 1e9, "twofold": base,
                    "twofold_ms": res[base], "time_ratio": res[var] / res[base], "what": what[var]}
    return out


def precision_tier(dev, log2n):
    """texp and tlog over float twofolds (float-float on the FP32 pipes) and
    over double twofolds (the FP64 + integer path) on the same x0 values, n =
    2^log2n each; Gelem/s and HBM GB/s of each kernel."""
    import torch
    from paper_1502_05216_gb300 import inputs as I, tf
    n = 1 << log2n
    out = {"n": n, "workload": "texp x0 uniform in [-88, 88]; tlog x0 log-uniform in [2^-126, 2^127]; "
                               "x1 = x0 u 2^-24 (float) or 2^-53 (double), same x0 and u"}
    for func in ("texp", "tlog"):
        x0f, x1f = I.workload_f32_big(func, n)
        x0d, x1d = I.double_of_f32(func, x0f)
        res = {}
        for dt, (a0, a1), fn, bpe in (("f32", (x0f, x1f), tf.FUNCS_F[func], 16),
                                      ("f64", (x0d, x1d), tf.FUNCS[func], 32)):
            d0, d1 = torch.from_numpy(a0).to(dev), torch.from_numpy(a1).to(dev)
            o = (torch.empty_like(d0), torch.empty_like(d0))
            ms = _time_launches(lambda: fn(d0, d1, out=o))
            res[dt] = {"ms": ms, "gelem_s": n / (ms * 1e-3) / 1e9, "hbm_gbs": bpe * n / (ms * 1e-3) / 1e9,
                       "hbm_frac": bpe * n / (ms * 1e-3) / 1e9 / hbm_peak()[0]}
            del d0, d1, o
        res["f32_over_f64"] = res["f64"]["ms"] / res["f32"]["ms"]
        out[func] = res
        del x0f, x1f, x0d, x1d
    torch.cuda.empty_cache()
    return out


def size_sweep(dev, dargs, max_lg=26):
    """texp and tlog (double) at n = 2^10 .. 2^26 (prefixes of the resident
    2^26 inputs), and up to 2^max_lg with inputs drawn for the purpose; up to
    2^18 the timed unit is a CUDA graph of 64 launches, so the host launch cost
    is out of the per-launch time."""
    import torch
    from paper_1502_05216_gb300 import inputs as I, tf
    out = {}
    for func in ("texp", "tlog"):
        rows = []
        for lg in (10, 14, 18, 22, 26, 28, 30):
            if lg > max_lg:
                break
            n = 1 << lg
            if lg <= 26:
                a0, a1 = dargs[func][0][:n], dargs[func][1][:n]
            else:
                a0, a1 = (torch.from_numpy(x).to(dev) for x in I.workload(func, n))
            o = (torch.empty(n, dtype=torch.float64, device=dev), torch.empty(n, dtype=torch.float64, device=dev))
            if lg <= 18:
                reps = 64
                s = torch.cuda.Stream(dev)
                s.wait_stream(torch.cuda.current_stream(dev))
                g = torch.cuda.CUDAGraph()
                with torch.cuda.stream(s):
                    tf.FUNCS[func](a0, a1, out=o, stream=s)
                    s.synchronize()
                    with torch.cuda.graph(g, stream=s):
                        for _ in range(reps):
                            tf.FUNCS[func](a0, a1, out=o, stream=s)
                torch.cuda.current_stream(dev).wait_stream(s)
                ms = _time_launches(g.replay) / reps
            else:
                ms = _time_launches(lambda: tf.FUNCS[func](a0, a1, out=o))
            rows.append({"n": n, "us": ms * 1e3, "gelem_s": n / (ms * 1e-3) / 1e9, "graph": lg <= 18})
            del o
            if lg > 26:
                del a0, a1
                torch.cuda.empty_cache()
        out[func] = rows
    return out


def hard_case_timing(dev, dargs, log2n=24):
    """texp and tlog (double) over the 2^24 hard-case set of the parity tests
    (thresholds of overflow, underflow and subnormal results, tiny and huge
    arguments, log near 1, subnormal y0, x1 = 0, half-ulp x1, IEEE specials)
    against the first 2^24 elements of their workloads: the cost of the lanes
    that leave the straight-line code (each warp votes once and runs its rare
    lanes' branch).  CUDA events, median of 5 launches."""
    import torch
    from paper_1502_05216_gb300 import inputs as I, tf
    n = 1 << log2n
    out = {"n": n}
    for func in METRIC_FUNCS:
        h = [torch.from_numpy(x).to(dev) for x in I.hard_cases(func, n, seed=29)]
        w = [x[:n] for x in dargs[func]]
        o = (torch.empty(n, dtype=torch.float64, device=dev), torch.empty(n, dtype=torch.float64, device=dev))
        ms_h = _time_launches(lambda: tf.FUNCS[func](*h, out=o))
        ms_w = _time_launches(lambda: tf.FUNCS[func](*w, out=o))
        out[func] = {"hard_ms": ms_h, "workload_ms": ms_w, "hard_gelem_s": n / (ms_h * 1e-3) / 1e9,
                     "workload_gelem_s": n / (ms_w * 1e-3) / 1e9, "time_ratio": ms_h / ms_w}
        del h, o
    torch.cuda.empty_cache()
    return out


def ours(a, world, rank, local):
    global FUNCS
    FUNCS = tuple(f for f in a.funcs.split(",") if f)
    import torch
    from paper_1502_05216_gb300 import build, inputs as I, tf
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    build.build()
    tf.load()
    n = 1 << a.log2n
    start = rank_start(rank, n)

    host = {f: I.workload(f, n, start=start) for f in FUNCS}
    dargs = {f: [torch.from_numpy(x).to(dev) for x in host[f]] for f in FUNCS}
    z0 = torch.empty(n, dtype=torch.float64, device=dev)
    z1 = torch.empty(n, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    def step(evs=None):
        for f in FUNCS:
            if evs is not None:
                evs[f][0].record(st)
            tf.FUNCS[f](*dargs[f], out=(z0, z1), stream=st)
            if evs is not None:
                evs[f][1].record(st)

    peak, sms = fp64_peak(dev)
    alu = alu_peak(dev, 0)
    alu_imad = alu_peak(dev, 1)
    for _ in range(a.warmup):
        step()
    evs = [{f: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for f in FUNCS}
           for _ in range(a.steps)]
    gpu_id = None
    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        gpu_id = gpu_id if gpu_id.startswith("GPU-") else "GPU-" + gpu_id
    except Exception:
        gpu_id = None
    clocks = Clocks(gpu_id)
    barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(st)
    for k in range(a.steps):
        step(evs[k])
    t1.record(st)
    barrier()
    ck = clocks.stop()
    ms = t0.elapsed_time(t1) / a.steps
    kern_ms = {f: statistics.mean(e[f][0].elapsed_time(e[f][1]) for e in evs) for f in FUNCS}
    ms = reduce_max(ms, world, dev)
    mfuncs = [f for f in METRIC_FUNCS if f in FUNCS] or list(FUNCS)
    metric_ms = reduce_max(sum(kern_ms[f] for f in mfuncs), world, dev)
    value = world * n * len(mfuncs) / (metric_ms * 1e-3) / 1e9
    step_value = world * n * len(FUNCS) / (ms * 1e-3) / 1e9

    # end to end through the host-array API: the metric's functions on pinned host
    # buffers, every byte crossing the GPU's host link inside the timed region
    e2e = None
    if not a.no_e2e:
        pin = {f: [torch.from_numpy(x).pin_memory() for x in host[f]] for f in mfuncs}
        outs = {f: (torch.empty(n, dtype=torch.float64, pin_memory=True),
                    torch.empty(n, dtype=torch.float64, pin_memory=True)) for f in mfuncs}
        h2d = sum(8 * n * len(host[f]) for f in mfuncs)
        d2h = 16 * n * len(mfuncs)
        res = {}
        for mode in ("zero-copy", "pipeline"):
            for f in mfuncs:
                tf.call_host(f, *pin[f], out=outs[f], device=dev, mode=mode)
            ke = max(3, a.steps // 2)
            barrier()
            c0 = time.perf_counter()
            for _ in range(ke):
                for f in mfuncs:
                    tf.call_host(f, *pin[f], out=outs[f], device=dev, mode=mode)
            barrier()
            dt = reduce_max((time.perf_counter() - c0) / ke, world, dev)
            res[mode] = {"value": world * n * len(mfuncs) / dt / 1e9, "ms_per_step": dt * 1e3}
        link = host_link(dev)
        moved = (h2d + d2h) / (res["zero-copy"]["ms_per_step"] * 1e-3) / 1e9
        link.update({"achieved_gbs": moved, "frac": moved / link["both_gbs"],
                     "note": "achieved = (h2d + d2h bytes per step) / zero-copy time per step; frac of both_gbs"})
        e2e = {"value": res["zero-copy"]["value"], "unit": "Gelem/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": res["zero-copy"]["ms_per_step"],
               "functions": mfuncs, "link": link,
               "mode": "zero-copy: the kernels load x0/x1 from pinned host memory and store z0/z1 there, "
                       "over the host link (tf.call_host default)",
               "pipeline": {"value": res["pipeline"]["value"], "ms_per_step": res["pipeline"]["ms_per_step"],
                            "mode": "chunked H2D copy, kernel, D2H copy over 3 streams (tf.HostPipeline)"}}
        del pin, outs

    # every rank runs its shard of the chains (the times are the slowest rank's)
    chain = None if a.no_chains else chains_bench(dev, rank, world)
    if rank != 0:
        return
    hpeak, hsrc = hbm_peak()
    counts, stamp = load_counts()
    current = stamp is not None and stamp == kernel_source_hash()
    mhz = ck.get("sm_mhz") or SM_MAX_MHZ
    dom = max(mfuncs, key=lambda f: kern_ms[f])
    d = kern_ms[dom] * 1e-3
    cnt = counts.get(dom, {})
    count_src = (f"ncu metric capture, {os.path.relpath(COUNTS_FILE, ROOT)} (kernel source hash {stamp}: "
                 f"{'current' if current else 'STALE: the kernels changed since the capture'})")
    views = {}
    if cnt:
        views["integer"] = {"achieved": cnt["alu"] * n / d / 1e9, "peak": alu / 1e9, "unit": "integer-ALU-pipe Ginst/s",
                            "inst_per_elem": cnt["alu"],
                            "peak_source": f"measured: integer-ALU calibration kernel on this GPU ({sms} SMs)"}
        views["fp64"] = {"achieved": cnt["fp64"] * n / d / 1e9, "peak": peak / 1e9, "unit": "FP64 Ginst/s",
                         "inst_per_elem": cnt["fp64"],
                         "peak_source": f"measured: DFMA calibration kernel on this GPU ({sms} SMs)"}
        for v in views.values():
            v["frac"] = v["achieved"] / v["peak"]
    hbm = {"achieved": BYTES_PER_ELEM[dom] * n / d / 1e9, "peak": hpeak, "unit": "GB/s",
           "frac": BYTES_PER_ELEM[dom] * n / d / 1e9 / hpeak, "peak_source": hsrc}
    # DRAM bytes per launch: the full-size capture when its n is the benchmark's,
    # else the small capture scaled by n (an underestimate: part of a small
    # launch's output is still in L2 when it ends)
    if cnt and current:
        traffic = cnt["traffic"] if cnt.get("traffic_n") == n else cnt["traffic_per_elem"] * n
    else:
        traffic = None
    if views:
        pipe = max(views, key=lambda k: views[k]["frac"])
        other = "fp64" if pipe == "integer" else "integer"
        roof = {"bound": "alu", "pipe": pipe, "kernel": dom, **views[pipe], "traffic": traffic,
                "traffic_unit": "bytes per launch (dram read + write)", "count_source": count_src,
                "counts_current": current, f"{other}_view": views[other], "hbm_view": hbm,
                "alu_peak_note": f"{alu / (sms * mhz * 1e6):.1f} ALU thread-instructions per SM per clock at the "
                                 f"sampled {mhz:.0f} MHz"}
    else:
        roof = {"bound": "hbm", "kernel": dom, **hbm, "traffic": None, "count_source": "no count table"}
    per = {}
    for f in FUNCS:
        t = kern_ms[f] * 1e-3
        c = counts.get(f)
        fr = {"hbm": BYTES_PER_ELEM[f] * n / t / 1e9 / hpeak}
        if c:
            fr["alu"] = c["alu"] * n / t / alu
            fr["fp64"] = c["fp64"] * n / t / peak
        b = max(fr, key=fr.get)
        per[f] = {"ms": kern_ms[f], "gelem_s": n / t / 1e9, "hbm_gbs": BYTES_PER_ELEM[f] * n / t / 1e9,
                  **{k + "_frac": v for k, v in fr.items()}, "binding": b, "binding_frac": fr[b]}
    hard = None if (a.no_hard or a.log2n < 24 or not set(METRIC_FUNCS) <= set(dargs)) else hard_case_timing(dev, dargs)
    sweep = None if (a.no_sweep or a.log2n < 26 or not set(METRIC_FUNCS) <= set(dargs)) else size_sweep(dev, dargs, a.sweep_max)
    tier = None if a.no_tier else precision_tier(dev, a.tier_log2n)
    coupled = (None if a.no_coupled or not {"texp", "texpm1", "tlog", "tlog1p"} <= set(dargs)
               else coupled_variants(dev, dargs, n))
    cpu = None
    if world == 1 and not a.no_cpu_baseline:
        rate, cores, sample, m, _ = oracle_rate(12.0)
        cpu = {"value": rate / 1e9, "unit": "Gelem/s", "cores": cores, "kind": "oracle", "sample": sample,
               "single_core": oracle_single_core(max(1 << 13, m // cores))}
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": "Gelem/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "functions": list(FUNCS), "metric_functions": mfuncs,
                   "value": "2n / (texp + tlog kernel time), CUDA events on the launching stream inside the "
                            "timed six-function step, summed over ranks",
                   "l2": "no flush: every input array (512 MiB) is larger than L2", "parallelism": f"dp{world}"},
        "metric_ms": metric_ms,
        "step": {"functions": list(FUNCS), "ms": ms, "gelem_s": step_value},
        "peaks": {"alu_ginst_s": alu / 1e9, "alu_per_sm_clk": alu / (sms * mhz * 1e6),
                  "alu_plus_imad_ginst_s": alu_imad / 1e9, "fp64_ginst_s": peak / 1e9,
                  "fp64_per_sm_clk": peak / (sms * mhz * 1e6), "hbm_gbs": hpeak, "sm_mhz": mhz,
                  "source": "alu, fp64: calibration kernels of libtfprobe.so timed here; hbm: " + hsrc},
        "roofline": roof, "per_func": per, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": len(FUNCS) * a.steps, "clocks": ck, "hard_cases": hard, "precision_tier": tier,
        "size_sweep": sweep, "variants": coupled, "chains": chain,
    }), flush=True)


def main():
    a = parse()
    if a.ncu_summary:
        N_FOR_SUMMARY[0] = a.ncu_n
        print(ncu_summary(a.ncu_summary))
        return
    world, rank, local = dist()
    if world != a.gpus and not (world == 1 and a.gpus == 1):
        if rank == 0:
            print(f"--gpus {a.gpus} but WORLD_SIZE={world}: launch with torchrun for N > 1", file=sys.stderr)
        if world == 1:
            sys.exit(2)
    if a.impl == "reference":
        reference_arm(a, world, rank)
    else:
        ours(a, world, rank, local)


if __name__ == "__main__":
    main()
