"""Batched chains of twofold operations: the host side of tf_chain.

A ``ChainBatch`` holds one step-major batch on the device (layout of
include/tf.h) and runs it two ways:

* ``run_fused``: every chain in one persistent launch (tf_chain);
* ``run_per_op``: the baseline, one launch per step and operation kind over
  the chains doing that operation (tf_chain_step with index lists).

Both can be captured in a CUDA graph together with the reset of the chain
states, so that a replay is one whole batch.  ``tune`` picks the fused
launch's block size and grid by timing the candidates on the batch itself.
All arithmetic runs in the CUDA kernels; this module only moves arrays,
builds the per-operation index lists and enqueues launches.
"""
from __future__ import annotations

import statistics

import numpy as np

from . import tf

# block sizes, grids (blocks per SM, 0 = one full wave) and chains per warp
# (0 = by length, see tf_chain) the tuner tries
TUNE_THREADS = (32, 64, 128, 256, 512)
TUNE_BLOCKS_PER_SM = (0, 1, 2, 3, 4)
TUNE_GROUPS = (0, 8, 32)


def shard(batch: dict, rank: int, world: int) -> dict:
    """Rank ``rank``'s share of a step-major batch for ``world`` GPUs: the
    chains c with c % world == rank, as a step-major batch of their own.  The
    chains keep their longest-first order, so every rank gets an even mix of
    long and short chains, and each chain keeps its state and its operations
    in order: a shard's results are those chains' results of the whole
    batch.  No data moves between ranks (the chains are independent)."""
    L = np.asarray(batch["length"], dtype=np.int64)
    ids = np.arange(rank, L.size, world, dtype=np.int64)
    Ls = L[ids]
    max_len = int(Ls[0]) if ids.size else 0
    active = np.searchsorted(-Ls, -np.arange(max_len), side="left")  # shard chains with L > t
    sb = np.zeros(max_len + 1, dtype=np.int64)
    sb[1:] = np.cumsum(active)
    t_of = np.repeat(np.arange(max_len, dtype=np.int64), active)
    keep = np.asarray(batch["step_base"], dtype=np.int64)[t_of] + ids[np.arange(t_of.size) - sb[t_of]]
    out = {"ops": batch["ops"][keep], "a0": batch["a0"][keep], "a1": batch["a1"][keep], "step_base": sb,
           "length": Ls.astype(np.int32), "s0": batch["s0"][ids], "s1": batch["s1"][ids], "max_len": max_len,
           "ids": ids}
    out["mix"] = np.bincount(out["ops"], minlength=4)
    return out


def per_op_lists(ops: np.ndarray, step_base: np.ndarray, max_len: int):
    """Index lists of the per-operation baseline: for every step t and op kind,
    the chains (positions within step t's block) that apply that op, all
    concatenated in (t, op) order as int32, and the non-empty launches as
    (op, t, offset, count).  Unknown op codes get no launch (a no-op)."""
    sb = np.asarray(step_base, dtype=np.int64)
    total = int(sb[-1])
    t_of = np.repeat(np.arange(max_len, dtype=np.int64), np.diff(sb))
    c_of = np.arange(total, dtype=np.int64) - sb[t_of]
    ops = np.asarray(ops)[:total]
    valid = ops < 4
    t_of, c_of = t_of[valid], c_of[valid]
    key = t_of * 4 + ops[valid].astype(np.int64)
    order = np.argsort(key, kind="stable")
    counts = np.bincount(key, minlength=4 * max_len)
    offs = np.concatenate([[0], np.cumsum(counts)])
    nz = np.nonzero(counts)[0]
    launches = [(int(k % 4), int(k // 4), int(offs[k]), int(counts[k])) for k in nz]
    return c_of[order].astype(np.int32), launches


class ChainBatch:
    def __init__(self, batch: dict, device="cuda"):
        import torch
        self.device = torch.device(device)
        d = self.device
        self.n = int(batch["s0"].shape[0])
        self.max_len = int(batch["max_len"])
        self.ops = torch.from_numpy(np.ascontiguousarray(batch["ops"], dtype=np.uint8)).to(d)
        self.a0 = torch.from_numpy(np.ascontiguousarray(batch["a0"], dtype=np.float64)).to(d)
        self.a1 = torch.from_numpy(np.ascontiguousarray(batch["a1"], dtype=np.float64)).to(d)
        self.step_base_host = np.ascontiguousarray(batch["step_base"], dtype=np.int64)
        self.step_base = torch.from_numpy(self.step_base_host).to(d)
        self.length = torch.from_numpy(np.ascontiguousarray(batch["length"], dtype=np.int32)).to(d)
        self.init0 = torch.from_numpy(np.ascontiguousarray(batch["s0"], dtype=np.float64)).to(d)
        self.init1 = torch.from_numpy(np.ascontiguousarray(batch["s1"], dtype=np.float64)).to(d)
        self.s0 = self.init0.clone()
        self.s1 = self.init1.clone()
        self.workspace = torch.zeros(tf.CHAIN_WORKSPACE, dtype=torch.uint8, device=d)
        self.total_ops = int(self.step_base_host[-1])
        self._launches = None
        self.sms = torch.cuda.get_device_properties(d).multi_processor_count

    # -- the two ways to run a batch -------------------------------------------------
    def reset(self, stream=None):
        """Chain states back to the initial ones (device copies on `stream`)."""
        import torch
        s = stream or torch.cuda.current_stream(self.device)
        with torch.cuda.stream(s):
            self.s0.copy_(self.init0)
            self.s1.copy_(self.init1)

    def run_fused(self, threads: int = 128, blocks: int = 0, group: int = 0, stream=None):
        tf.chain(self.ops, self.a0, self.a1, self.step_base, self.length, self.s0, self.s1,
                 self.max_len, self.workspace, threads=threads, blocks=blocks, group=group, stream=stream)

    def _build_per_op(self):
        import torch
        idx, self._launches = per_op_lists(self.ops.cpu().numpy(), self.step_base_host, self.max_len)
        self.idx = torch.from_numpy(idx).to(self.device)

    @property
    def per_op_launches(self) -> int:
        if self._launches is None:
            self._build_per_op()
        return len(self._launches)

    def run_per_op(self, stream=None):
        if self._launches is None:
            self._build_per_op()
        sb = self.step_base_host
        for op, t, off, cnt in self._launches:
            tf.chain_step(op, self.idx[off:off + cnt], int(sb[t]), self.a0, self.a1, self.s0, self.s1,
                          stream=stream)

    # -- CUDA graphs ------------------------------------------------------------------
    def graph(self, mode: str = "fused", threads: int = 128, blocks: int = 0, group: int = 0):
        """A CUDA graph of one whole batch: reset the states, then run it
        (mode "fused" or "per_op").  Replay with .replay()."""
        import torch
        if mode == "per_op" and self._launches is None:
            self._build_per_op()
        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            # one eager run first, so that nothing is first touched under capture
            self.reset(s)
            self._run(mode, threads, blocks, group, s)
            s.synchronize()
            with torch.cuda.graph(g, stream=s):
                self.reset(s)
                self._run(mode, threads, blocks, group, s)
        torch.cuda.current_stream(self.device).wait_stream(s)
        return g

    def _run(self, mode, threads, blocks, group, stream):
        if mode == "fused":
            self.run_fused(threads, blocks, group, stream)
        elif mode == "per_op":
            self.run_per_op(stream)
        else:
            raise ValueError(mode)

    def time_graph(self, g, reps: int = 5) -> float:
        """Median milliseconds of one replay (CUDA events on the current stream)."""
        import torch
        st = torch.cuda.current_stream(self.device)
        g.replay()
        torch.cuda.synchronize(self.device)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            g.replay()
            e1.record(st)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    # -- autotuner --------------------------------------------------------------------
    def tune(self, reps: int = 3):
        """Time every (group, threads, blocks) candidate of the fused launch on
        this batch and return (best config dict, table of all timings)."""
        table = []
        for grp in TUNE_GROUPS:
            for th in TUNE_THREADS:
                for bps in TUNE_BLOCKS_PER_SM:
                    blocks = bps * self.sms
                    g = self.graph("fused", th, blocks, grp)
                    ms = self.time_graph(g, reps)
                    table.append({"group": grp, "threads": th, "blocks": blocks, "ms": ms})
                    del g
        best = min(table, key=lambda r: r["ms"])
        return {"group": best["group"], "threads": best["threads"], "blocks": best["blocks"]}, table

    def state(self):
        """Final chain states as numpy arrays (s0, s1)."""
        return self.s0.cpu().numpy(), self.s1.cpu().numpy()
