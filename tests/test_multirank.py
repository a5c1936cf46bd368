"""The N > 1 path of bench.py on CPU: two gloo ranks.

The path partitions: every rank evaluates its own n elements (weak scaling)
and the only collectives are the barrier and the max-over-ranks timing.  Here
two processes check that their shards are disjoint and together are exactly
the single-process workload of 2n elements (inputs depend on the element
index only), that their chain shards together hold every chain of the batch
once, and that reduce_max returns the slowest rank's time."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_1502_05216_gb300 import inputs as I
        shards = {}
        for func in ("texp", "tlog", "tadd"):
            shards[func] = I.workload(func, n, start=bench.rank_start(rank, n))
        from paper_1502_05216_gb300 import chains
        cs = chains.shard(I.chains(700, seed=44, mean_len=20.0, cap=100), rank, world)
        shards["chains"] = {k: cs[k] for k in ("ids", "length", "s0", "ops")}
        gathered = [None] * world
        dist.all_gather_object(gathered, shards)
        slowest = bench.reduce_max(10.0 + rank, world, "cpu")
        dist.barrier()
        if rank == 0:
            out.put((gathered, slowest))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_shard_and_reduce():
    world, n = 2, 5000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, slowest = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_1502_05216_gb300 import inputs as I
    assert slowest == 10.0 + world - 1
    for func in ("texp", "tlog", "tadd"):
        whole = I.workload(func, world * n)
        for k, arr in enumerate(whole):
            joined = np.concatenate([gathered[r][func][k] for r in range(world)])
            assert np.array_equal(joined.view(np.int64), arr.view(np.int64)), (func, k)
    # chains: each rank builds its shard alone; together they are every chain once,
    # with its state, and the ops of the whole batch
    b = I.chains(700, seed=44, mean_len=20.0, cap=100)
    ids = np.concatenate([gathered[r]["chains"]["ids"] for r in range(world)])
    assert np.array_equal(np.sort(ids), np.arange(700))
    for r in range(world):
        g = gathered[r]["chains"]
        assert np.array_equal(g["length"], b["length"][g["ids"]]) and np.array_equal(g["s0"], b["s0"][g["ids"]])
    assert sum(gathered[r]["chains"]["ops"].size for r in range(world)) == b["ops"].size
