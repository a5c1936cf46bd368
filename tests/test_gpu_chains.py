"""Parity of the chain kernels (tf_chain, tf_chain_step) with the CPU oracle.

A chain applies tadd/tmul/texp/tlog in sequence to a twofold state.  Checked:
  * the fused persistent launch and the per-operation baseline give the same
    final states bit for bit, under every launch configuration and in CUDA
    graphs (both run the same device operations in the same order per chain);
  * the final state z0 + z1 is within 2^-97 K |F| of the exact result F of
    the chain, K its condition sum (oracle.chain): each operation makes a
    relative error of at most ~2^-100 and the later ones propagate it;
  * a chain of one operation equals the elementwise entry point bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_1502_05216_gb300 import inputs as I

pytestmark = pytest.mark.gpu

EPS = 2.0**-97


@pytest.fixture(scope="module")
def mods():
    import torch
    from paper_1502_05216_gb300 import build, chains, tf
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    build.build()
    tf.load()
    return tf, chains


def check_oracle(batch, z0, z1, where):
    Fh, Fl, K = oracle.chain(batch)
    # |z0 + z1 - F| with the large parts cancelled first
    err = np.abs((z0 - Fh) + (z1 - Fl))
    A = np.abs(Fh)
    tol = EPS * K * A + 2.0**-1060
    bad = np.nonzero(~(err <= tol))[0]
    assert bad.size == 0, (f"{where}: {bad.size} chains beyond 2^-97 K |F|; first {bad[:5]}: "
                           f"err/|F| {err[bad[:5]] / A[bad[:5]]}, K {K[bad[:5]]}")
    rel = err / A
    return {"chains": int(z0.size), "max_rel_log2": float(np.log2(rel.max())) if rel.max() > 0 else -np.inf,
            "max_rel_over_K_log2": float(np.log2((rel / K).max())) if rel.max() > 0 else -np.inf,
            "max_K_log2": float(np.log2(K.max()))}


def same(a, b):
    """Bitwise equal, or both NaN: which NaN an operation with several NaN
    operands returns depends on the order the compiler gives the operands
    (IEEE 754 leaves the payload open), and two kernels may order them
    differently."""
    return np.all((a.view(np.int64) == b.view(np.int64)) | (np.isnan(a) & np.isnan(b)))


def run_both(chains, batch):
    cb = chains.ChainBatch(batch)
    cb.reset()
    cb.run_fused()
    f = cb.state()
    cb.reset()
    cb.run_per_op()
    p = cb.state()
    return cb, f, p


def test_fused_equals_per_op_and_oracle(mods):
    tf, chains = mods
    batch = I.chains(4096, seed=21, mean_len=64.0, cap=512)
    cb, f, p = run_both(chains, batch)
    assert np.array_equal(f[0].view(np.int64), p[0].view(np.int64))
    assert np.array_equal(f[1].view(np.int64), p[1].view(np.int64))
    print(check_oracle(batch, *f, "4096 chains"))


@pytest.mark.parametrize("threads,blocks,group", [(32, 0, 0), (64, 1, 0), (256, 0, 0), (512, 3, 0), (128, 1000, 0),
                                                (128, 0, 1), (64, 0, 7), (128, 5, 16), (256, 0, 31), (32, 2, 32)])
def test_launch_configs_agree(mods, threads, blocks, group):
    """Block size, grid size, chains per warp and the work queue change who runs
    a chain, never its result."""
    tf, chains = mods
    batch = I.chains(3000, seed=22, mean_len=32.0, cap=300)
    cb = chains.ChainBatch(batch)
    cb.reset()
    cb.run_per_op()
    ref = cb.state()
    cb.reset()
    cb.run_fused(threads, blocks, group)
    got = cb.state()
    assert np.array_equal(ref[0].view(np.int64), got[0].view(np.int64))
    assert np.array_equal(ref[1].view(np.int64), got[1].view(np.int64))


def test_too_large_block_is_rejected(mods):
    """A block size whose registers do not fit, or a group outside 0 .. 32, is
    refused before launching."""
    tf, chains = mods
    batch = I.chains(64, seed=26, mean_len=4.0, cap=8)
    cb = chains.ChainBatch(batch)
    with pytest.raises(tf.TwofoldError, match="invalid argument"):
        cb.run_fused(1024, 0)
    for g in (-1, 33):
        with pytest.raises(tf.TwofoldError, match="invalid argument"):
            cb.run_fused(128, 0, g)


def test_length_tiers_cover_every_chain(mods):
    """The length tiers of group 0 split the chains at max_len / 1.78 .. / 4.7:
    a batch with lengths at, just above and just below every boundary (and
    ties across them) runs every chain exactly once, bitwise as the
    per-operation baseline."""
    tf, chains = mods
    rng = np.random.default_rng(27)
    max_len = 600
    cuts = [int(max_len / f) for f in (1.78, 2.87, 3.97, 4.58, 4.7)]
    lens = [max_len] + [c + d for c in cuts for d in (-1, 0, 1) for _ in range(rng.integers(1, 40))]
    lens += list(rng.integers(1, 120, 3000))
    base = I.chains(len(lens), seed=28, mean_len=1e9, cap=max_len)   # every chain max_len long
    L = np.sort(np.array(lens, np.int64))[::-1]
    # keep each chain's first L steps of the step-major stream (the ops stay feasible)
    active = np.searchsorted(-L, -np.arange(max_len), side="left")
    sb = np.zeros(max_len + 1, np.int64)
    sb[1:] = np.cumsum(active)
    keep = np.concatenate([np.arange(base["step_base"][t], base["step_base"][t] + active[t]) for t in range(max_len)])
    batch = {"ops": base["ops"][keep], "a0": base["a0"][keep], "a1": base["a1"][keep], "step_base": sb,
             "length": L.astype(np.int32), "s0": base["s0"], "s1": base["s1"], "max_len": max_len}
    cb = chains.ChainBatch(batch)
    cb.reset()
    cb.run_per_op()
    ref = cb.state()
    for group in (0, 3):
        cb.reset()
        cb.run_fused(64, 0, group)
        got = cb.state()
        assert np.array_equal(ref[0].view(np.int64), got[0].view(np.int64)), group
        assert np.array_equal(ref[1].view(np.int64), got[1].view(np.int64)), group
    check_oracle(batch, *got, "tier boundaries")


@pytest.mark.parametrize("threads,blocks", [(128, 0), (32, 1), (64, 3)])
def test_equal_length_batch_packs(mods, threads, blocks):
    """Many chains of the maximum length (every chain in the longest tier):
    group 0 packs them by the launch's warp count (from one chain per warp up
    to 32, down to a single small block) and still runs every chain exactly
    once, bitwise as the per-operation baseline."""
    tf, chains = mods
    batch = I.chains(5000, seed=30, mean_len=1e9, cap=40)
    cb = chains.ChainBatch(batch)
    cb.reset()
    cb.run_per_op()
    ref = cb.state()
    cb.reset()
    cb.run_fused(threads, blocks, 0)
    got = cb.state()
    assert np.array_equal(ref[0].view(np.int64), got[0].view(np.int64))
    assert np.array_equal(ref[1].view(np.int64), got[1].view(np.int64))


def test_graphs_replay(mods):
    import torch
    tf, chains = mods
    batch = I.chains(2048, seed=23, mean_len=40.0, cap=400)
    cb = chains.ChainBatch(batch)
    cb.reset()
    cb.run_fused()
    ref = cb.state()
    for mode, group in (("fused", 0), ("fused", 32), ("per_op", 0)):
        g = cb.graph(mode, group=group)
        for _ in range(2):
            cb.s0.zero_()
            g.replay()
            torch.cuda.synchronize()
            got = cb.state()
            assert np.array_equal(ref[0].view(np.int64), got[0].view(np.int64)), mode
            assert np.array_equal(ref[1].view(np.int64), got[1].view(np.int64)), mode


@pytest.mark.parametrize("group", [0, 32])
def test_single_op_chains_equal_elementwise(mods, group):
    """A chain of length 1 is the elementwise function of its state and operand,
    bitwise, on regular values and on every pairing of the IEEE specials (NaN,
    infinities, signed zeros, subnormals, the largest double) in both parts:
    one chain per warp (group 0: every chain is the longest) runs the plain
    step loop, 32 per warp the cheap/costly phases."""
    import torch
    tf, chains = mods
    n = 1000
    x0, x1 = I.exp_args(n, 31)
    x0 = np.abs(x0) % 13.0 + 2.0**-20
    x1 = x0 * (np.arange(n) % 7 - 3) * 2.0**-55
    y0, y1 = I.arith_args(n, 32)
    sp = I.SPECIALS
    m = sp.size
    pairs = np.stack(np.meshgrid(np.arange(m), np.arange(m), indexing="ij"), -1).reshape(-1, 2)
    small = np.array([0.0, -0.0, 2.0**-60, -(2.0**-1074), np.inf, np.nan])
    sx0 = np.repeat(sp[pairs[:, 0]], small.size)
    sy0 = np.repeat(sp[pairs[:, 1]], small.size)
    sx1 = np.tile(small, pairs.shape[0])
    sy1 = np.roll(sx1, 1)
    x0, x1, y0, y1 = (np.concatenate([a, b]) for a, b in ((x0, sx0), (x1, sx1), (y0, sy0), (y1, sy1)))
    n = x0.size
    for op, name in ((0, "tadd"), (1, "tmul"), (2, "texp"), (3, "tlog")):
        batch = {"ops": np.full(n, op, np.uint8), "a0": y0, "a1": y1, "step_base": np.array([0, n], np.int64),
                 "length": np.ones(n, np.int32), "s0": x0, "s1": x1, "max_len": 1}
        cb = chains.ChainBatch(batch)
        cb.run_fused(128, 0, group)
        got = cb.state()
        d = [torch.from_numpy(a).cuda() for a in ((x0, x1, y0, y1) if op < 2 else (x0, x1))]
        z0, z1 = tf.FUNCS[name](*d)
        assert same(z0.cpu().numpy(), got[0]), name
        assert same(z1.cpu().numpy(), got[1]), name
        reg = slice(0, 1000)  # regular values: bitwise
        assert np.array_equal(z1.cpu().numpy()[reg].view(np.int64), got[1][reg].view(np.int64)), name


def test_mixed_cheap_ops_equal_per_op(mods):
    """Warps whose lanes mix tadd, tmul and unknown op codes in their cheap
    phases, on special states and operands: bitwise the per-operation kernels,
    NaN for NaN."""
    tf, chains = mods
    sp = I.SPECIALS
    rng = np.random.default_rng(29)
    n, L = 4096, 6
    s0 = sp[rng.integers(0, sp.size, n)]
    s1 = np.where(rng.random(n) < 0.5, 0.0, s0 * 2.0**-60)
    tot = n * L
    ops = rng.choice(np.array([0, 1, 0, 1, 9], np.uint8), tot)
    a0 = np.where(rng.random(tot) < 0.3, sp[rng.integers(0, sp.size, tot)], rng.standard_normal(tot) * 4)
    with np.errstate(invalid="ignore", over="ignore"):
        a1 = np.where(rng.random(tot) < 0.2, sp[rng.integers(0, sp.size, tot)], a0 * 2.0**-57)
    batch = {"ops": ops, "a0": a0, "a1": a1, "step_base": np.arange(L + 1, dtype=np.int64) * n,
             "length": np.full(n, L, np.int32), "s0": s0, "s1": s1, "max_len": L}
    cb = chains.ChainBatch(batch)
    cb.reset()
    cb.run_per_op()
    ref = cb.state()
    for group in (32, 5):
        cb.reset()
        cb.run_fused(128, 0, group)
        got = cb.state()
        assert same(ref[0], got[0]) and same(ref[1], got[1]), group
        assert np.isfinite(got[0]).mean() > 0.3  # most chains stay finite


def test_edge_batches(mods):
    """One chain; all chains of equal length; an unknown op code is a no-op."""
    tf, chains = mods
    b1 = I.chains(1, seed=24, mean_len=100.0, cap=200)
    cb, f, p = run_both(chains, b1)
    assert np.array_equal(f[0].view(np.int64), p[0].view(np.int64))
    check_oracle(b1, *f, "one chain")
    b2 = I.chains(500, seed=25, mean_len=1e9, cap=50)  # every chain hits the cap
    assert np.all(b2["length"] == 50)
    cb, f, p = run_both(chains, b2)
    assert np.array_equal(f[1].view(np.int64), p[1].view(np.int64))
    check_oracle(b2, *f, "equal lengths")
    b3 = dict(b2)
    b3["ops"] = b2["ops"].copy()
    b3["ops"][b2["step_base"][49]:b2["step_base"][50]] = 200  # last step: unknown op everywhere
    cb, f3, p3 = run_both(chains, b3)
    assert np.array_equal(f3[0].view(np.int64), p3[0].view(np.int64))
    check_oracle(b3, *f3, "unknown op")
    b4 = dict(b2)
    b4["ops"] = b2["ops"][:b2["step_base"][49]]
    b4["step_base"] = b2["step_base"][:50]
    b4["length"] = np.full(500, 49, np.int32)
    b4["max_len"] = 49
    cb = chains.ChainBatch(b4)
    cb.run_fused()
    f4 = cb.state()
    assert np.array_equal(f3[0].view(np.int64), f4[0].view(np.int64))


def test_full_size_batch(mods):
    """The full batched-chains workload: 65,536 chains, mean length 256, cap
    4096; every chain checked against the oracle, fused == per-op bitwise."""
    tf, chains = mods
    batch = I.chains(65536)
    cb, f, p = run_both(chains, batch)
    assert np.array_equal(f[0].view(np.int64), p[0].view(np.int64))
    assert np.array_equal(f[1].view(np.int64), p[1].view(np.int64))
    st = check_oracle(batch, *f, "65536 chains")
    st["ops"] = int(batch["ops"].size)
    st["mix"] = batch["mix"].tolist()
    print(st)
