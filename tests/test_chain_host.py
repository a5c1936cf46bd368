"""Host side of the batched chains, without a GPU: the seeded generator keeps
its stated layout and ranges, and the per-operation index lists replay exactly
the operations of every chain in order."""
import numpy as np

from paper_1502_05216_gb300 import inputs as I
from paper_1502_05216_gb300.chains import per_op_lists, shard


def test_generator_layout_and_ranges():
    b = I.chains(3000, seed=41, mean_len=50.0, cap=400)
    L, sb = b["length"], b["step_base"]
    assert np.all(np.diff(L) <= 0) and L[0] == b["max_len"] and L.min() >= 1 and L.max() <= 400
    # step t's block holds exactly the chains still running
    assert np.array_equal(np.diff(sb), [(L > t).sum() for t in range(b["max_len"])])
    assert sb[0] == 0 and sb[-1] == b["ops"].size == L.sum()
    assert set(np.unique(b["ops"])) <= {0, 1, 2, 3}
    arith = b["ops"] < 2
    assert np.all(b["a0"][arith] > 0) and np.all(b["a0"][~arith] == 0) and np.all(b["a1"][~arith] == 0)
    assert np.all(np.abs(b["a1"][arith]) <= b["a0"][arith] * 2.0**-53)
    assert np.all((b["s0"] >= 1) & (b["s0"] < 2))
    assert abs(L.mean() / 50.0 - 1) < 0.1  # geometric with the stated mean (few capped)
    assert np.array_equal(b["mix"], np.bincount(b["ops"], minlength=4))


def test_generator_is_deterministic():
    a = I.chains(500, seed=42, mean_len=20.0, cap=100)
    b = I.chains(500, seed=42, mean_len=20.0, cap=100)
    for k in ("ops", "a0", "a1", "step_base", "length", "s0", "s1"):
        assert np.array_equal(a[k], b[k])


def test_states_stay_in_range():
    """Followed in plain double, every state stays positive within [2^-20, 2^20]
    (up to the rounding of the simulation)."""
    b = I.chains(2000, seed=43, mean_len=64.0, cap=300)
    s = b["s0"].copy()
    lo, hi = 2.0**-20 * (1 - 1e-9), 2.0**20 * (1 + 1e-9)
    for t in range(b["max_len"]):
        m = int(b["step_base"][t + 1] - b["step_base"][t])
        blk = slice(int(b["step_base"][t]), int(b["step_base"][t + 1]))
        op, a = b["ops"][blk], b["a0"][blk]
        st = s[:m]
        with np.errstate(over="ignore", invalid="ignore", divide="ignore"):  # np.where evaluates every branch
            s[:m] = np.where(op == 0, st + a, np.where(op == 1, st * a, np.where(op == 2, np.exp(st), np.log(st))))
        assert np.all((s[:m] >= lo) & (s[:m] <= hi)), t


def test_per_op_lists_replay_each_chain():
    b = I.chains(400, seed=44, mean_len=16.0, cap=80)
    b["ops"][5] = 9  # an unknown op code gets no launch
    idx, launches = per_op_lists(b["ops"], b["step_base"], b["max_len"])
    seq = {c: [] for c in range(400)}
    last_t = -1
    for op, t, off, cnt in launches:
        assert t >= last_t
        last_t = t
        for c in idx[off:off + cnt]:
            seq[int(c)].append((t, op))
    for c in range(400):
        want = [(t, int(b["ops"][b["step_base"][t] + c])) for t in range(int(b["length"][c]))
                if b["ops"][b["step_base"][t] + c] < 4]
        assert seq[c] == want, c


def _chain_ops(b, c):
    """(ops, a0, a1) of chain c of a step-major batch, in step order."""
    k = b["step_base"][:b["length"][c]] + c
    return b["ops"][k], b["a0"][k], b["a1"][k]


def test_shards_partition_the_batch():
    """The shards of 3 ranks are disjoint, cover every chain, are step-major
    batches themselves (non-increasing lengths, consistent step_base), and
    hold each chain's state and operations unchanged."""
    b = I.chains(1001, seed=43, mean_len=30.0, cap=200)
    world = 3
    seen = np.zeros(1001, bool)
    for r in range(world):
        s = shard(b, r, world)
        assert not seen[s["ids"]].any()
        seen[s["ids"]] = True
        L, sb = s["length"], s["step_base"]
        assert np.all(np.diff(L) <= 0) and s["max_len"] == L[0]
        assert np.array_equal(np.diff(sb), [(L > t).sum() for t in range(s["max_len"])])
        assert sb[-1] == s["ops"].size == L.sum()
        assert np.array_equal(s["s0"], b["s0"][s["ids"]]) and np.array_equal(s["s1"], b["s1"][s["ids"]])
        for j in (0, 1, L.size // 2, L.size - 1):
            for x, y in zip(_chain_ops(s, j), _chain_ops(b, s["ids"][j])):
                assert np.array_equal(x, y)
        # the longest-first order gives every rank an even share of the work
        assert abs(L.sum() / (b["length"].sum() / world) - 1) < 0.1
    assert seen.all()
    assert shard(b, 0, 1)["ops"].tobytes() == b["ops"].tobytes()
