"""Bounds of every store (GPU): sentinel-filled slack around the outputs.

compute-sanitizer is not available on this machine, so out-of-bounds stores are
caught with canaries instead: each output lives inside a larger buffer whose
slack before and after it holds a sentinel bit pattern (a signalling-NaN
payload no kernel produces), and every launch must leave that slack, and the
inputs, bit for bit as they were.  Sizes n = 1 .. 1023 cover every ragged tail
of the 2-per-thread double kernels and the 4-per-thread float kernels and
partial blocks and warps; each runs through the 128-bit vector kernel (all
pointers 16-byte aligned) and the scalar kernel (all pointers offset by one
element), and the first n outputs must equal those of one launch over all
1023 elements.  The fused chain kernel's state arrays get the same check.
"""
import numpy as np
import pytest

from paper_1502_05216_gb300 import inputs as I

pytestmark = pytest.mark.gpu

UNARY = ("texp", "texpm1", "tlog", "tlog1p")
BINARY = ("tadd", "tmul")
NMAX = 1023
PAD = 64                                   # elements of slack on each side (even: keeps 16-byte alignment)
SENT64 = np.int64(0x7FF4DEADBEEF0001)     # signalling-NaN payload, double
SENT32 = np.int32(0x7FA5A5A5)             # signalling-NaN payload, float


@pytest.fixture(scope="module")
def tf():
    import torch
    from paper_1502_05216_gb300 import build, tf as tfmod
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    build.build()
    tfmod.load()
    return tfmod


def _padded(data, n, shift, f32):
    """A device buffer of n + 2 PAD + 1 elements of sentinel with data[:n] (or
    nothing) at offset PAD + shift; returns (buffer, view)."""
    import torch
    dt = torch.float32 if f32 else torch.float64
    it = torch.int32 if f32 else torch.int64
    buf = torch.full((n + 2 * PAD + 1,), int(SENT32 if f32 else SENT64), dtype=it, device="cuda:0").view(dt)
    view = buf[PAD + shift:PAD + shift + n]
    if data is not None:
        view.copy_(torch.from_numpy(np.ascontiguousarray(data[:n])).to("cuda:0"))
    return buf, view


def _bits(t, f32):
    import torch
    return t.view(torch.int32 if f32 else torch.int64).cpu().numpy()


def _check_slack(buf, n, shift, f32, where):
    b = _bits(buf, f32)
    s = SENT32 if f32 else SENT64
    lo, hi = PAD + shift, PAD + shift + n
    bad_lo = np.nonzero(b[:lo] != s)[0]
    bad_hi = np.nonzero(b[hi:] != s)[0]
    assert bad_lo.size == 0, f"{where}: store {lo - bad_lo[-1]} element(s) before the output"
    assert bad_hi.size == 0, f"{where}: store {bad_hi[0] + 1} element(s) past the end"


def _run_sizes(tf, fn, args, f32, where):
    import torch
    ref = None
    sizes = range(1, NMAX + 1)
    # the reference: one launch over all NMAX elements
    full_in = [_padded(a, NMAX, 0, f32)[1] for a in args]
    r0 = torch.empty(NMAX, dtype=full_in[0].dtype, device="cuda:0")
    r1 = torch.empty_like(r0)
    fn(*full_in, out=(r0, r1))
    ref = (_bits(r0, f32), _bits(r1, f32))
    for shift in (0, 1):                     # vector kernel, scalar kernel
        for n in sizes:
            ins = [_padded(a, n, shift, f32) for a in args]
            o0 = _padded(None, n, shift, f32)
            o1 = _padded(None, n, shift, f32)
            before = [_bits(b, f32) for b, _ in ins]
            fn(*[v for _, v in ins], out=(o0[1], o1[1]))
            torch.cuda.synchronize()
            w = f"{where} n={n} {'scalar' if shift else 'vector'}"
            _check_slack(o0[0], n, shift, f32, w + " z0")
            _check_slack(o1[0], n, shift, f32, w + " z1")
            for (b, _), bb in zip(ins, before):
                assert np.array_equal(_bits(b, f32), bb), f"{w}: an input buffer changed"
            assert np.array_equal(_bits(o0[1], f32), ref[0][:n]), f"{w}: z0 differs from the full launch"
            assert np.array_equal(_bits(o1[1], f32), ref[1][:n]), f"{w}: z1 differs from the full launch"


@pytest.mark.parametrize("func", UNARY + BINARY)
def test_double_slack(tf, func):
    _run_sizes(tf, tf.FUNCS[func], I.workload(func, NMAX, start=5000), False, func)


@pytest.mark.parametrize("func", UNARY)
def test_float_slack(tf, func):
    _run_sizes(tf, tf.FUNCS_F[func], I.workload_f32(func, NMAX, start=5000), True, func + "f")


@pytest.mark.parametrize("func", UNARY)
def test_dotted_slack(tf, func):
    """x1 = NULL (the dotted variants) through both kernels."""
    import torch
    x0, _ = I.workload(func, NMAX, start=7000)
    for shift in (0, 1):
        for n in (1, 2, 3, 7, 64, 255, 256, 257, 1023):
            _, v = _padded(x0, n, shift, False)
            o0 = _padded(None, n, shift, False)
            o1 = _padded(None, n, shift, False)
            tf.FUNCS[func](v, None, out=(o0[1], o1[1]))
            torch.cuda.synchronize()
            _check_slack(o0[0], n, shift, False, f"{func} dotted n={n} z0")
            _check_slack(o1[0], n, shift, False, f"{func} dotted n={n} z1")


def test_chain_state_slack(tf):
    """The fused chain kernel updates s0/s1 of n_chains chains and nothing
    around them; the per-op step kernel likewise."""
    import torch
    from paper_1502_05216_gb300 import chains
    for n_chains in (1, 31, 33, 777):
        batch = I.chains(n_chains, seed=61, mean_len=24.0, cap=100)
        cb = chains.ChainBatch(batch, "cuda:0")
        for kind in ("fused", "per_op"):
            b0, cb.s0 = _padded(batch["s0"], n_chains, 0, False)
            b1, cb.s1 = _padded(batch["s1"], n_chains, 0, False)
            if kind == "fused":
                cb.run_fused()
            else:
                cb.run_per_op()
            torch.cuda.synchronize()
            _check_slack(b0, n_chains, 0, False, f"chains {n_chains} {kind} s0")
            _check_slack(b1, n_chains, 0, False, f"chains {n_chains} {kind} s1")
