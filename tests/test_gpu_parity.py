"""Parity of the CUDA kernels (through the C ABI) with the CPU oracle.

Every test here runs the sm_103a kernels of libtf.so on cuda:0 via the Python
binding (argument marshalling only) and compares each output element with the
binary128 oracle on the same seeded inputs:
  * z0 equals the correctly rounded f(x0) in >= 99.999% of the elements and is
    never more than 1 ulp away (bitwise for tadd/tmul);
  * z0 + z1 is within 2^-100 relative (+ 2^-1074 absolute) of f(x0 + x1);
  * where the special-value rules fix z1 (NaN, infinities, underflow), z1 is
    that value bitwise.
"""
import numpy as np
import pytest

import oracle
import tfcheck
from paper_1502_05216_gb300 import inputs as I

pytestmark = pytest.mark.gpu

UNARY = ("texp", "texpm1", "tlog", "tlog1p")
BINARY = ("tadd", "tmul")


@pytest.fixture(scope="module")
def tf():
    import torch
    from paper_1502_05216_gb300 import build, tf as tfmod
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    build.build()
    tfmod.load()
    return tfmod


def _dev(a):
    import torch
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to("cuda:0")


def run(tf, func, *arrays):
    import torch
    z0, z1 = tf.FUNCS[func](*[_dev(a) for a in arrays])
    torch.cuda.synchronize()
    return z0.cpu().numpy(), z1.cpu().numpy()


def check(tf, func, args, where, rate=0.99999):
    z0, z1 = run(tf, func, *args)
    orc = oracle.evaluate(func, *args)
    if func in BINARY:
        assert np.array_equal(z0.view(np.int64), orc.Z0.view(np.int64)) or \
            np.all((z0 == orc.Z0) | (np.isnan(z0) & np.isnan(orc.Z0))), f"{where}: z0 not bitwise"
    return tfcheck.check(z0, z1, orc, "f64", rate, where, func, args)


@pytest.mark.parametrize("func", UNARY + BINARY)
def test_workload_parity(tf, func):
    """Each function's own workload distribution, n spanning many tiles with a ragged tail."""
    n = 2**17 + 37
    st = check(tf, func, I.workload(func, n), f"{func} workload")
    print(func, st)


def test_texp_uniform_config(tf):
    """texp over x0 uniform in [-708, 709], n = 2^18, seed 0."""
    st = check(tf, "texp", I.texp_uniform(2**18, 0), "texp uniform 2^18")
    print(st)


@pytest.mark.parametrize("func", UNARY)
def test_dotted_argument(tf, func):
    """x1 = NULL (the paper's texp0/texpm10/tlog0/tlog1p0)."""
    x0, _ = I.workload(func, 2**14 + 5)
    z0, z1 = run(tf, func, x0, None)
    orc = oracle.evaluate(func, x0, None)
    tfcheck.check(z0, z1, orc, "f64", 0.99999, f"{func} dotted", func, (x0, None))
    # the main part depends on x0 only
    x0, x1 = I.workload(func, 2**14 + 5)
    w0, _ = run(tf, func, x0, x1)
    assert np.array_equal(z0.view(np.int64), w0.view(np.int64))


@pytest.mark.parametrize("func", UNARY + BINARY)
@pytest.mark.parametrize("n", [1, 2, 3, 31, 33, 255, 257, 1023])
def test_small_sizes(tf, func, n):
    check(tf, func, I.workload(func, n, start=1000), f"{func} n={n}")


@pytest.mark.parametrize("func", UNARY)
def test_hard_cases(tf, func):
    """Thresholds of overflow/subnormal/underflow, log near 1, log1p near -1,
    subnormal and huge arguments, x1 = 0 and half-ulp x1, IEEE specials."""
    st = check(tf, func, I.hard_cases(func, 2**16), f"{func} hard cases")
    print(func, st)


@pytest.mark.parametrize("func", UNARY)
def test_special_values(tf, func):
    """Every pairing of the IEEE special values as (x0, x1)."""
    s = I.SPECIALS
    x0 = np.repeat(s, s.shape[0])
    x1 = np.tile(s, s.shape[0])
    check(tf, func, (x0, x1), f"{func} specials", rate=1.0)


@pytest.mark.parametrize("func", UNARY + BINARY)
def test_misaligned_equals_aligned(tf, func):
    """Pointers 8- but not 16-byte aligned take the scalar kernel: same bits."""
    import torch
    n = 4099
    args = I.workload(func, n)
    ref0, ref1 = run(tf, func, *args)
    bufs = []
    for a in args:
        b = torch.zeros(n + 1, dtype=torch.float64, device="cuda:0")
        b[1:] = torch.from_numpy(a).to("cuda:0")
        bufs.append(b[1:])
    o0 = torch.zeros(n + 1, dtype=torch.float64, device="cuda:0")
    o1 = torch.zeros(n + 1, dtype=torch.float64, device="cuda:0")
    tf.FUNCS[func](*bufs, out=(o0[1:], o1[1:]))
    torch.cuda.synchronize()
    assert np.array_equal(o0[1:].cpu().numpy().view(np.int64), ref0.view(np.int64))
    assert np.array_equal(o1[1:].cpu().numpy().view(np.int64), ref1.view(np.int64))
    assert o0[0].item() == 0 and o1[0].item() == 0


def _sprinkled(func, n, seed):
    """The workload with a special value every 97 elements (cycling through the
    IEEE specials, in x0 or x1) and, for the logarithms, a y0 next to 1 every 53:
    most warps mix the lanes of the kernels' straight-line paths with lanes
    that send the whole warp to the per-element form."""
    x0, x1 = (a.copy() for a in I.workload(func, n))
    sp = I.SPECIALS
    idx = np.arange(5, n, 97)
    x0[idx[::2]] = sp[np.arange(idx[::2].size) % sp.size]
    x1[idx[1::2]] = sp[np.arange(idx[1::2].size) % sp.size]
    if func in ("tlog", "tlog1p"):
        near = np.arange(11, n, 53)
        u = I.uniform(seed, 1, near.size)
        x0[near] = (1.0 + (u - 0.5) * 2.0**-9) - (1.0 if func == "tlog1p" else 0.0)
    return x0, x1


@pytest.mark.parametrize("func", UNARY)
def test_mixed_warps_equal_scalar_kernel(tf, func):
    """The vector kernel evaluates a thread's two elements in one call (texp,
    tlog) or one after the other, with warp-wide votes choosing the form; the
    scalar kernel (pointers not 16-byte aligned) evaluates each element alone.
    On warps that mix special, rare and ordinary lanes both give the same bits,
    and match the oracle."""
    import torch
    n = 4099
    args = _sprinkled(func, n, 41)
    ref0, ref1 = run(tf, func, *args)
    bufs = []
    for a in args:
        b = torch.zeros(n + 1, dtype=torch.float64, device="cuda:0")
        b[1:] = torch.from_numpy(a).to("cuda:0")
        bufs.append(b[1:])
    o0 = torch.zeros(n + 1, dtype=torch.float64, device="cuda:0")
    o1 = torch.zeros(n + 1, dtype=torch.float64, device="cuda:0")
    tf.FUNCS[func](*bufs, out=(o0[1:], o1[1:]))
    torch.cuda.synchronize()
    assert np.array_equal(o0[1:].cpu().numpy().view(np.int64), ref0.view(np.int64))
    assert np.array_equal(o1[1:].cpu().numpy().view(np.int64), ref1.view(np.int64))
    check(tf, func, args, f"{func} mixed warps", rate=1.0)


@pytest.mark.parametrize("func", UNARY)
def test_in_place(tf, func):
    """z0 may alias x0 and z1 may alias x1."""
    import torch
    n = 3001
    x0, x1 = I.workload(func, n)
    ref0, ref1 = run(tf, func, x0, x1)
    a, b = _dev(x0), _dev(x1)
    tf.FUNCS[func](a, b, out=(a, b))
    torch.cuda.synchronize()
    assert np.array_equal(a.cpu().numpy().view(np.int64), ref0.view(np.int64))
    assert np.array_equal(b.cpu().numpy().view(np.int64), ref1.view(np.int64))


def test_side_stream_and_empty(tf):
    """Work goes to the given stream; n = 0 is a no-op."""
    import torch
    x0, x1 = I.workload("texp", 5000)
    ref0, ref1 = run(tf, "texp", x0, x1)
    s = torch.cuda.Stream()
    a, b = _dev(x0), _dev(x1)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        z0, z1 = tf.texp(a, b, stream=s)
    s.synchronize()
    assert np.array_equal(z0.cpu().numpy().view(np.int64), ref0.view(np.int64))
    e = torch.empty(0, dtype=torch.float64, device="cuda:0")
    tf.texp(e, e, out=(e, e))
    torch.cuda.synchronize()


# ---- full size, in the launch configuration the benchmark times -------------------

N_FULL = 2**26
SAMPLE_SLICES = 48
SLICE = 1024


def _sample_starts(n):
    step = n // SAMPLE_SLICES
    return [k * step + (k * 7919) % (step - SLICE) for k in range(SAMPLE_SLICES - 1)] + [n - SLICE]


@pytest.mark.parametrize("func", UNARY + BINARY)
def test_full_size_sampled(tf, func):
    """n = 2^26 on the device; 48 slices of 1024 outputs (the last one the tail)
    are checked element by element against the oracle."""
    import torch
    args = I.workload(func, N_FULL)
    dargs = [_dev(a) for a in args]
    z0, z1 = tf.FUNCS[func](*dargs)
    torch.cuda.synchronize()
    idx = np.concatenate([np.arange(s, s + SLICE) for s in _sample_starts(N_FULL)])
    ti = torch.from_numpy(idx).to("cuda:0")
    h0 = z0[ti].cpu().numpy()
    h1 = z1[ti].cpu().numpy()
    sub = [a[idx] for a in args]
    orc = oracle.evaluate(func, *sub)
    st = tfcheck.check(h0, h1, orc, "f64", 0.99999, f"{func} 2^26 sampled", func, sub)
    print(func, st)


@pytest.mark.parametrize("func", UNARY + BINARY)
@pytest.mark.parametrize("mode", ["zero-copy", "pipeline"])
def test_host_api_equals_device_call(tf, func, mode):
    """The host-array API (tf.call_host): the zero-copy mode, whose kernel reads
    and writes pinned host memory directly, and the chunked copy pipeline give
    the device call's results bit for bit, including a ragged last chunk."""
    import torch
    n = (1 << 22) + 4099
    args = I.workload(func, n, start=77)
    pin = [torch.from_numpy(a).pin_memory() for a in args]
    z0, z1 = tf.call_host(func, *pin, mode=mode)
    ref0, ref1 = run(tf, func, *args)
    assert np.array_equal(z0.numpy().view(np.int64), ref0.view(np.int64))
    assert np.array_equal(z1.numpy().view(np.int64), ref1.view(np.int64))


@pytest.mark.parametrize("func", ("texp", "tlog"))
def test_hard_cases_2p24(tf, func):
    """The 2^24-element hard-case set (thresholds, subnormal results, log near 1
    and of subnormals, x1 = 0 and half-ulp x1, IEEE specials), every element
    against the oracle."""
    st = check(tf, func, I.hard_cases(func, 2**24, seed=29), f"{func} hard cases 2^24")
    print(func, st)


@pytest.mark.parametrize("func", ("texp", "tmul"))
@pytest.mark.parametrize("aligned", [True, False])
def test_beyond_2p31_elements(tf, func, aligned):
    """n = 2^31 + 5 elements (64-bit element indices, 16 GiB per array): the
    128-bit vector kernel (aligned) and the scalar one (the input offset by one
    element).  x0 = -700 + 1400 ((40503 i) mod 2^16) / 2^16 is made on the
    device from the element index i, with exact operations, so the host
    reproduces it bit for bit; x1 = NULL (dotted), and tmul squares x0 (both
    operands the same array).  Outputs at both ends, around 2^30 and 2^31 and
    at 4096 random indices are checked against the oracle."""
    import torch
    n = (1 << 31) + 5
    off = 0 if aligned else 1
    buf = torch.empty(n + off, dtype=torch.float64, device="cuda:0")
    x0 = buf[off:]
    chunk = 1 << 28
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        i = torch.arange(s, e, dtype=torch.int64, device="cuda:0")
        x0[s:e] = ((i * 40503) % 65536).to(torch.float64) * (1400.0 / 65536) - 700.0
        del i
    z0, z1 = tf.FUNCS[func](x0, None) if func == "texp" else tf.FUNCS[func](x0, None, x0, None)
    torch.cuda.synchronize()
    rng = np.random.default_rng(31)
    idx = np.unique(np.concatenate([np.arange(0, 8), np.arange((1 << 30) - 4, (1 << 30) + 4),
                                    np.arange((1 << 31) - 8, (1 << 31) + 4), np.arange(n - 8, n),
                                    rng.integers(0, n, 4096)]))
    ti = torch.from_numpy(idx).to("cuda:0")
    h0, h1 = z0[ti].cpu().numpy(), z1[ti].cpu().numpy()
    hx = x0[ti].cpu().numpy()
    del z0, z1, x0, buf, ti
    torch.cuda.empty_cache()
    want = ((idx * 40503) % 65536).astype(np.float64) * (1400.0 / 65536) - 700.0
    assert np.array_equal(hx.view(np.int64), want.view(np.int64)), "device inputs differ from the host formula"
    args = (want, None) if func == "texp" else (want, None, want, None)
    orc = oracle.evaluate(func, *args)
    st = tfcheck.check(h0, h1, orc, "f64", 0.99999, f"{func} n=2^31+5 aligned={aligned}", func, args)
    print(func, aligned, st)
