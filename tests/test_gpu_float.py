"""Parity of the float-twofold kernels (tf_texpf, tf_texpm1f, tf_tlogf,
tf_tlog1pf) with the CPU oracle in float mode.

Same bar as the double path, at float precision: z0 equals f(x0) correctly
rounded to float in >= 99.999% of the elements and is never more than 1 float
ulp away; z0 + z1 is within 2^-44 |F| + 2^-23 |G| + 2^-149 of f(x0 + x1)
(tests/tfcheck.py); special-value z1 bitwise.
"""
import numpy as np
import pytest

import oracle
import tfcheck
from paper_1502_05216_gb300 import inputs as I

pytestmark = pytest.mark.gpu

UNARY = ("texp", "texpm1", "tlog", "tlog1p")


@pytest.fixture(scope="module")
def tf():
    import torch
    from paper_1502_05216_gb300 import build, tf as tfmod
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    build.build()
    tfmod.load()
    return tfmod


def run(tf, func, x0, x1):
    import torch
    d = [None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda() for a in (x0, x1)]
    z0, z1 = tf.FUNCS_F[func](*d)
    torch.cuda.synchronize()
    return z0.cpu().numpy(), z1.cpu().numpy()


def check(tf, func, x0, x1, where, rate=0.99999):
    z0, z1 = run(tf, func, x0, x1)
    orc = oracle.evaluate(func, x0.astype(np.float64), None if x1 is None else x1.astype(np.float64),
                          dtype="f32")
    return tfcheck.check(z0.astype(np.float64), z1.astype(np.float64), orc, "f32", rate, where)


@pytest.mark.parametrize("func", UNARY)
def test_workload_parity_f32(tf, func):
    st = check(tf, func, *I.workload_f32(func, 2**17 + 37), f"{func}f workload")
    print(func, st)


@pytest.mark.parametrize("func", UNARY)
def test_hard_cases_f32(tf, func):
    st = check(tf, func, *I.hard_cases_f32(func, 2**16), f"{func}f hard cases")
    print(func, st)


@pytest.mark.parametrize("func", UNARY)
def test_special_values_f32(tf, func):
    s = I.SPECIALS_F
    x0 = np.repeat(s, s.shape[0])
    x1 = np.tile(s, s.shape[0])
    check(tf, func, x0, x1, f"{func}f specials", rate=1.0)


@pytest.mark.parametrize("func", UNARY)
def test_dotted_f32(tf, func):
    x0, x1 = I.workload_f32(func, 2**14 + 3)
    z0, _ = run(tf, func, x0, None)
    check(tf, func, x0, None, f"{func}f dotted")
    w0, _ = run(tf, func, x0, x1)
    assert np.array_equal(z0.view(np.int32), w0.view(np.int32))  # main part depends on x0 only


@pytest.mark.parametrize("func", UNARY)
@pytest.mark.parametrize("n", [1, 3, 4, 5, 127, 1025])
def test_small_sizes_f32(tf, func, n):
    check(tf, func, *I.workload_f32(func, n, start=77), f"{func}f n={n}")


@pytest.mark.parametrize("func", UNARY)
def test_misaligned_equals_aligned_f32(tf, func):
    """Pointers 4- but not 16-byte aligned take the scalar kernel: same bits."""
    import torch
    n = 4099
    x0, x1 = I.workload_f32(func, n)
    ref = run(tf, func, x0, x1)
    bufs = []
    for a in (x0, x1):
        b = torch.zeros(n + 1, dtype=torch.float32, device="cuda:0")
        b[1:] = torch.from_numpy(a).cuda()
        bufs.append(b[1:])
    o0 = torch.zeros(n + 1, dtype=torch.float32, device="cuda:0")
    o1 = torch.zeros(n + 1, dtype=torch.float32, device="cuda:0")
    tf.FUNCS_F[func](bufs[0], bufs[1], out=(o0[1:], o1[1:]))
    torch.cuda.synchronize()
    assert np.array_equal(o0[1:].cpu().numpy().view(np.int32), ref[0].view(np.int32))
    assert np.array_equal(o1[1:].cpu().numpy().view(np.int32), ref[1].view(np.int32))


@pytest.mark.parametrize("func", UNARY)
def test_mixed_warps_equal_scalar_kernel_f32(tf, func):
    """The vector kernel evaluates a thread's four elements in calls of two
    (texpf) or four (tlogf) with warp-wide votes choosing the form, or one after
    the other; the scalar kernel evaluates each element alone.  With a special
    value every 97 elements (in x0 or x1) and, for the logarithms, a y0 next to
    1 every 53, most warps mix both kinds of lanes: same bits, and the oracle's
    bar."""
    import torch
    n = 4099
    x0, x1 = (a.copy() for a in I.workload_f32(func, n))
    sp = I.SPECIALS_F.astype(np.float32)
    idx = np.arange(5, n, 97)
    x0[idx[::2]] = sp[np.arange(idx[::2].size) % sp.size]
    x1[idx[1::2]] = sp[np.arange(idx[1::2].size) % sp.size]
    if func in ("tlog", "tlog1p"):
        near = np.arange(11, n, 53)
        u = I.uniform(43, 1, near.size)
        x0[near] = ((1.0 + (u - 0.5) * 2.0**-9) - (1.0 if func == "tlog1p" else 0.0)).astype(np.float32)
    ref = run(tf, func, x0, x1)
    bufs = []
    for a in (x0, x1):
        b = torch.zeros(n + 1, dtype=torch.float32, device="cuda:0")
        b[1:] = torch.from_numpy(a).cuda()
        bufs.append(b[1:])
    o0 = torch.zeros(n + 1, dtype=torch.float32, device="cuda:0")
    o1 = torch.zeros(n + 1, dtype=torch.float32, device="cuda:0")
    tf.FUNCS_F[func](bufs[0], bufs[1], out=(o0[1:], o1[1:]))
    torch.cuda.synchronize()
    assert np.array_equal(o0[1:].cpu().numpy().view(np.int32), ref[0].view(np.int32))
    assert np.array_equal(o1[1:].cpu().numpy().view(np.int32), ref[1].view(np.int32))
    check(tf, func, x0, x1, f"{func}f mixed warps", rate=1.0)


@pytest.mark.parametrize("func", ("texp", "tlog"))
def test_full_size_sampled_f32(tf, func):
    """n = 2^28 floats (the precision-tier size), every 2^11-th element and the
    ragged tail checked against the oracle."""
    import torch
    n = 2**28
    x0, x1 = I.workload_f32(func, n)
    d0, d1 = torch.from_numpy(x0).cuda(), torch.from_numpy(x1).cuda()
    z0, z1 = tf.FUNCS_F[func](d0, d1)
    torch.cuda.synchronize()
    idx = np.concatenate([np.arange(0, n, 2**11), np.arange(n - 1000, n)])
    ti = torch.from_numpy(idx).cuda()
    h0, h1 = z0[ti].cpu().numpy(), z1[ti].cpu().numpy()
    orc = oracle.evaluate(func, x0[idx].astype(np.float64), x1[idx].astype(np.float64), dtype="f32")
    st = tfcheck.check(h0.astype(np.float64), h1.astype(np.float64), orc, "f32", 0.99999, f"{func}f 2^28 sampled")
    print(func, st)


@pytest.mark.parametrize("func", UNARY)
def test_precision_tier_same_x0(tf, func):
    """The precision tier: each function over float twofolds and over double
    twofolds on the same x0 values (x1 = x0 u 2^-24 and x0 u 2^-53, same u),
    each checked against the oracle at its own precision; prints both error
    statistics side by side."""
    import torch
    n = 2**16
    x0f, x1f = I.workload_f32(func, n, start=3 << 20)
    x0d, x1d = I.double_of_f32(func, x0f, start=3 << 20)
    stf = check(tf, func, x0f, x1f, f"{func}f tier")
    d = [torch.from_numpy(a).cuda() for a in (x0d, x1d)]
    z0, z1 = tf.FUNCS[func](*d)
    torch.cuda.synchronize()
    orc = oracle.evaluate(func, x0d, x1d)
    std = tfcheck.check(z0.cpu().numpy(), z1.cpu().numpy(), orc, "f64", 0.99999, f"{func} tier", func, (x0d, x1d))
    print(f"tier {func}: f32 max 2^{stf['max_rel_log2']:.1f} mean 2^{stf['mean_rel_log2']:.1f} | "
          f"f64 max 2^{std['max_rel_log2']:.1f} mean 2^{std['mean_rel_log2']:.1f}")


@pytest.mark.parametrize("aligned", [True, False])
def test_beyond_2p31_elements_f32(tf, aligned):
    """n = 2^31 + 7 float twofolds (64-bit element indices, 8 GiB per array):
    the 4-wide vector kernel (aligned) and the scalar one (offset by one
    element).  x0 = -80 + 160 ((40503 i) mod 2^16) / 2^16 is made on the device
    from the index with exact float operations (the host reproduces it bit for
    bit), x1 = NULL.  Outputs at both ends, around 2^30 and 2^31 and at 4096
    random indices are checked against the oracle."""
    import torch
    n = (1 << 31) + 7
    off = 0 if aligned else 1
    buf = torch.empty(n + off, dtype=torch.float32, device="cuda:0")
    x0 = buf[off:]
    chunk = 1 << 28
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        i = torch.arange(s, e, dtype=torch.int64, device="cuda:0")
        x0[s:e] = ((i * 40503) % 65536).to(torch.float32) * (160.0 / 65536) - 80.0
        del i
    z0, z1 = tf.FUNCS_F["texp"](x0, None)
    torch.cuda.synchronize()
    rng = np.random.default_rng(37)
    idx = np.unique(np.concatenate([np.arange(0, 8), np.arange((1 << 30) - 4, (1 << 30) + 4),
                                    np.arange((1 << 31) - 8, (1 << 31) + 4), np.arange(n - 8, n),
                                    rng.integers(0, n, 4096)]))
    ti = torch.from_numpy(idx).to("cuda:0")
    h0, h1, hx = z0[ti].cpu().numpy(), z1[ti].cpu().numpy(), x0[ti].cpu().numpy()
    del z0, z1, x0, buf, ti
    torch.cuda.empty_cache()
    want = (((idx * 40503) % 65536).astype(np.float32) * np.float32(160.0 / 65536) - np.float32(80.0))
    assert np.array_equal(hx.view(np.int32), want.view(np.int32)), "device inputs differ from the host formula"
    orc = oracle.evaluate("texp", want.astype(np.float64), None, dtype="f32")
    st = tfcheck.check(h0.astype(np.float64), h1.astype(np.float64), orc, "f32", 0.99999,
                       f"texpf n=2^31+7 aligned={aligned}")
    print(aligned, st)
