"""Coupled results (pexp, pexpm1, plog, plog1p) and twofold results of coupled
arguments (texpp, texpm1p, tlogp, tlog1pp) through the C ABI, against the oracle.

* p-functions: z0 + z1 is exactly the twofold function's value (itself
  parity-tested) with z0 = RN(z0 + z1); z0 = RN(f(x0 + x1)) (the oracle's
  coupled answer, an exact rational renormalisation of its binary128 value)
  wherever the twofold's error bound cannot reach a rounding midpoint (z1
  carries the x1 term to 1x, so near log(1), or for subnormal results, RN(F) is
  not always decidable from the 2x value), and within one ulp everywhere; with
  x1 = NULL (pexp0, ...) the answer is the coupled f(x0).
* t...p functions on coupled arguments: the same parity as the twofold
  functions, and bitwise the twofold function's result (the renormalising path
  they skip is never needed for these arguments).
"""
import numpy as np
import pytest

import oracle
import tfcheck
from paper_1502_05216_gb300 import inputs as I

pytestmark = pytest.mark.gpu

P_FUNCS = ("pexp", "pexpm1", "plog", "plog1p")
TP_FUNCS = ("texpp", "texpm1p", "tlogp", "tlog1pp")


@pytest.fixture(scope="module")
def tf():
    import torch
    from paper_1502_05216_gb300 import build, tf as tfmod
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    build.build()
    tfmod.load()
    return tfmod


def run(fn, x0, x1):
    import torch
    d = [None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0") for a in (x0, x1)]
    z0, z1 = fn(*d)
    torch.cuda.synchronize()
    return z0.cpu().numpy(), z1.cpu().numpy()


def _args(base, n):
    x0, x1 = I.workload(base, n)
    h0, h1 = I.hard_cases(base, n // 4)
    return np.concatenate([x0, h0]), np.concatenate([x1, h1])


def _two_sum(a, b):
    """Knuth's TwoSum in numpy: s = RN(a + b) and e = a + b - s exactly."""
    s = a + b
    bp = s - a
    ap = s - bp
    return s, (a - ap) + (b - bp)


def _check_coupled(tf, func, x0, x1, where):
    base = tf.BASE_OF[func]
    z0, z1 = run(tf.FUNCS_C[func], x0, x1)
    w0, w1 = run(tf.FUNCS[base], x0, x1)       # the twofold result (parity-tested itself)
    # the renormalisation is exact: z0 + z1 = w0 + w1, z0 = RN(w0 + w1)
    fin = np.isfinite(w0) & np.isfinite(w1) & (w1 != 0)
    with np.errstate(invalid="ignore", over="ignore"):
        s, e = _two_sum(w0, w1)
    assert np.array_equal(z0[fin], s[fin]) and np.array_equal(z1[fin], e[fin]), f"{where}: not RN(w0 + w1) + rest"
    keep = ~fin
    assert np.array_equal(z0[keep].view(np.int64), w0[keep].view(np.int64)), f"{where}: special z0 changed"
    assert np.array_equal(z1[keep].view(np.int64), w1[keep].view(np.int64)), f"{where}: special z1 changed"
    # and z0 is the correctly rounded f(x0 + x1) wherever the twofold's own error
    # bound (2^-100 |F| + 2^-53 |F - f(x0)| + 2^-1074: z1 holds the deviation to
    # half its ulp plus 2^-100 |F|) cannot reach a rounding midpoint; within one
    # ulp everywhere
    twofold = oracle.evaluate(base, x0, x1)
    orc = oracle.coupled(twofold)
    rel_tol, ulp_tol, abs_tol = tfcheck.TOL["f64"]
    with np.errstate(invalid="ignore", over="ignore"):
        bound = rel_tol * twofold.A + ulp_tol * np.abs(twofold.Gh) + abs_tol
        to_mid = np.spacing(np.abs(orc.Z0)) / 2 - np.abs(orc.Gh + orc.Gl)
    decided = np.isfinite(orc.Z0) & np.isfinite(bound) & (bound < to_mid)
    ok = (z0 == orc.Z0) | (np.isnan(z0) & np.isnan(orc.Z0)) | ~decided
    assert np.count_nonzero(~ok) <= 1e-5 * x0.size, f"{where}: {np.count_nonzero(~ok)} decided main parts differ from RN(F)"
    assert np.all(tfcheck.ulp_distance(z0, orc.Z0) <= 1), f"{where}: a main part more than 1 ulp from RN(F)"
    return int(np.count_nonzero(~decided & np.isfinite(orc.Z0)))


@pytest.mark.parametrize("func", P_FUNCS)
def test_coupled_result(tf, func):
    base = tf.BASE_OF[func]
    x0, x1 = _args(base, 2**14 + 11)
    _check_coupled(tf, func, x0, x1, func)


@pytest.mark.parametrize("func", P_FUNCS)
def test_coupled_dotted(tf, func):
    base = tf.BASE_OF[func]
    x0, _ = I.workload(base, 4099)
    _check_coupled(tf, func, x0, None, func + "0")


@pytest.mark.parametrize("func", TP_FUNCS)
def test_coupled_argument(tf, func):
    base = tf.BASE_OF[func]
    x0, x1 = I.workload(base, 2**14 + 11)
    z0, z1 = run(tf.FUNCS_C[func], x0, x1)
    tfcheck.check(z0, z1, oracle.evaluate(base, x0, x1), "f64", 0.99999, func, base, (x0, x1))
    w0, w1 = run(tf.FUNCS[base], x0, x1)
    assert np.array_equal(z0.view(np.int64), w0.view(np.int64)), f"{func}: z0 differs from {base}"
    assert np.array_equal(z1.view(np.int64), w1.view(np.int64)), f"{func}: z1 differs from {base}"
