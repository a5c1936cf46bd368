"""Per-function accuracy against the binary128 oracle, double and float.

For every twofold function, on its workload (2^20 elements) and on its hard
cases (2^16), the parity bar is asserted (tests/tfcheck.py: every element
within half an ulp of the ideal deviation G plus 2^-100 |F|, 2^-44 for float),
and the paper's own acceptance thresholds (Analysis > Accuracy, stored in
tests/golden/paper_thresholds.txt) are asserted on the error the method adds
beyond z1's own rounding (the "excess", relative to |F|): its mean within the
average (L1) threshold and at most 2 elements per million above the maximal
(L0) one.  One table row per set is printed (run with -s to see it):

  main-part mismatches (z0 != RN(f(x0))), max and mean of |z0 + z1 - F| / |F|,
  max and mean of the excess, and how many elements exceed the relative term
  (2^-100, 2^-44 float) in total error -- z1 is one double, so a large
  deviation G alone can put half an ulp of z1 above that line -- and in excess.

Statistics cover results whose z1 is a normal number, as the paper's do.
"""
import math
import os

import numpy as np
import pytest

import oracle
import tfcheck
from paper_1502_05216_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DOUBLE = ("texp", "texpm1", "tlog", "tlog1p", "tadd", "tmul")
FLOAT = ("texp", "texpm1", "tlog", "tlog1p")
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_thresholds.txt")


def thresholds():
    out = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def paper_limits(func, dtype):
    """(L1, L0, warnings per element) for a function: the paper gives one pair
    for the exponents and one for the logarithms, per format; tadd and tmul
    take the exponents' (the stricter) pair."""
    t = thresholds()
    fam = "_log" if func in ("tlog", "tlog1p") else ""
    pre = "double" if dtype == "f64" else "float"
    return 2.0 ** t[f"{pre}{fam}_L1"], 2.0 ** t[f"{pre}{fam}_L0"], t["warnings_per_million"] * 1e-6


def assert_paper(st, func, dtype, where):
    L1, L0, warn = paper_limits(func, dtype)
    ex = st["excess"]
    over = int(np.count_nonzero(ex > L0))
    allowed = math.floor(warn * st["n"])
    assert over <= allowed, f"{where}: {over} elements beyond the paper's L0 2^{math.log2(L0):.0f} (allowed {allowed})"
    mean = float(ex.mean()) if ex.size else 0.0
    assert mean <= L1, f"{where}: mean excess 2^{math.log2(mean):.1f} above the paper's L1 2^{math.log2(L1):.0f}"


@pytest.fixture(scope="module")
def tf():
    import torch
    from paper_1502_05216_gb300 import build, tf as tfmod
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    build.build()
    tfmod.load()
    return tfmod


def _row(name, where, st):
    print(f"| {name} | {where} | {st['n']} | {st['mainpart_mismatch']} | 2^{st['max_rel_log2']:.1f} | "
          f"2^{st['mean_rel_log2']:.1f} | 2^{st['max_excess_rel_log2']:.1f} | 2^{st['mean_excess_rel_log2']:.1f} | "
          f"{st['beyond_rel_tol']} | {st['excess_beyond_rel_tol']} |")


@pytest.mark.parametrize("func", DOUBLE)
def test_accuracy_double(tf, func):
    import torch
    sets = [("workload", I.workload(func, 1 << 20))]
    if func in FLOAT:
        sets.append(("hard cases", I.hard_cases(func, 1 << 16)))
    for where, args in sets:
        dev = [torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0") for a in args]
        z0, z1 = tf.FUNCS[func](*dev)
        torch.cuda.synchronize()
        st = tfcheck.check(z0.cpu().numpy(), z1.cpu().numpy(), oracle.evaluate(func, *args), "f64", 0.99999,
                           f"{func} {where}", func, args)
        _row(func, where, st)
        assert_paper(st, func, "f64", f"{func} {where}")


@pytest.mark.parametrize("func", FLOAT)
def test_accuracy_float(tf, func):
    import torch
    for where, (x0, x1) in (("workload", I.workload_f32(func, 1 << 20)), ("hard cases", I.hard_cases_f32(func, 1 << 16))):
        d0, d1 = (torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0") for a in (x0, x1))
        z0, z1 = tf.FUNCS_F[func](d0, d1)
        torch.cuda.synchronize()
        orc = oracle.evaluate(func, x0.astype(np.float64), x1.astype(np.float64), dtype="f32")
        st = tfcheck.check(z0.cpu().numpy().astype(np.float64), z1.cpu().numpy().astype(np.float64), orc, "f32",
                           0.99999, f"{func}f {where}")
        _row(func + "f", where, st)
        assert_paper(st, func, "f32", f"{func}f {where}")
