"""Per-function accuracy against the binary128 oracle, double and float.

For every twofold function, on its workload (2^20 elements) and on its hard
cases (2^16), the parity bar is asserted (tests/tfcheck.py) and one table row is
printed (run with -s to see it):

  main-part mismatches (z0 != RN(f(x0))), max and mean of |z0 + z1 - F| / |F|,
  the largest error beyond half an ulp of z1 (what the method adds to z1's own
  rounding), and how many elements exceed 2^-100 (2^-44 for float) in total
  relative error -- z1 is one double, so a large deviation G alone can put
  half an ulp of z1 above that line (the tolerance's 2^-52 |G| term).

Statistics cover results whose z1 is a normal number, as the paper's do.
"""
import numpy as np
import pytest

import oracle
import tfcheck
from paper_1502_05216_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DOUBLE = ("texp", "texpm1", "tlog", "tlog1p", "tadd", "tmul")
FLOAT = ("texp", "texpm1", "tlog", "tlog1p")


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
          f"2^{st['mean_rel_log2']:.1f} | 2^{st['max_excess_rel_log2']:.1f} | {st['beyond_rel_tol']} |")


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
