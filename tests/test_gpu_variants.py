"""tf_texp_tables, texp through the paper's own table reduction (A/B variant of
tf_texp), against the oracle: the same bar as tf_texp (z0 correctly rounded in
>= 99.999% and never more than 1 ulp off, z0 + z1 within 2^-100 relative, the
special-value rules bitwise), on the texp workload, the uniform configuration,
the hard cases (overflow / subnormal / underflow thresholds, tiny arguments),
every pairing of the IEEE specials and small ragged sizes.  Its main part is
bitwise tf_texp's."""
import numpy as np
import pytest

import oracle
import tfcheck
from paper_1502_05216_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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
    d = [None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to("cuda:0")
         for a in (x0, x1)]
    z0, z1 = fn(*d)
    torch.cuda.synchronize()
    return z0.cpu().numpy(), z1.cpu().numpy()


def check(tf, args, where, rate=0.99999):
    x0, x1 = args
    z0, z1 = run(tf.texp_tables, x0, x1)
    st = tfcheck.check(z0, z1, oracle.evaluate("texp", x0, x1), "f64", rate, where, "texp", args)
    w0, _ = run(tf.texp, x0, x1)
    same = (z0 == w0) | (np.isnan(z0) & np.isnan(w0))
    assert np.count_nonzero(~same) <= (1 - rate) * x0.size, f"{where}: main part differs from tf_texp"
    return st


def test_tables_workload(tf):
    print(check(tf, I.workload("texp", 2**17 + 37), "texp_tables workload"))


def test_tables_uniform_config(tf):
    print(check(tf, I.texp_uniform(2**18, 0), "texp_tables uniform 2^18"))


def test_tables_hard_cases(tf):
    print(check(tf, I.hard_cases("texp", 2**16), "texp_tables hard cases"))


def test_tables_special_values(tf):
    s = I.SPECIALS
    check(tf, (np.repeat(s, s.shape[0]), np.tile(s, s.shape[0])), "texp_tables specials", rate=1.0)


@pytest.mark.parametrize("n", [1, 3, 33, 257])
def test_tables_small_sizes(tf, n):
    check(tf, I.workload("texp", n, start=1000), f"texp_tables n={n}")


def test_tables_dotted(tf):
    x0, _ = I.workload("texp", 4099)
    z0, z1 = run(tf.texp_tables, x0, None)
    tfcheck.check(z0, z1, oracle.evaluate("texp", x0, None), "f64", 0.99999, "texp_tables dotted", "texp",
                  (x0, None))
