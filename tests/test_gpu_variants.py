"""The A/B variants against the oracle, with the same bar as the function each
computes (z0 correctly rounded in >= 99.999% and never more than 1 ulp off,
z0 + z1 within half an ulp of the ideal deviation plus 2^-100 |F|, the
special-value rules bitwise), on that function's workload, its hard cases,
every pairing of the IEEE specials, dotted arguments and small ragged sizes;
their main parts equal the default kernels' bitwise:

  * tf_texp_tables: texp through the paper's own table reduction (Function
    pexp0(): x = 2^L m + 2^-K n + y), also on the uniform texp configuration;
  * tf_tlog_newton_fp64, tf_tlog1p_newton_fp64: tlog and tlog1p with the
    Newton step in binary64 ("Twofold logarithm" > "Newton inversion"), also
    on the log edge cases (cell borders, near 1, near -1, tiny and huge)."""
import numpy as np
import pytest

import oracle
import tfcheck
from paper_1502_05216_gb300 import inputs as I

pytestmark = pytest.mark.gpu

VARIANTS = ("texp_tables", "tlog_newton_fp64", "tlog1p_newton_fp64")


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


def check(tf, var, args, where, rate=0.99999):
    fn, base = tf.VARIANT_FUNCS[var]
    x0, x1 = args
    z0, z1 = run(fn, x0, x1)
    st = tfcheck.check(z0, z1, oracle.evaluate(base, x0, x1), "f64", rate, where, base, args)
    w0, _ = run(tf.FUNCS[base], x0, x1)
    same = (z0 == w0) | (np.isnan(z0) & np.isnan(w0))
    assert np.count_nonzero(~same) <= (1 - rate) * x0.size, f"{where}: main part differs from tf_{base}"
    return st


@pytest.mark.parametrize("var", VARIANTS)
def test_variant_workload(tf, var):
    base = tf.VARIANT_FUNCS[var][1]
    print(check(tf, var, I.workload(base, 2**17 + 37), f"{var} workload"))


def test_tables_uniform_config(tf):
    print(check(tf, "texp_tables", I.texp_uniform(2**18, 0), "texp_tables uniform 2^18"))


@pytest.mark.parametrize("var", VARIANTS)
def test_variant_hard_cases(tf, var):
    base = tf.VARIANT_FUNCS[var][1]
    print(check(tf, var, I.hard_cases(base, 2**16), f"{var} hard cases"))


@pytest.mark.parametrize("var", VARIANTS)
def test_variant_special_values(tf, var):
    s = I.SPECIALS
    check(tf, var, (np.repeat(s, s.shape[0]), np.tile(s, s.shape[0])), f"{var} specials", rate=1.0)


@pytest.mark.parametrize("var", VARIANTS)
@pytest.mark.parametrize("n", [1, 3, 33, 257])
def test_variant_small_sizes(tf, var, n):
    base = tf.VARIANT_FUNCS[var][1]
    check(tf, var, I.workload(base, n, start=1000), f"{var} n={n}")


@pytest.mark.parametrize("var", VARIANTS)
def test_variant_dotted(tf, var):
    fn, base = tf.VARIANT_FUNCS[var]
    x0, _ = I.workload(base, 4099)
    z0, z1 = run(fn, x0, None)
    tfcheck.check(z0, z1, oracle.evaluate(base, x0, None), "f64", 0.99999, f"{var} dotted", base, (x0, None))


@pytest.mark.parametrize("var", ("tlog_newton_fp64", "tlog1p_newton_fp64"))
def test_newton_fp64_log_edges(tf, var):
    """The log edge cases of test_gpu_log_edges (table-cell borders, the z split,
    near 1 and -1, tiny and huge arguments) through the binary64 Newton step."""
    import test_gpu_log_edges as E
    base = tf.VARIANT_FUNCS[var][1]
    x0, x1 = E.tlog_edges() if base == "tlog" else E.tlog1p_edges()
    check(tf, var, (x0, x1), f"{var} edges", rate=0.9999)
