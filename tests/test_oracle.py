"""The CPU oracle against its pins (no GPU)."""
import pytest

import oracle
import oracle_pins as P


@pytest.fixture(scope="module")
def lib():
    return oracle.load()


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(lib, pin):
    fails = pin(lib)
    assert not fails, f"{len(fails)} failures, e.g. {fails[:5]}"


def test_golden_constants_match_decimal():
    import decimal
    g = P.golden_constants()
    c = decimal.Context(prec=80)
    assert abs(g["ln2"] - c.ln(decimal.Decimal(2))) < decimal.Decimal(10) ** -78
    assert abs(g["e"] - c.exp(decimal.Decimal(1))) < decimal.Decimal(10) ** -78


def test_oracle_parallel_equals_serial(lib):
    """The OpenMP loop must not change any answer."""
    import numpy as np
    from paper_1502_05216_gb300 import inputs as I
    x0, x1 = I.exp_args(20000, 170)
    t = oracle.threads()
    a = oracle.evaluate("texp", x0, x1, lib=lib)
    oracle.set_threads(1)
    try:
        b = oracle.evaluate("texp", x0, x1, lib=lib)
    finally:
        oracle.set_threads(t)
    for k in ("Z0", "Gh", "Gl", "A"):
        assert np.array_equal(getattr(a, k), getattr(b, k))
