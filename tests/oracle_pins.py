"""Pins of the CPU oracle against things other than itself.

Each ``pin_*`` function runs one family of checks against an oracle library
handle and returns a list of failure strings (empty = pinned).  They are used
twice: ``test_oracle.py`` asserts that the real oracle passes all of them, and
``test_oracle_planted.py`` builds oracles with planted mistakes and asserts
that each is caught by at least one pin.

What the oracle is pinned to:
  * Python's ``decimal`` module at 60+ significant digits (an independent
    arbitrary-precision exp/ln) for the main part Z0 and the full value F;
  * exact rational arithmetic (``fractions``) for tadd/tmul and for the
    Taylor series of expm1/log1p near 0;
  * closed forms: exp(0) = 1, expm1(+-0) = +-0, log(1) = 0, log1p(+-0) = +-0,
    exp(twofold k ln 2) = 2^k, log(2^k) = k ln 2 (ln 2 from tests/golden);
  * invariants: monotonicity of Z0, exp(x) exp(-x) = 1, Z0 independent of x1,
    log(exp(x)) = x, log1p(y) = log(1 + y) when 1 + y is exact;
  * the special-value rules (NaN, infinities, overflow/underflow);
  * arguments whose f(x0) lies next to a rounding midpoint, from the Taylor
    series (the binary128 step flags them and a decimal re-decision runs),
    and the re-decision and rounding helpers on constructed cases.
"""
from __future__ import annotations

import decimal
import math
import os
from fractions import Fraction

import numpy as np

import oracle
from paper_1502_05216_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
UNARY = ("texp", "texpm1", "tlog", "tlog1p")


def _hiprec(fn):
    """Run a pin with a 120-digit decimal context, so that plain operators on
    Decimals (not only the explicit context calls) keep full precision."""
    import functools

    @functools.wraps(fn)
    def run(*a, **k):
        with decimal.localcontext(decimal.Context(prec=120, Emax=999999, Emin=-999999)):
            return fn(*a, **k)
    return run


def golden_constants():
    out = {}
    with open(os.path.join(GOLDEN, "constants.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out[k] = decimal.Decimal(v)
    return out


def _ctx(digits=60):
    return decimal.Context(prec=digits + 40, Emax=999999, Emin=-999999)


def dec_eval(func: str, d: decimal.Decimal, digits=60) -> decimal.Decimal:
    """f(d) in decimal for an exact decimal argument d (independent of the oracle)."""
    c = _ctx(digits)
    if func == "texp":
        return c.exp(d)
    if func == "texpm1":
        if abs(d) < decimal.Decimal("1e-3"):
            term, s, k = d, d, 1
            while True:
                k += 1
                term = c.divide(c.multiply(term, d), k)
                if term == 0 or abs(term) < abs(s) * decimal.Decimal(10) ** -(digits + 20):
                    return s
                s = c.add(s, term)
        return c.subtract(c.exp(d), 1)
    if func == "tlog":
        return c.ln(d)
    if func == "tlog1p":
        return c.ln(c.add(d, 1))
    raise KeyError(func)


def _D(x):
    return decimal.Decimal(float(x))


def _u(seed, n, stream=0):
    return I.uniform(seed, stream, n)


def mainpart_points():
    """Argument sets per function: the workloads plus the awkward ranges."""
    n = 150
    pts = {}
    x = [I.exp_args(n, 100)[0], I.texp_uniform(n, 101)[0],
         -745.13 + (745.13 - 708.40) * _u(102, 60),          # subnormal results
         709.70 + 0.0827 * _u(103, 30), np.array([1.0, -1.0, 0.5, 1e-300, -1e-300])]
    pts["texp"] = np.concatenate(x)
    x = [I.exp_args(n, 110)[0], -40.0 + 39.0 * _u(111, 40),
         np.exp2(-60 + 40 * _u(112, 40)) * np.where(_u(113, 40) < 0.5, -1, 1), np.array([1.0, -1.0])]
    pts["texpm1"] = np.concatenate(x)
    x = [I.log_args(n, 120)[0], 1.0 + np.exp2(-52 + 50 * _u(121, 40)) * np.where(_u(122, 40) < 0.5, -1, 1),
         np.exp2(-1074 + 52 * _u(123, 30)), np.array([2.0, 0.5, 10.0, 5e-324, 1.7976931348623157e308])]
    pts["tlog"] = np.concatenate(x)
    x = [I.log1p_args(n, 130)[0], -1.0 + np.exp2(-52 + 51 * _u(131, 40)),
         np.exp2(-60 + 40 * _u(132, 40)) * np.where(_u(133, 40) < 0.5, -1, 1), np.array([1.0, -0.5, 1e300])]
    pts["tlog1p"] = np.concatenate(x)
    return pts


@_hiprec
def pin_mainpart_decimal(lib):
    """Z0 equals the decimal value rounded to the nearest double."""
    fails = []
    for func, x0 in mainpart_points().items():
        r = oracle.evaluate(func, x0, None, lib=lib)
        for i, x in enumerate(x0):
            want = oracle.round_to_double(dec_eval(func, _D(x)))
            if not (r.Z0[i] == want or (math.isnan(want) and math.isnan(r.Z0[i]))):
                fails.append(f"{func}({x!r}): Z0={r.Z0[i]!r} decimal={want!r}")
    return fails


def _close(G_h, G_l, G_dec, F_dec, rel=decimal.Decimal(2) ** -104):
    c = _ctx(80)
    diff = abs(c.subtract(c.add(_D(G_h), _D(G_l)), G_dec))
    return diff <= rel * abs(F_dec) + decimal.Decimal(2) ** -1074


@_hiprec
def pin_deviation_decimal(lib):
    """Gh + Gl equals F - Z0 with F = f(x0 + x1) evaluated in decimal from the
    exact sum x0 + x1 (coupled and loosely coupled x1)."""
    fails = []
    pts = mainpart_points()
    for func in UNARY:
        x0 = pts[func]
        # skip arguments whose result is not a finite nonzero value
        for scale, seed in ((2.0**-53, 140), (2.0**-30, 141)):
            x1 = x0 * (2 * _u(seed, x0.shape[0]) - 1) * scale
            r = oracle.evaluate(func, x0, x1, lib=lib)
            c = _ctx(80)
            for i in range(x0.shape[0]):
                if r.flags[i] & oracle.FL_EXACT:
                    continue
                d = c.add(_D(x0[i]), _D(x1[i]))
                if func == "tlog" and d <= 0 or func == "tlog1p" and d <= -1:
                    continue
                F = dec_eval(func, d, 70)
                G = c.subtract(F, _D(r.Z0[i]))
                if not _close(r.Gh[i], r.Gl[i], G, F):
                    fails.append(f"{func}({x0[i]!r}+{x1[i]!r}): G={r.Gh[i]!r}+{r.Gl[i]!r} decimal={G:.6e}")
    return fails


@_hiprec
def pin_closed_forms(lib):
    fails = []
    ln2 = golden_constants()["ln2"]
    c = _ctx(80)
    # exp(0) = 1 and expm1(+-0) = +-0, log(1) = 0, log1p(+-0) = +-0, z1 = 0
    for func, x, want in (("texp", 0.0, 1.0), ("texpm1", 0.0, 0.0), ("texpm1", -0.0, -0.0),
                          ("tlog", 1.0, 0.0), ("tlog1p", 0.0, 0.0), ("tlog1p", -0.0, -0.0)):
        r = oracle.evaluate(func, np.array([x]), np.array([0.0]), lib=lib)
        if not (r.Z0[0] == want and math.copysign(1, r.Z0[0]) == math.copysign(1, want)
                and r.Gh[0] == 0 and r.Gl[0] == 0):
            fails.append(f"{func}({x}) = {r.Z0[0]!r} + {r.Gh[0]!r}, want {want!r} + 0")
    # exp of the twofold k*ln2 is 2^k to 2^-100; log(2^k) is k*ln2 to 2^-100
    ks = np.arange(-1000, 1001, 7)
    x0 = np.array([float(k * ln2) for k in ks])
    x1 = np.array([float(c.subtract(k * ln2, _D(a))) for k, a in zip(ks, x0)])
    r = oracle.evaluate("texp", x0, x1, lib=lib)
    for i, k in enumerate(ks):
        v = c.add(c.add(_D(r.Z0[i]), _D(r.Gh[i])), _D(r.Gl[i]))
        delta = _D(x0[i]) + _D(x1[i]) - k * ln2   # |delta| <= 2^-97: e^delta = 1 + delta + O(2^-195)
        want = c.power(2, int(k)) * (1 + delta)
        if abs(v - want) > want * decimal.Decimal(2) ** -100 + decimal.Decimal(2) ** -1073:
            fails.append(f"texp({k} ln2) = {v:.30e}, want 2^{k}")
    ks = np.arange(-1074, 1024, 5)
    y0 = np.array([math.ldexp(1.0, int(k)) for k in ks])
    r = oracle.evaluate("tlog", y0, np.zeros_like(y0), lib=lib)
    for i, k in enumerate(ks):
        v = c.add(c.add(_D(r.Z0[i]), _D(r.Gh[i])), _D(r.Gl[i]))
        want = k * ln2
        if abs(v - want) > abs(want) * decimal.Decimal(2) ** -100:
            fails.append(f"tlog(2^{k}) = {v:.30e}, want {want:.30e}")
    return fails


def _series(func, x: Fraction, terms=7):
    s, p = Fraction(0), Fraction(1)
    for j in range(1, terms + 1):
        p = p * x
        if func == "texpm1":
            s += p / math.factorial(j)
        else:
            s += (-1) ** (j + 1) * p / j
    return s


@_hiprec
def pin_series(lib):
    """expm1 and log1p near 0 against their Taylor series in exact rationals."""
    fails = []
    x0 = np.exp2(-90 + 70 * _u(150, 200)) * np.where(_u(151, 200) < 0.5, -1, 1)
    for func in ("texpm1", "tlog1p"):
        r = oracle.evaluate(func, x0, np.zeros_like(x0), lib=lib)
        for i, x in enumerate(x0):
            S = _series(func, Fraction(float(x)))
            if float(S) != r.Z0[i]:
                fails.append(f"{func}({x!r}) Z0={r.Z0[i]!r} series={float(S)!r}")
            got = Fraction(float(r.Z0[i])) + Fraction(float(r.Gh[i])) + Fraction(float(r.Gl[i]))
            if abs(got - S) > abs(S) * Fraction(1, 2**104):
                fails.append(f"{func}({x!r}) Z0+G off the series by {float(abs(got - S) / abs(S)):.3e}")
    return fails


@_hiprec
def pin_invariants(lib):
    fails = []
    # Z0 monotone in x0
    for func, gen in (("texp", I.exp_args), ("texpm1", I.exp_args), ("tlog", I.log_args),
                      ("tlog1p", I.log1p_args)):
        x0 = np.sort(gen(4000, 160)[0])
        r = oracle.evaluate(func, x0, None, lib=lib)
        if np.any(np.diff(r.Z0) < 0):
            fails.append(f"{func}: Z0 not monotone")
    # main part independent of x1
    x0, x1 = I.exp_args(2000, 161)
    for func in ("texp", "texpm1"):
        a = oracle.evaluate(func, x0, None, lib=lib)
        b = oracle.evaluate(func, x0, x1 * 2.0**20, lib=lib)
        if not np.array_equal(a.Z0, b.Z0):
            fails.append(f"{func}: Z0 depends on x1")
    # exp(x) exp(-x) = 1
    x0 = (2 * _u(162, 300) - 1) * 600  # e^-x stays well above the subnormal range
    p = oracle.evaluate("texp", x0, None, lib=lib)
    m = oracle.evaluate("texp", -x0, None, lib=lib)
    for i in range(x0.shape[0]):
        a = Fraction(float(p.Z0[i])) + Fraction(float(p.Gh[i])) + Fraction(float(p.Gl[i]))
        b = Fraction(float(m.Z0[i])) + Fraction(float(m.Gh[i])) + Fraction(float(m.Gl[i]))
        if abs(a * b - 1) > Fraction(1, 2**102):
            fails.append(f"texp({x0[i]!r}) * texp(-x) - 1 = {float(a * b - 1):.3e}")
    # log(exp(x)) = x, with exp(x) as the twofold (Z0, Gh)
    x0 = np.exp2(-4 + 13 * _u(163, 300)) * np.where(_u(164, 300) < 0.5, -1, 1)
    e = oracle.evaluate("texp", x0, None, lib=lib)
    l = oracle.evaluate("tlog", e.Z0, e.Gh, lib=lib)
    for i in range(x0.shape[0]):
        v = Fraction(float(l.Z0[i])) + Fraction(float(l.Gh[i])) + Fraction(float(l.Gl[i]))
        if abs(v - Fraction(float(x0[i]))) > abs(Fraction(float(x0[i]))) * Fraction(1, 2**100):
            fails.append(f"tlog(texp({x0[i]!r})) = {float(v)!r}")
    # log1p(y) = log(1 + y) when 1 + y is exact
    y = np.ldexp(np.floor(_u(165, 300) * 2**20), -18) - 0.5  # multiples of 2^-18 in [-0.5, 3.5)
    a = oracle.evaluate("tlog1p", y, None, lib=lib)
    b = oracle.evaluate("tlog", 1.0 + y, None, lib=lib)
    if not np.array_equal(a.Z0, b.Z0):
        fails.append("tlog1p(y) main part != tlog(1 + y) main part")
    d = np.abs((a.Gh - b.Gh) + (a.Gl - b.Gl))
    if np.any(d > np.abs(a.Z0) * 2.0**-104):
        fails.append("tlog1p(y) deviation != tlog(1 + y) deviation")
    return fails


@_hiprec
def pin_special(lib):
    """The special-value rules (NaN, infinities, overflow, underflow, domain)."""
    inf, nan = math.inf, math.nan
    cases = [  # func, x0, x1, Z0, z1
        ("texp", nan, 0.0, nan, nan), ("texp", 1.0, nan, math.e, nan),
        ("texp", inf, 0.0, inf, 0.0), ("texp", -inf, 0.0, 0.0, 0.0),
        ("texp", 710.0, 1e-300, inf, 0.0), ("texp", -746.0, 0.0, 0.0, 0.0),
        ("texp", 1.0, inf, math.e, inf),
        ("texpm1", -inf, 0.0, -1.0, 0.0), ("texpm1", inf, 0.0, inf, 0.0),
        ("texpm1", 710.0, 0.0, inf, 0.0), ("texpm1", nan, 0.0, nan, nan),
        ("tlog", -1.0, 0.0, nan, nan), ("tlog", 0.0, 0.0, -inf, 0.0), ("tlog", -0.0, 0.0, -inf, 0.0),
        ("tlog", inf, 0.0, inf, 0.0), ("tlog", 1.0, nan, 0.0, nan), ("tlog", nan, 0.0, nan, nan),
        ("tlog", 1.0, -2.0, 0.0, nan), ("tlog", 1.0, -1.0, 0.0, -inf), ("tlog", 2.0, inf, math.log(2), inf),
        ("tlog1p", -1.0, 0.0, -inf, 0.0), ("tlog1p", -2.0, 0.0, nan, nan), ("tlog1p", inf, 0.0, inf, 0.0),
        ("tlog1p", 0.0, -1.0, 0.0, -inf), ("tlog1p", 0.0, -3.0, 0.0, nan),
    ]
    fails = []
    for func, x0, x1, Z0, z1 in cases:
        r = oracle.evaluate(func, np.array([x0]), np.array([x1]), lib=lib)
        okz = (r.Z0[0] == Z0) or (math.isnan(Z0) and math.isnan(r.Z0[0]))
        okg = bool(r.flags[0] & oracle.FL_EXACT) and ((r.Gh[0] == z1) or (math.isnan(z1) and math.isnan(r.Gh[0])))
        if not (okz and okg):
            fails.append(f"{func}({x0}, {x1}) = ({r.Z0[0]}, {r.Gh[0]}, flags {r.flags[0]}), want ({Z0}, {z1})")
    return fails


@_hiprec
def pin_arith(lib):
    """tadd/tmul: Z0 is the plain double op; Gh + Gl is the exact deviation."""
    fails = []
    x0, x1, y0, y1 = I.workload("tadd", 400, 0)
    for func, op in (("tadd", lambda a, b: a + b), ("tmul", lambda a, b: a * b)):
        r = oracle.evaluate(func, x0, x1, y0, y1, lib=lib)
        if not np.array_equal(r.Z0, op(x0, y0)):
            fails.append(f"{func}: Z0 is not the plain double op")
        for i in range(x0.shape[0]):
            X = Fraction(float(x0[i])) + Fraction(float(x1[i]))
            Y = Fraction(float(y0[i])) + Fraction(float(y1[i]))
            F = op(X, Y)
            G = F - Fraction(float(r.Z0[i]))
            got = Fraction(float(r.Gh[i])) + Fraction(float(r.Gl[i]))
            scale = abs(F) if func == "tmul" else abs(X) + abs(Y)
            if abs(got - G) > scale * Fraction(1, 2**104):
                fails.append(f"{func}[{i}]: G={float(got)!r}, exact {float(G)!r}")
    return fails


@_hiprec
def pin_cancellation(lib):
    """Twofold arguments whose parts cancel: 1 + y0 + y1 (log1p) or y0 + y1 (log)
    far below the parts, including a y0 that 1 + y0 would round away, and exp
    arguments whose parts are far apart or huge.  The exact sum comes from
    rationals, its log or exp from decimal."""
    dbl_max = 1.7976931348623157e308
    cases = [("tlog1p", 5e-324, -1.0), ("tlog1p", 2.0**-60, -1.0), ("tlog1p", dbl_max, -dbl_max),
             ("tlog1p", 0.75, -1.5), ("tlog1p", -0.5, -0.25), ("tlog1p", 2.0**-30, -1.0 + 2.0**-40),
             ("tlog", 1.0, -0.75), ("tlog", 3.0, -2.9999999999999996), ("tlog", 2.0**-1000, -2.0**-1001),
             ("texpm1", -dbl_max, dbl_max * 2.0**-60), ("texpm1", -800.0, 799.5)]
    fails = []
    c = _ctx(80)
    for func, y0, y1 in cases:
        r = oracle.evaluate(func, np.array([y0]), np.array([y1]), lib=lib)
        s = (Fraction(1) if func == "tlog1p" else Fraction(0)) + Fraction(y0) + Fraction(y1)
        sd = c.divide(decimal.Decimal(s.numerator), decimal.Decimal(s.denominator))
        F = c.ln(sd) if func in ("tlog", "tlog1p") else c.exp(sd) - (1 if func == "texpm1" else 0)
        got = c.add(c.add(_D(r.Z0[0]), _D(r.Gh[0])), _D(r.Gl[0]))
        if got.is_nan() or abs(got - F) > abs(F) * decimal.Decimal(2) ** -104:
            fails.append(f"{func}({y0!r} + {y1!r}) = {got:.25e}, want {F:.25e}")
    return fails


def mainpart_points_f32():
    """Float arguments per function: the float workloads plus the thresholds."""
    n = 120
    pts = {}
    for func in UNARY:
        pts[func] = [I.workload_f32(func, n, start=500)[0], I.hard_cases_f32(func, 100, seed=150)[0][:90]]
    pts["texp"].append(np.float32([88.72283, 88.72284, -103.97207, -103.97208, -87.33654, 0.0, 1.0]))
    pts["tlog"].append(np.float32([1.0, 2.0, 0.5, 1.0000001, 0.99999994, 2.0**-149, 3.4028235e38]))
    pts["tlog1p"].append(np.float32([-0.99999994, 1e-30, -1e-30, 1.0, 3.4028235e38]))
    pts["texpm1"].append(np.float32([1e-30, -1e-30, -88.0, 88.7, 0.3465736]))
    out = {}
    for func, parts in pts.items():
        x = np.concatenate(parts).astype(np.float64)
        out[func] = x[np.isfinite(x)]
    return out


@_hiprec
def pin_mainpart_decimal_f32(lib):
    """Float twofolds: Z0 equals the decimal value rounded to the nearest float."""
    fails = []
    for func, x0 in mainpart_points_f32().items():
        r = oracle.evaluate(func, x0, None, lib=lib, dtype="f32")
        for i, x in enumerate(x0):
            if func == "tlog" and x < 0 or func == "tlog1p" and x < -1:
                continue
            want = oracle.round_to_float(dec_eval(func, _D(x)))
            if not (r.Z0[i] == want or (math.isnan(want) and math.isnan(r.Z0[i]))):
                fails.append(f"{func}f({x!r}): Z0={r.Z0[i]!r} decimal={want!r}")
    return fails


@_hiprec
def pin_deviation_decimal_f32(lib):
    """Float twofolds: Gh + Gl equals F - Z0, F = f(x0 + x1) in decimal."""
    fails = []
    c = _ctx(80)
    for func, x0 in mainpart_points_f32().items():
        x1 = (x0 * (2 * _u(160, x0.shape[0]) - 1) * 2.0**-24).astype(np.float32).astype(np.float64)
        r = oracle.evaluate(func, x0, x1, lib=lib, dtype="f32")
        for i in range(x0.shape[0]):
            if r.flags[i] & oracle.FL_EXACT:
                continue
            d = c.add(_D(x0[i]), _D(x1[i]))
            if func == "tlog" and d <= 0 or func == "tlog1p" and d <= -1:
                continue
            F = dec_eval(func, d, 70)
            G = c.subtract(F, _D(r.Z0[i]))
            if not _close(r.Gh[i], r.Gl[i], G, F):
                fails.append(f"{func}f({x0[i]!r}+{x1[i]!r}): G={r.Gh[i]!r}+{r.Gl[i]!r} decimal={G:.6e}")
    return fails


def _chain_batch(ops_list, a_list, s_init):
    """A step-major batch (include/tf.h layout) from per-chain lists of op codes,
    operands (a0, a1) and initial states (s0, s1); chains must be given
    longest first."""
    n = len(ops_list)
    L = np.array([len(o) for o in ops_list], dtype=np.int32)
    assert np.all(np.diff(L) <= 0)
    max_len = int(L.max())
    active = [int(np.sum(L > t)) for t in range(max_len)]
    sb = np.zeros(max_len + 1, dtype=np.int64)
    sb[1:] = np.cumsum(active)
    ops = np.zeros(int(sb[-1]), dtype=np.uint8)
    a0 = np.zeros(int(sb[-1]))
    a1 = np.zeros(int(sb[-1]))
    for c in range(n):
        for t, op in enumerate(ops_list[c]):
            k = sb[t] + c
            ops[k] = op
            a0[k], a1[k] = a_list[c][t]
    s0 = np.array([s[0] for s in s_init])
    s1 = np.array([s[1] for s in s_init])
    return {"ops": ops, "a0": a0, "a1": a1, "step_base": sb, "length": L, "s0": s0, "s1": s1,
            "max_len": max_len}


@_hiprec
def pin_chain_decimal(lib):
    """Chains of the batched workload (short ones) against the same operations
    applied in 80-digit decimal arithmetic to the exact inputs: the oracle's F
    must agree to 2^-100 K relative (binary128 makes ~2^-112 per operation)."""
    b = I.chains(300, seed=171, mean_len=8.0, cap=40)
    Fh, Fl, K = oracle.chain(b, lib=lib)
    ctx = _ctx(80)
    fails = []
    for c in range(b["s0"].shape[0]):
        s = _D(b["s0"][c]) + _D(b["s1"][c])
        for t in range(int(b["length"][c])):
            k = int(b["step_base"][t]) + c
            op = int(b["ops"][k])
            a = _D(b["a0"][k]) + _D(b["a1"][k])
            s = (s + a) if op == 0 else (s * a) if op == 1 else ctx.exp(s) if op == 2 else ctx.ln(s)
        F = _D(Fh[c]) + _D(Fl[c])
        if abs(F - s) > abs(s) * decimal.Decimal(2) ** -100 * decimal.Decimal(K[c]):
            fails.append((c, float(F), float(s)))
    return fails


def pin_chain_condition(lib):
    """The condition sum K in closed form (k <- gain k + 1 per operation): one
    operation gives K = 1; exp then log gives 1/|log e^s| + 1 = 1/|s| + 1; an
    add then a product gives 1 * 1 + 1 = 2.  And the values: log(exp(s)) = s,
    (s + a) b and s b exactly."""
    s = 0.75
    b = _chain_batch([[2, 3], [0, 1], [1], [2], [3]],
                     [[(0.0, 0.0), (0.0, 0.0)], [(0.25, 0.0), (3.0, 0.0)], [(2.0, 0.0)], [(0.0, 0.0)],
                      [(0.0, 0.0)]],
                     [(s, 0.0), (s, 0.0), (s, 0.0), (s, 0.0), (2.5, 0.0)])
    Fh, Fl, K = oracle.chain(b, lib=lib)
    fails = []
    want = {0: 1.0 / s + 1.0, 1: 2.0, 2: 1.0, 3: 1.0, 4: 1.0}
    for c, w in want.items():
        if abs(K[c] - w) > 1e-12 * w:
            fails.append(("K", c, K[c], w))
    if abs(Fh[0] - s) > 2.0**-110 or abs((Fh[0] - s) + Fl[0]) > 2.0**-110:
        fails.append(("log(exp(s))", Fh[0], Fl[0]))
    if Fh[1] != 3.0 or Fl[1] != 0.0:            # (0.75 + 0.25) * 3 exactly
        fails.append(("(s + a) b", Fh[1], Fl[1]))
    if Fh[2] != 1.5 or Fl[2] != 0.0:
        fails.append(("s b", Fh[2], Fl[2]))
    return fails


@_hiprec
def pin_coupled_decimal(lib):
    """oracle.coupled: Z0 is RN(f(x0 + x1)) with f evaluated in decimal from the
    exact sum x0 + x1, Gh + Gl the remainder; for x1 = 0 the answer is
    unchanged (Z0 = RN(f(x0)) is already the coupled main part)."""
    fails = []
    pts = mainpart_points()
    c = _ctx(80)
    for func in UNARY:
        x0 = pts[func]
        r0 = oracle.evaluate(func, x0, None, lib=lib)
        c0 = oracle.coupled(r0)
        same = (c0.Z0 == r0.Z0) | (np.isnan(c0.Z0) & np.isnan(r0.Z0))
        if not np.all(same):
            fails.append(f"{func}: coupled changed Z0 of a dotted argument at {np.nonzero(~same)[0][:3]}")
        for scale, seed in ((2.0**-53, 150), (2.0**-30, 151)):
            x1 = x0 * (2 * _u(seed, x0.shape[0]) - 1) * scale
            r = oracle.coupled(oracle.evaluate(func, x0, x1, lib=lib))
            for i in range(x0.shape[0]):
                if r.flags[i] & oracle.FL_EXACT:
                    continue
                d = c.add(_D(x0[i]), _D(x1[i]))
                if func == "tlog" and d <= 0 or func == "tlog1p" and d <= -1:
                    continue
                F = dec_eval(func, d, 70)
                want = oracle.round_to_double(F)
                if not (r.Z0[i] == want or (math.isinf(want) and r.Z0[i] == want)):
                    fails.append(f"coupled {func}({x0[i]!r}+{x1[i]!r}): Z0={r.Z0[i]!r} decimal={want!r}")
                    continue
                if math.isfinite(want) and not _close(r.Gh[i], r.Gl[i], c.subtract(F, _D(want)), F):
                    fails.append(f"coupled {func}({x0[i]!r}+{x1[i]!r}): remainder {r.Gh[i]!r}+{r.Gl[i]!r}")
    return fails


# Arguments whose f(x0) lies next to the midpoint of two adjacent doubles,
# found from the Taylor series (not by search): the second-order term of the
# series lands exactly on the half spacing and the third-order term, 2^-50 of a
# spacing or less away from it, decides the rounding.  The expected main part
# is written from that reading of the series; the pin checks it against decimal
# too.  Each lies within 2^-50 of a spacing of the midpoint, so the binary128
# step flags it and the oracle's decimal re-decision runs on it.
NEAR_MIDPOINT = [
    # f, x0, RN(f(x0)): series and midpoint
    ("texp", 2.0**-53, 1.0 + 2.0**-52),            # 1 + 2^-53 + 2^-107 + ..: above the midpoint 1 + 2^-53
    ("texp", -(2.0**-54), 1.0),                    # 1 - 2^-54 + 2^-109 - ..: above the midpoint 1 - 2^-54
    ("texpm1", 2.0**-52, 2.0**-52 + 2.0**-104),    # 2^-52 + 2^-105 + 2^-158.6: above 2^-52 + 2^-105
    ("texpm1", -(2.0**-53), -(2.0**-53)),          # -2^-53 + 2^-107 - 2^-161.6: beyond -(2^-53 - 2^-107)
    ("tlog", 1.0 - 2.0**-52, -(2.0**-52 + 2.0**-104)),   # -2^-52 - 2^-105 - 2^-157.6
    ("tlog1p", -(2.0**-52), -(2.0**-52 + 2.0**-104)),    # the same value
    ("tlog1p", 2.0**-53, 2.0**-53),                # 2^-53 - 2^-107 + 2^-160.6: above 2^-53 - 2^-107
]


def _rn_double_exact(v: decimal.Decimal) -> float:
    """Nearest double of a decimal value by exact rational division (Python's
    int / int true division is correctly rounded), independent of the oracle's
    own rounding helpers."""
    f = Fraction(v)
    return f.numerator / f.denominator


def _raw(lib, func, x0, x1=None, f32=False):
    """The binary128 step alone (before any re-decision): Z0, Gh, Gl, flags."""
    import ctypes
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    x1 = None if x1 is None else np.ascontiguousarray(x1, dtype=np.float64)
    n = x0.shape[0]
    Z0, Gh, Gl, A = (np.empty(n) for _ in range(4))
    fl = np.empty(n, dtype=np.uint32)
    dp = lambda a: None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    rc = lib.tfo_eval2(oracle.KINDS[func], int(f32), n, dp(x0), dp(x1), None, None, dp(Z0), dp(Gh), dp(Gl),
                       dp(A), fl.ctypes.data_as(ctypes.POINTER(ctypes.c_uint)))
    assert rc == 0
    return Z0, Gh, Gl, fl


@_hiprec
def pin_near_midpoint(lib):
    """Arguments whose f(x0) lies within 2^-50 of a spacing of a rounding
    midpoint (NEAR_MIDPOINT): the binary128 step flags each one; the oracle's
    answer has the main part the series fixes, equal to the decimal value
    rounded by exact rational division, and Gh + Gl = F - Z0 in decimal for
    x1 = 0 and two small x1.  The re-decision itself is then checked on a
    binary128 main part that landed on the wrong side of the midpoint (one
    spacing off, with G moved to keep Z0 + G = F): it must return the right
    main part and keep Z0 + G = F (a wrong shift of G moves F by a whole
    spacing).  Finally the rounding helpers that the re-decision uses must
    round exact midpoints to even and their neighbours to nearest."""
    fails = []
    c = _ctx(80)
    for func, x, want in NEAR_MIDPOINT:
        x0 = np.array([x, x, x])
        x1 = np.array([0.0, x * 2.0**-60, -x * 2.0**-57])
        Z0c, Ghc, Glc, fl = _raw(lib, func, x0, x1)
        if not all(fl & oracle.FL_AMBIG):
            fails.append(f"{func}({x!r}): not flagged as near a midpoint")
        dec = _rn_double_exact(dec_eval(func, _D(x), 80))
        if dec != want:
            fails.append(f"{func}({x!r}): decimal rounds to {dec!r}, the series to {want!r}")
        r = oracle.evaluate(func, x0, x1, lib=lib)
        for i in range(3):
            if r.Z0[i] != want:
                fails.append(f"{func}({x!r}): Z0 = {r.Z0[i]!r}, want {want!r}")
                continue
            F = dec_eval(func, c.add(_D(x0[i]), _D(x1[i])), 70)
            if not _close(r.Gh[i], r.Gl[i], c.subtract(F, _D(want)), F):
                fails.append(f"{func}({x!r}+{x1[i]!r}): G = {r.Gh[i]!r} + {r.Gl[i]!r}")
        # a main part on the wrong side of the midpoint: the spacing step of
        # the true value's binade toward the other neighbour
        other = float(np.nextafter(want, -np.inf if dec_eval(func, _D(x), 80) < _D(want) else np.inf))
        other = other if other != want else float(np.nextafter(want, np.inf))
        F0 = Fraction(float(Z0c[0])) + Fraction(float(Ghc[0])) + Fraction(float(Glc[0]))
        if float(Z0c[0]) == want:
            # move the binary128 answer to the other neighbour, keeping F
            Z0s = np.array([other])
            Ghs = np.array([float(Fraction(float(Ghc[0])) + Fraction(want) - Fraction(other))])
        else:
            Z0s, Ghs = Z0c[:1].copy(), Ghc[:1].copy()
        fls = np.array([oracle.FL_AMBIG], dtype=np.uint32)
        oracle.redecide(func, x0[:1], Z0s, Ghs, fls)
        F1 = Fraction(float(Z0s[0])) + Fraction(float(Ghs[0])) + Fraction(float(Glc[0]))
        if Z0s[0] != want:
            fails.append(f"re-decision of {func}({x!r}): Z0 = {Z0s[0]!r}, want {want!r}")
        if abs(F1 - F0) > abs(F0) * Fraction(1, 2**100):
            fails.append(f"re-decision of {func}({x!r}) moved Z0 + G by {float(F1 - F0)!r}")
    # rounding helpers: exact midpoints go to even, a hair off goes to nearest
    # (the decimal sums below are exact at 2000 digits: a subnormal double has
    # up to 751 significant digits)
    with decimal.localcontext(decimal.Context(prec=2000, Emax=999999, Emin=-999999)):
        fails += _rounding_helper_checks()
    return fails


def _rounding_helper_checks():
    fails = []
    D = decimal.Decimal
    for lo in (1.0, 1.0 + 2.0**-52, 2.0**-1074, 3 * 2.0**-1074, 0.75, 2.0**1023 * 1.5):
        hi = float(np.nextafter(lo, np.inf))
        mid = (D(lo) + D(hi)) / 2
        even = lo if (np.array(lo).view(np.int64) & 1) == 0 else hi
        eps = (D(hi) - D(lo)) * D(2) ** -60
        for sgn in (1, -1):
            for v, w in ((mid, even), (mid + eps, hi), (mid - eps, lo)):
                got = oracle.round_to_double(sgn * v)
                if got != sgn * w:
                    fails.append(f"round_to_double({sgn * v:.25e}) = {got!r}, want {sgn * w!r}")
    for lo in (np.float32(1.0), np.float32(1.0) + np.float32(2.0**-23), np.float32(2.0**-149), np.float32(0.75)):
        hi = np.nextafter(lo, np.float32(np.inf))
        mid = (D(float(lo)) + D(float(hi))) / 2
        even = lo if (np.array(lo).view(np.int32) & 1) == 0 else hi
        eps = (D(float(hi)) - D(float(lo))) * D(2) ** -60
        for sgn in (1, -1):
            for v, w in ((mid, even), (mid + eps, hi), (mid - eps, lo)):
                got = oracle.round_to_float(sgn * v)
                if got != sgn * float(w):
                    fails.append(f"round_to_float({sgn * v:.25e}) = {got!r}, want {sgn * float(w)!r}")
    if oracle.round_to_double(D(2) ** 1024 - D(2) ** 970) != math.inf:
        fails.append("round_to_double: 2^1024 - 2^970 must overflow")
    if oracle.round_to_double(D(2) ** 1024 - D(2) ** 970 - 1) != 1.7976931348623157e308:
        fails.append("round_to_double: just below 2^1024 - 2^970 must give the largest double")
    return fails


ALL_PINS = [pin_mainpart_decimal, pin_deviation_decimal, pin_closed_forms, pin_series,
            pin_invariants, pin_special, pin_arith, pin_cancellation, pin_chain_decimal,
            pin_chain_condition, pin_mainpart_decimal_f32, pin_deviation_decimal_f32,
            pin_coupled_decimal, pin_near_midpoint]
