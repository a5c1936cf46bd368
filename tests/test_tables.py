"""The committed constant tables of the kernels (csrc/tf_tables.h) against their
mathematical definitions, recomputed here with Python's decimal module (no GPU).

The build refuses a header that differs from its generator's output; this test
checks the generator's output itself, entry by entry (every entry of the small
tables, a stride of the large ones), from the definitions stated in the kernels:

  TF_TFIX_TABLE[j]  2^(j/65536) in units 2^-127 (round to nearest)
  TF_HC_m           1/(m+1)! in units 2^-127 (m <= 4) or 2^-72;  TF_HC68_m in units 2^-68
  TF_LN2FIX         ln 2 in units 2^-128;  TF_C0 + TF_C12FIX 2^-148 = ln2/65536
  TF_CFIX136        ln2/65536 in units 2^-136
  TF_LG_m           (-1)^m / (m+1) in units 2^-62, m = 0 .. 4
  TF_LOG2T[j]       {-log c2_j in units 2^-128, C2_j = round(2^42 / (2^18 + j)), 0}
  TF_LOGT[i]        {-log c_i in units 2^-128, C_i = round(2^34 / i), c_i = C_i 2^-24 as a double}
  TF_LOGU[i]        {-log c_i in units 2^-128, C_i = ceil(2^34 / i), 0}
  TF_LOG2U[j]       {-log c2_j in units 2^-128, C2_j = ceil(2^42 / (2^18 + j)), 0}, j = 0 .. 362
  TF_PX_C[n]        e^(n/256) in units 2^-124
  TF_PX_E[m]        e^(2m) = E 2^e, E in [2^127, 2^128)
  TF_FLOGT[i]       {c = RN_float(2048/i), -log c as a float pair, c - 1}
  TF_FT / TF_FE[j]  2^(j/512) and 2^(j/512) - 1 as float pairs
  TF_FNLN2[n]       n ln2 as a float pair, n = -160 .. 140
  TF_F_C0..C2       ln2/512 split, C0 with 7 bits;  TF_F_L0..L2  ln 2 split

and replays four steps of the double kernels: the exp core's FP64 reduction
with exact rationals (exactness, and the bound on the reduced argument that
the degree-6 H assumes), that H bit for bit in integers (its error bound), the
logarithm's second table reduction in integers (its bound), and tlog's
sign-free reduction and seed in integers (signs and bounds).
"""
import decimal
import math
import os
import re
import struct

import numpy as np

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_1502_05216_gb300", "csrc", "tf_tables.h")
D = decimal.Decimal
C = decimal.Context(prec=70, Emax=99999, Emin=-99999)
SRC = open(HDR).read()
LN2 = C.ln(D(2))


def _ints(name, width):
    body = re.search(r"\b%s\[[0-9]+\]\[%d\] = \{(.*?)\};" % (name, width), SRC, re.S).group(1)
    rows = re.findall(r"\{([^}]*)\}", body)
    return [[int(v[:-3], 16) if v.startswith("0x") else int(v[:-3]) for v in (x.strip() for x in r.split(","))]
            for r in rows]


def _floats(name, width):
    body = re.search(r"\b%s\[[0-9]+\]\[%d\] = \{(.*?)\};" % (name, width), SRC, re.S).group(1)
    rows = re.findall(r"\{([^}]*)\}", body)
    return [[float.fromhex(v.strip().rstrip("f")) for v in r.split(",")] for r in rows]


def _define(name):
    return re.search(r"#define %s (.*)" % name, SRC).group(1).split("/*")[0].strip()


def _u128(text):
    lo, hi = re.findall(r"0x([0-9a-f]+)ull", text)
    return int(lo, 16) | (int(hi, 16) << 64)


def _fx(v, units):
    """round(v 2^units) as an int, ties to even."""
    return int(C.multiply(v, C.power(2, units)).to_integral_value(rounding=decimal.ROUND_HALF_EVEN))


def _f32(x):
    return float(np.float32(x))


def test_exp_table_and_constants():
    tab = _ints("TF_TFIX_TABLE", 2)
    assert len(tab) == 65537
    for j in list(range(-32768, 32769, 97)) + [-32768, -1, 0, 1, 32767, 32768]:
        lo, hi = tab[j + 32768]
        assert lo | (hi << 64) == _fx(C.power(2, C.divide(D(j), 65536)), 127), j
    fact = 1
    for m in range(10):
        fact *= m + 1
        v = C.divide(1, D(fact))
        d = _define(f"TF_HC_{m}")
        got = _u128(d) if m <= 4 else int(d.rstrip("ul").replace("0x", ""), 16)
        assert got == _fx(v, 127 if m <= 4 else 72), m
        if 3 <= m <= 6:
            assert int(_define(f"TF_HC68_{m}").rstrip("ul").replace("0x", ""), 16) == _fx(v, 68), m
    assert _u128(_define("TF_LN2FIX")) == _fx(LN2, 128)
    c0 = D(float.fromhex(_define("TF_C0")))
    c12 = C.multiply(D(_u128(_define("TF_C12FIX"))), C.power(2, -148))
    assert abs(C.subtract(C.add(c0, c12), C.divide(LN2, 65536))) < C.power(2, -148)
    assert _u128(_define("TF_CFIX136")) == _fx(C.divide(LN2, 65536), 136)
    # C0 has at most 26 significant bits (N C0 exact for |N| < 2^27)
    assert (c0 * D(2) ** 42) == int(c0 * D(2) ** 42) and c0 * D(2) ** 42 < 2**26
    assert float.fromhex(_define("TF_INV_C")) == float(C.divide(65536, LN2))
    for m in range(5):
        v = int(_define(f"TF_LG_{m}").split("0x")[1].rstrip("ul)"), 16)
        v = v - (1 << 64) if v >> 63 else v
        assert v == _fx(C.divide(D((-1) ** m), D(m + 1)), 62), m


def test_log_table():
    tab = _ints("TF_LOGT", 4)
    assert len(tab) == 725
    for i in range(724, 1449, 7):
        lo, hi, Ci, cbits = tab[i - 724]
        assert Ci == int(C.divide(D(2) ** 34, D(i)).to_integral_value(rounding=decimal.ROUND_HALF_EVEN))
        c = C.multiply(D(Ci), C.power(2, -24))
        assert D(struct.unpack("<d", struct.pack("<Q", cbits))[0]) == c
        L = lo | (hi << 64)
        L = L - (1 << 128) if L >> 127 else L
        assert L == _fx(C.minus(C.ln(c)), 128), i
        # the reduced argument stays below 2^-10.4 over the cell
        for z in (D(i) / 1024 - D(1) / 2048, D(i) / 1024 + D(1) / 2048):
            z = min(max(z, D("0.7071067811865475")), D("1.414213562373095"))
            assert abs(C.subtract(C.multiply(z, c), 1)) < D(2) ** D("-10.4")


def test_second_log_table():
    tab = _ints("TF_LOG2T", 4)
    assert len(tab) == 401 and int(_define("TF_LOG2T_HALF")) == 200
    for j in range(-200, 201):
        lo, hi, C2, zero = tab[j + 200]
        assert C2 == int(C.divide(D(2) ** 42, D(2**18 + j)).to_integral_value(rounding=decimal.ROUND_HALF_EVEN))
        assert zero == 0
        c = C.multiply(D(C2), C.power(2, -24))
        L = lo | (hi << 64)
        L = L - (1 << 128) if L >> 127 else L
        assert L == _fx(C.minus(C.ln(c)), 128), j
        # the second reduced argument stays below 2^-18.9 over the cell of t1
        for t1 in (D(j) / 2**18 - D(1) / 2**19, D(j) / 2**18 + D(1) / 2**19):
            assert abs(C.subtract(C.multiply(1 + t1, c), 1)) < D(2) ** D("-18.9")
    assert tab[200][2] == 1 << 24 and tab[200][0] == tab[200][1] == 0  # j = 0: c2 = 1


def test_paper_reduction_tables():
    ctab = _ints("TF_PX_C", 2)
    assert len(ctab) == 1023
    for n in range(-511, 512, 5):
        lo, hi = ctab[n + 511]
        assert lo | (hi << 64) == _fx(C.exp(C.divide(D(n), 256)), 124), n
    etab = _ints("TF_PX_E", 4)
    assert len(etab) == 747
    for m in range(-373, 374, 3):
        lo, hi, e, _ = etab[m + 373]
        E = lo | (hi << 64)
        e = e - (1 << 64) if e >> 63 else e
        assert (1 << 127) <= E < (1 << 128)
        v = C.multiply(D(E), C.power(2, e))
        exact = C.exp(D(2 * m))
        assert abs(C.divide(C.subtract(v, exact), exact)) < C.power(2, -127), m


def test_float_tables():
    L0, L1, L2 = (float.fromhex(_define(f"TF_F_L{k}").rstrip("f")) for k in range(3))
    assert abs(C.subtract(D(L0) + D(L1) + D(L2), LN2)) < C.power(2, -68)
    C0, C1, C2 = (float.fromhex(_define(f"TF_F_C{k}").rstrip("f")) for k in range(3))
    assert abs(C.subtract(D(C0) + D(C1) + D(C2), C.divide(LN2, 512))) <= C.power(2, -68)  # half an ulp of C2
    assert (int(D(C0) * D(2) ** 16) == D(C0) * D(2) ** 16) and int(_define("TF_F_TAB_HALF")) == 256
    for name, minus1 in (("TF_FT_TABLE", False), ("TF_FE_TABLE", True)):
        tab = _floats(name, 2)
        assert len(tab) == 513
        for j in range(-256, 257, 3):
            h, l = tab[j + 256]
            v = C.power(2, C.divide(D(j), 512)) - (1 if minus1 else 0)
            assert h == _f32(v) and abs(C.subtract(D(h) + D(l), v)) <= abs(v) * C.power(2, -47) + C.power(2, -160)
    tab = _floats("TF_FNLN2_TABLE", 2)
    assert len(tab) == 301 and int(_define("TF_FNLN2_LO").strip("()")) == -160
    for n in range(-160, 141):
        h, l = tab[n + 160]
        v = D(n) * LN2
        assert h == _f32(v) and abs(C.subtract(D(h) + D(l), v)) <= abs(v) * C.power(2, -48)
    tab = _floats("TF_FLOGT", 4)
    assert len(tab) == 1449
    for i in range(1448, 2897, 7):
        c, h, l, cm1 = tab[i - 1448]
        assert c == _f32(C.divide(2048, D(i)))
        assert D(cm1) == D(c) - 1
        L = C.minus(C.ln(D(c)))
        assert abs(C.subtract(D(h) + D(l), L)) <= abs(L) * C.power(2, -47) + C.power(2, -80)


def _fma(a, b, c):
    """RN(a b + c) for doubles, from the exact rational value."""
    from fractions import Fraction
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def test_exp_reduction_is_exact():
    """The exp core's FP64 reduction (fx_reduce) as the kernel computes it,
    replayed with exact rationals: N = RN(x 65536/ln2) from the low word of
    fma(x, INV_C, 1.5 2^52), r0 = fma(-N, C0, x) is exactly x - N C0 (no
    rounding), and r = x - N ln2/65536 stays below 2^-17.52 for x over the
    clamped range [-746, 710] (random, near the thresholds, tiny); e^x's
    non-negative form (r + ln2/65536 at N - 1 for a negative r) lies in
    [0, 2^-16.52)."""
    from fractions import Fraction
    inv_c = float.fromhex(_define("TF_INV_C"))
    c0 = float.fromhex(_define("TF_C0"))
    ln2_q = Fraction(C.multiply(LN2, C.power(2, 200)).to_integral_value()) / 2**200
    shift = float.fromhex("0x1.8p52")
    rng = np.random.default_rng(5)
    xs = list(rng.uniform(-746.0, 710.0, 4000)) + list(np.exp2(rng.uniform(-60, 9.5, 2000)) * rng.choice([-1, 1], 2000))
    xs += [-746.0, 710.0, -745.1332191019412, 709.782712893384, -708.3964185322641, 512.0, -512.0,
           511.99999999999994, 2.0**-17, -(2.0**-17), 5e-324, 0.0]
    for x in xs:
        t = _fma(x, inv_c, shift)
        n = int(t - shift)  # the low word of t, as __double2loint
        nd = float(n)
        assert nd == t - shift and abs(n) < 2**27
        r0 = _fma(-nd, c0, x)
        assert Fraction(r0) == Fraction(x) - Fraction(n) * Fraction(c0), x  # exact
        r = Fraction(x) - n * ln2_q / 65536
        assert abs(r) < Fraction(2) ** -17 * Fraction(0.6974), x  # 2^-17.52
        # e^x's form (kPos): a negative r moves to N - 1 and r + ln2/65536
        rp = r + ln2_q / 65536 if r < 0 else r
        assert 0 <= rp < Fraction(2) ** -16 * Fraction(0.6974), x  # 2^-16.52


def test_exp_core_H6_error_bound():
    """The exp core's degree-6 H(r) = (e^r - 1)/r (fx_H6) replayed bit for bit
    in Python integers (the same words, shifts and truncated products) for
    |r| < 2^-17.52 of either sign and for 0 <= r < 2^-16.52 (e^x's non-negative
    reduction), against the exact rational series: the result, in units
    2^-127, is within 2^-118 of H(r)."""
    from fractions import Fraction
    M64, M128 = (1 << 64) - 1, (1 << 128) - 1
    hc68 = {m: int(_define(f"TF_HC68_{m}").rstrip("ul").replace("0x", ""), 16) for m in range(3, 7)}
    hc = {m: _u128(_define(f"TF_HC_{m}")) for m in range(3)}

    def mulshift0(a, b):  # (a b) >> 128 from three partial products, truncated
        p = (a >> 64) * (b >> 64) + (((a >> 64) * (b & M64)) >> 64) + (((a & M64) * (b >> 64)) >> 64)
        return p & M128

    def addsub(c, t, neg):
        return (c - t if neg else c + t) & M128

    def h6(A, neg):
        a = A >> 64
        h = hc68[6]
        for m in (5, 4, 3):
            t = ((a * h) >> 64) >> 8
            h = (hc68[m] - t if neg else hc68[m] + t) & M64
        A8 = A >> 8
        rh = (((A8 >> 64) * h + (((A8 & M64) * h) >> 64)) >> 5) & M128
        H = addsub(hc[2], rh, neg)
        H = addsub(hc[1], mulshift0(A8, H), neg)
        return addsub(hc[0], mulshift0(A8, H), neg)

    rng = np.random.default_rng(6)
    cases = []
    for top, signs in ((int(2.0**-17.52 * 2.0**136), (False, True)), (int(2.0**-16.52 * 2.0**136), (False,))):
        As = [int(rng.integers(0, 1 << 62)) * (top >> 62) + int(rng.integers(0, 1 << 62)) for _ in range(3000)]
        cases += [(min(A, top - 1), neg) for A in As + [0, 1, top - 1, top // 2, 1 << 100] for neg in signs]
    worst = Fraction(0)
    for A, neg in cases:
        r = Fraction(-A if neg else A, 1 << 136)
        exact = sum(r ** m / math.factorial(m + 1) for m in range(12))
        got = Fraction(h6(A, neg), 1 << 127)
        worst = max(worst, abs(got - exact))
    assert worst < Fraction(1, 1 << 118), math.log2(worst)


def test_log_second_reduction_replay():
    """The logarithm's two table reductions (log_core, non-centre cells) replayed
    in integers for random z in [sqrt(1/2), sqrt(2)): T1 = t1 2^136 exactly
    from C_i, j = round(2^18 t1) from T1's top word as the kernel forms it, T2
    = floor(|T1| C2_j / 2^24) (signed) + (C2_j - 2^24) 2^112; then |t2| <
    2^-18.9 and T2 is within one unit of the exact ((1 + t1) c2_j - 1) 2^136."""
    from fractions import Fraction
    logt = _ints("TF_LOGT", 4)
    log2t = _ints("TF_LOG2T", 4)
    rng = np.random.default_rng(7)
    zs = rng.uniform(0.70710678118654757, 1.4142135623730949, 20000)
    for z in zs:
        z = float(z)
        i = min(max(int(round(1024 * z)), 724), 1448)
        Ci = logt[i - 724][2]
        T1 = int(Fraction(z) * Ci * 2**112) - 2**136  # t1 2^136 (exact: z has 53 bits)
        assert Fraction(z) * Ci * 2**112 - 2**136 == T1
        assert abs(T1) < 2**(136 - 10.4)
        hi = T1 >> 64  # arithmetic
        j = (hi + (1 << 53)) >> 54
        assert -200 <= j <= 200
        C2 = log2t[j + 200][2]
        pr = (abs(T1) * C2) >> 24
        T2 = (pr if T1 >= 0 else -pr) + (C2 - (1 << 24)) * 2**112
        exact = (Fraction(T1, 2**136) + 1) * Fraction(C2, 2**24) - 1
        assert abs(Fraction(T2, 2**136) - exact) <= Fraction(1, 2**136)
        assert abs(T2) < 2**(136 - 18.9), (z, j)


def test_log_rounded_up_tables():
    """The rounded-up pair of tlog's sign-free core: C = ceil(...), so that z c_i
    >= 1 over cell i = floor(1024 z) and (1 + t1) c2_j >= 1 over cell j =
    floor(2^18 t1); the reduced arguments stay below 2^-9.49 and 2^-17.97."""
    tab = _ints("TF_LOGU", 4)
    assert len(tab) == 725 and int(_define("TF_LOGU_LO")) == 724 and int(_define("TF_LOGU_HI")) == 1448
    zsplit = D(0x16A09E00000000) / D(2**52)
    for i in range(724, 1449):
        lo, hi, Ci, zero = tab[i - 724]
        assert Ci == -(-(2**34) // i) and zero == 0
        c = C.multiply(D(Ci), C.power(2, -24))
        L = lo | (hi << 64)
        L = L - (1 << 128) if L >> 127 else L
        if i % 7 == 0 or i in (724, 1023, 1024, 1448):
            assert L == _fx(C.minus(C.ln(c)), 128), i
        assert C.multiply(D(i) / 1024, c) >= 1
        assert C.subtract(C.multiply(min(D(i + 1) / 1024, zsplit), c), 1) < D(2) ** D("-9.49")
    tab2 = _ints("TF_LOG2U", 4)
    jmax = int(_define("TF_LOG2U_HI"))
    assert jmax == 362 and len(tab2) == jmax + 1
    for j in range(0, jmax + 1):
        lo, hi, C2, zero = tab2[j]
        assert C2 == -(-(2**42) // (2**18 + j)) and zero == 0 and C2 <= 1 << 24
        c = C.multiply(D(C2), C.power(2, -24))
        L = lo | (hi << 64)
        L = L - (1 << 128) if L >> 127 else L
        if j % 5 == 0 or j == jmax:
            assert L == _fx(C.minus(C.ln(c)), 128), j
        assert C.multiply(1 + D(j) / 2**18, c) >= 1
        assert C.subtract(C.multiply(1 + D(j + 1) / 2**18, c), 1) < D(2) ** D("-17.97")
    assert tab2[0][2] == 1 << 24 and tab2[0][0] == tab2[0][1] == 0  # j = 0: c2 = 1


def test_log_sign_free_reduction_replay():
    """tlog's sign-free core (log_core_up) replayed in integers as the kernel
    forms each value, for random z over the split's range [0.7071056,
    1.4142112) and every cell's ends: T1 = (Z C_i 2^59) mod 2^128 equals
    t1 2^136 exactly and lies in [0, 2^126.51); j = T1's top word >> 54 is in
    [0, 362]; T2 = floor(T1 C2_j / 2^24) - (2^24 - C2_j) 2^112 lies in [0,
    2^118.03) and within one unit of ((1 + t1) c2_j - 1) 2^136; the seed
    R = t G(t) with G = 1 - t (1/2 - t/3) in truncated 64-bit steps is within
    2^-68 of log1p(t) (t taken to 2^-71, R to 2^-69), so that the Newton
    residual u = (1 + t) e^-R - 1 is below 2^-67.9 and the u^2/2 that the step
    drops below 2^-136."""
    from fractions import Fraction
    logu = _ints("TF_LOGU", 4)
    log2u = _ints("TF_LOG2U", 4)
    LG0, LG1, LG2 = (int(_define("TF_LG_%d" % m).split("0x")[1][:16], 16) for m in range(3))
    LG1 = (1 << 64) - LG1  # TF_LG_1 is -1/2 in two's complement
    assert LG0 == 1 << 62 and LG1 == 1 << 61 and LG2 == _fx(D(1) / 3, 62)
    M128 = (1 << 128) - 1
    lo_z, hi_z = 0x16A09E00000000, 0x2D413C00000000  # Z = z 2^53 over the split's range
    rng = np.random.default_rng(11)
    Zs = [int(v) for v in rng.integers(lo_z, hi_z, 20000)]
    for i in range(724, 1449):
        Zs += [max(i << 43, lo_z), min(((i + 1) << 43) - 1, hi_z - 1)]
    Zs += [1 << 53, (1 << 53) - 1, (1 << 53) + 1]
    worst = Fraction(0)
    for Z in Zs:
        i = Z >> 43
        assert 724 <= i <= 1448
        Ci = logu[i - 724][2]
        T1 = ((Z * Ci) << 59) & M128
        exact1 = Fraction(Z * Ci, 2**77) - 1
        assert Fraction(T1, 2**136) == exact1 and 0 <= T1 < 2 ** (136 - 9.49)
        j = (T1 >> 64) >> 54
        assert 0 <= j <= 362
        C2 = log2u[j][2]
        T2 = (((T1 * C2) >> 24) - (((1 << 24) - C2) << 112)) & M128
        assert T2 < 2 ** (136 - 17.97), (Z, j)
        exact2 = (exact1 + 1) * Fraction(C2, 2**24) - 1
        assert 0 <= Fraction(T2, 2**136) - exact2 + Fraction(1, 2**136) <= Fraction(1, 2**136)
        t71 = (T2 >> 64) >> 1
        g = LG1 - ((t71 * LG2) >> 71)
        g = LG0 - ((t71 * g) >> 71)
        r69 = (t71 * g) >> 64
        t = Fraction(T2, 2**136)
        # log1p(t) by its alternating series to far beyond 2^-80 (t < 2^-17.97)
        lp = sum(Fraction((-1) ** (m + 1), m) * t**m for m in range(1, 7))
        err = abs(Fraction(r69, 2**69) - lp)
        worst = max(worst, err)
    assert worst < Fraction(1, 2**68), math.log2(worst)
