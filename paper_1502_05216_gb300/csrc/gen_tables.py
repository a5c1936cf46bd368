"""Generate tf_tables.h: the constants of the CUDA twofold exp/log kernels.

Run:  python gen_tables.py > tf_tables.h   (the build checks the file is current)

All values come from Python's decimal module at 120 significant digits.

  TF_C0     ln2/65536 rounded down to 26 significant bits, so that N*C0 is exact
      for |N| < 2^27 (argument reduction x = N ln2/65536 + r).
  TF_INV_C  65536/ln2 rounded to double.

Float twofold (float-float on the FP32 pipes) constants:
  TF_F_INV_C   512/ln2 rounded to float.
  TF_F_C0..C2  ln2/512 = C0 + C1 + C2, C0 with 7 significant bits (N*C0 exact
      for |N| < 2^17), C1, C2 floats (rounded to nearest).
  TF_F_L0..L2  ln2 = L0 + L1 + L2, L0 with 16 significant bits (n*L0 exact for
      |n| < 2^8), L1, L2 floats.
  TF_F_R3..R5  1/3! .. 1/5! rounded to float (the dotted Taylor tail).
  TF_FLOGT[i] for i = 1448 .. 2896: {c_i, -log c_i as (hi, lo) floats, c_i - 1}
      with c_i = RN_float(2048 / i): the reciprocal table of the float
      logarithm, log z = -log c_i + log1p(z c_i - 1), |z c_i - 1| < 2^-11.4.
  TF_FT[j], TF_FE[j]  2^(j/512) and 2^(j/512) - 1 as (hi, lo) floats, j = -256 .. 256.
  TF_FNLN2[n]  n ln2 as (hi, lo) floats (hi = RN_float(n ln2), lo = RN_float of the
      rest), n = -160 .. 140: the n ln2 term of the float logarithm.

Fixed-point constants of the integer exp core (unsigned integers, rounded to
nearest, each with its unit):
  TF_TFIX[j]   2^(j/65536), units 2^-127, as (lo64, hi64), j = -32768 .. 32768:
      the table of the reduction x = k ln2 + j ln2/65536 + r (a 2^16-step
      version of the paper's tabulated e^c, "Twofold exponent" > "Function
      pexp0()"); e^c - 1 of "Function pexpm10()" is TF_TFIX[j] - 2^127,
      exactly.  1 MiB; computed by exact integer iteration of 2^(1/65536) at
      256 bits and rounded to nearest.
  TF_HC_m      1/(m+1)!, the coefficients of H(r) = (e^r - 1)/r = sum r^m/(m+1)!:
      m = 0 .. 4 in units 2^-127 as (lo64, hi64), m = 5 .. 9 in units 2^-72
      (the degree-9 H of the logarithm's Newton step).
  TF_HC68_m    1/(m+1)!, m = 3 .. 6, units 2^-68 (the 64-bit levels of the
      degree-6 H of the exp core).
  TF_C12FIX    ln2/65536 - C0 (> 0), units 2^-148: the tail of the reduction constant.
  TF_CFIX136   ln2/65536, units 2^-136: the step that moves a negative reduced
      argument of e^x to N - 1 and r + ln2/65536.
  TF_LN2FIX    ln2, units 2^-128 (the n ln2 term of the logarithm).
  TF_LOGT[i] for i = 724 .. 1448 (z = i/1024 covers [sqrt(1/2), sqrt(2))):
      {-log(c_i) in units 2^-128 as a two's complement (lo64, hi64), C_i, the
      bits of c_i as a double} with c_i = C_i 2^-24, C_i = round(2^34 / i): the
      reciprocal table of the logarithm, log z = -log c_i + log1p(t) with
      t = z c_i - 1 exact and |t| < 2^-10.4.
  TF_PX_C[n], TF_PX_E[m]  the tables of the paper's own reduction (Function
      pexp0(): x = 2^L m + 2^-K n + y, y exact), with K = 8 and L = 1:
      TF_PX_C[n] = e^(n/256), n = -511 .. 511, units 2^-124 as (lo64, hi64);
      TF_PX_E[m] = e^(2m) = E_m 2^e_m, m = -373 .. 373, as {lo64, hi64, e_m, 0}
      with E_m in [2^127, 2^128) (rounded to nearest).
  TF_LOG2T[j] for j = -200 .. 200: {-log(c2_j) in units 2^-128 as a two's
      complement (lo64, hi64), C2_j, 0} with c2_j = C2_j 2^-24, C2_j =
      round(2^42 / (2^18 + j)): the second reciprocal table of the logarithm,
      t2 = (1 + t) c2_j - 1 with j = round(2^18 t), |t2| < 2^-18.9.
  TF_LOGU[i], TF_LOG2U[j]  the same two reductions rounded up for tlog's main
      path (n != 0): i = floor(1024 z), C_i = ceil(2^34 / i), so that t1 = z c_i
      - 1 lies in [0, 2^-9.49); j = floor(2^18 t1) in [0, 362], C2_j = ceil(2^42
      / (2^18 + j)), so that t2 = (1 + t1) c2_j - 1 lies in [0, 2^-17.97).  Rows
      {-log c in units 2^-128 as (lo64, hi64), C, 0}.
  TF_LG_m      (-1)^m / (m+1), m = 0 .. 4, units 2^-62 (two's complement): the
      coefficients of log1p(t)/t.
"""
import decimal
import math
import struct
import sys

D = decimal.Decimal
CTX = decimal.Context(prec=120, Emax=99999, Emin=-99999)


def f32_nearest(v):
    """The float nearest to the Decimal v (ties to even), as a Python float."""
    import numpy as np
    c = np.float32(float(v))
    best = None
    for x in (np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))):
        d = abs(CTX.subtract(D(float(x)), v))
        even = (int(np.array(x, dtype=np.float32).view(np.int32)) & 1) == 0
        key = (d, not even)
        if best is None or key < best[0]:
            best = (key, float(x))
    return best[1]


def fsplit_exact(v, n=2):
    out = []
    for _ in range(n):
        h = f32_nearest(v)
        out.append(h)
        v = CTX.subtract(v, D(h))
    return out


def hexf(x):
    return float.hex(x) + "f"


def trunc_bits(v, bits):
    """v truncated to `bits` significant bits (as a double, exact)."""
    import math
    mant, ex = math.frexp(float(v))
    scaled = CTX.multiply(v, CTX.power(2, bits - ex))
    return float(CTX.multiply(D(int(scaled.to_integral_value(rounding=decimal.ROUND_FLOOR))), CTX.power(2, ex - bits)))


def hexd(x):
    return float.hex(x)


def pow2_table(steps, half, unit):
    """round(2^(j/steps) 2^unit) for j = -half .. half: each power by exact
    integer multiplication of a 256-bit fixed-point 2^(+-1/steps) (taken from a
    120-digit decimal value), truncated per step; the accumulated error stays
    below 2^-230 relative, far inside the final rounding to 2^-unit."""
    P = 256
    scale = CTX.power(D(2), P)  # exact at 120 digits (2^256 has 78)
    up = int(CTX.multiply(CTX.power(D(2), CTX.divide(D(1), steps)), scale))
    dn = int(CTX.multiply(CTX.power(D(2), CTX.divide(D(-1), steps)), scale))
    pos, neg = [1 << P], [1 << P]
    for _ in range(half):
        pos.append(pos[-1] * up >> P)
        neg.append(neg[-1] * dn >> P)
    half_unit = 1 << (P - unit - 1)
    vals = neg[:0:-1] + pos
    return [(v + half_unit) >> (P - unit) for v in vals]


def main(out=sys.stdout):
    ln2 = CTX.ln(D(2))
    c = CTX.divide(ln2, 65536)
    C0 = trunc_bits(c, 26)
    inv_c = float(CTX.divide(65536, ln2))
    w = out.write
    w("/* Generated by gen_tables.py -- do not edit.  Constants of the twofold exp/log\n"
      "   kernels, from 120-digit decimal values. */\n")
    w("#pragma once\n\n")
    w("#ifndef TF_TABLE_QUALIFIER\n#define TF_TABLE_QUALIFIER static const\n#endif\n\n")
    w(f"#define TF_TAB_BITS 16\n")
    w(f"#define TF_TAB_HALF 32768     /* table index j = -32768 .. 32768, step ln2/65536 */\n")
    w(f"#define TF_INV_C {hexd(inv_c)}  /* 65536/ln2 */\n")
    w(f"#define TF_C0 {hexd(C0)}\n")
    w("\n")
    # float twofold constants
    cf = CTX.divide(ln2, 512)
    FC0 = trunc_bits(cf, 7)
    FC1, FC2 = fsplit_exact(CTX.subtract(cf, D(FC0)), 2)
    FL0 = trunc_bits(ln2, 16)
    FL1, FL2 = fsplit_exact(CTX.subtract(ln2, D(FL0)), 2)
    w("/* float twofold path */\n")
    w(f"#define TF_F_TAB_HALF 256\n#define TF_F_INV_C {hexf(f32_nearest(CTX.divide(512, ln2)))}\n")
    w(f"#define TF_F_C0 {hexf(FC0)}\n#define TF_F_C1 {hexf(FC1)}\n#define TF_F_C2 {hexf(FC2)}\n")
    w(f"#define TF_F_L0 {hexf(FL0)}\n#define TF_F_L1 {hexf(FL1)}\n#define TF_F_L2 {hexf(FL2)}\n")
    for m in range(3, 6):
        w(f"#define TF_F_R{m} {hexf(f32_nearest(CTX.divide(1, D(math.factorial(m)))))}\n")
    w("#define TF_FLOGT_LO 1448\n#define TF_FLOGT_HI 2896\n")
    w("/* {c_i, -log c_i hi, lo, c_i - 1} floats, c_i = RN_float(2048 / i), i = 1448 .. 2896 */\n")
    w("TF_TABLE_QUALIFIER float TF_FLOGT[1449][4] = {\n")
    for i in range(1448, 2897):
        cf = f32_nearest(CTX.divide(D(2048), D(i)))
        L = CTX.minus(CTX.ln(D(cf)))
        h, l = fsplit_exact(L, 2)
        cm1 = CTX.subtract(D(cf), 1)
        assert D(f32_nearest(cm1)) == cm1  # c - 1 exact in float (Sterbenz)
        z_lo, z_hi = D(i) / 2048 - D(1) / 4096, D(i) / 2048 + D(1) / 4096
        for zz in (max(z_lo, D("0.70710678")), min(z_hi, D("1.41421357"))):
            assert abs(CTX.subtract(CTX.multiply(zz, D(cf)), 1)) < D(2) ** D("-11.4"), (i, zz)
        w(f"  {{{hexf(cf)}, {hexf(h)}, {hexf(l)}, {hexf(f32_nearest(cm1))}}},\n")
    w("};\n")
    w("#define TF_FNLN2_LO (-160)\n")
    w("/* n ln2 as (hi, lo) floats, n = -160 .. 140; index n + 160 */\n")
    w("TF_TABLE_QUALIFIER float TF_FNLN2_TABLE[301][2] = {\n")
    for n in range(-160, 141):
        h, l = fsplit_exact(CTX.multiply(D(n), ln2), 2)
        w(f"  {{{hexf(h)}, {hexf(l)}}},\n")
    w("};\n")
    for name, minus1 in (("TF_FT", False), ("TF_FE", True)):
        w(f"/* {'2^(j/512) - 1' if minus1 else '2^(j/512)'} as (hi, lo) floats; index j + 256 */\n")
        w(f"TF_TABLE_QUALIFIER float {name}_TABLE[513][2] = {{\n")
        for j in range(-256, 257):
            v = CTX.power(D(2), CTX.divide(D(j), 512))
            if minus1:
                v = CTX.subtract(v, 1)
            h, l = fsplit_exact(v, 2)
            w(f"  {{{hexf(h)}, {hexf(l)}}},\n")
        w("};\n")
    w("\n")
    def fixed(v, unit_exp):
        """round(v * 2^unit_exp) as a Python int (v a Decimal)."""
        return int(CTX.multiply(v, CTX.power(2, unit_exp)).to_integral_value(rounding=decimal.ROUND_HALF_EVEN))

    def u128(x):
        assert 0 <= x < 2**128
        return f"0x{x & (2**64 - 1):016x}ull, 0x{x >> 64:016x}ull"

    w("/* coefficients 1/(m+1)! of H(r) = (e^r - 1)/r: m = 0 .. 4 in units 2^-127 as\n"
      "   {lo64, hi64}, m = 5 .. 9 in units 2^-72 */\n")
    for m in range(0, 10):
        v = CTX.divide(1, D(math.factorial(m + 1)))
        if m <= 4:
            w(f"#define TF_HC_{m} {{{u128(fixed(v, 127))}}}\n")
        else:
            x = fixed(v, 72)
            assert x < 2**64
            w(f"#define TF_HC_{m} 0x{x:016x}ull\n")
    w("/* coefficients 1/(m+1)! of the exp core's H, m = 3 .. 6, units 2^-68 */\n")
    for m in range(3, 7):
        x = fixed(CTX.divide(1, D(math.factorial(m + 1))), 68)
        assert x < 2**64
        w(f"#define TF_HC68_{m} 0x{x:016x}ull\n")
    c12 = CTX.subtract(c, D(C0))
    assert c12 > 0 and fixed(c12, 148) < 2**106
    w(f"#define TF_C12FIX {{{u128(fixed(c12, 148))}}}\n\n")
    w(f"#define TF_CFIX136 {{{u128(fixed(c, 136))}}}\n\n")
    w(f"#define TF_LN2FIX {{{u128(fixed(ln2, 128))}}}\n\n")
    w("/* coefficients (-1)^m/(m+1) of log1p(t)/t, units 2^-62, two's complement */\n")
    for m in range(0, 5):
        x = fixed(CTX.divide(D((-1) ** m), D(m + 1)), 62)
        w(f"#define TF_LG_{m} ((long long)0x{x & (2**64 - 1):016x}ull)\n")
    w("\n#define TF_LOGT_LO 724\n#define TF_LOGT_HI 1448\n")
    w("/* {-log(c_i) units 2^-128 as (lo64, hi64), C_i, bits of c_i} for i = 724 .. 1448,\n"
      "   c_i = C_i 2^-24 */\n")
    w("TF_TABLE_QUALIFIER unsigned long long TF_LOGT[725][4] = {\n")
    for i in range(724, 1449):
        C = int(CTX.divide(D(2**34), D(i)).to_integral_value(rounding=decimal.ROUND_HALF_EVEN))
        c = CTX.divide(D(C), D(2**24))
        L = fixed(CTX.minus(CTX.ln(c)), 128)
        assert abs(L) < 2**126.5 and C < 2**25
        z_lo, z_hi = D(i) / 1024 - D(1) / 2048, D(i) / 1024 + D(1) / 2048
        for zz in (max(z_lo, D("0.70710678118654752440")), min(z_hi, D("1.41421356237309504880"))):
            assert abs(CTX.subtract(CTX.multiply(zz, c), 1)) < D(2) ** D("-10.4"), (i, zz)
        cd = float(c)
        assert D(cd) == c
        Lu = L & (2**128 - 1)
        w(f"  {{0x{Lu & (2**64 - 1):016x}ull, 0x{Lu >> 64:016x}ull, {C}ull, 0x{struct.unpack('<Q', struct.pack('<d', cd))[0]:016x}ull}},\n")
    w("};\n\n")
    w("#define TF_LOG2T_HALF 200\n")
    w("/* {-log(c2_j) units 2^-128 as (lo64, hi64), C2_j, 0} for j = -200 .. 200,\n"
      "   c2_j = C2_j 2^-24, C2_j = round(2^42 / (2^18 + j)) */\n")
    w("TF_TABLE_QUALIFIER unsigned long long TF_LOG2T[401][4] = {\n")
    for j in range(-200, 201):
        C = int(CTX.divide(D(2**42), D(2**18 + j)).to_integral_value(rounding=decimal.ROUND_HALF_EVEN))
        c = CTX.divide(D(C), D(2**24))
        L = fixed(CTX.minus(CTX.ln(c)), 128)
        for t1 in (D(j) / 2**18 - D(1) / 2**19, D(j) / 2**18 + D(1) / 2**19):
            assert abs(CTX.subtract(CTX.multiply(1 + t1, c), 1)) < D(2) ** D("-18.9"), (j, t1)
        Lu = L & (2**128 - 1)
        w(f"  {{0x{Lu & (2**64 - 1):016x}ull, 0x{Lu >> 64:016x}ull, {C}ull, 0ull}},\n")
    w("};\n\n")
    # the sign-free pair of reciprocal tables of tlog's main path (n != 0):
    # rounded up, indexed by floor, so that both reduced arguments are >= 0
    w("\n#define TF_LOGU_LO 724\n#define TF_LOGU_HI 1448\n")
    w("/* {-log(c_i) units 2^-128 as (lo64, hi64), C_i, 0} for i = 724 .. 1448, c_i = C_i 2^-24,\n"
      "   C_i = ceil(2^34 / i): t1 = z c_i - 1 in [0, 2^-9.49) for i = floor(1024 z) */\n")
    w("TF_TABLE_QUALIFIER unsigned long long TF_LOGU[725][4] = {\n")
    zsplit = D(0x16a09e00000000) / D(2**52)  # the split's upper bound on z (log_split)
    jmax = 0
    for i in range(724, 1449):
        C = -(-(2**34) // i)
        c = CTX.divide(D(C), D(2**24))
        L = fixed(CTX.minus(CTX.ln(c)), 128)
        assert abs(L) < 2**126.5 and C < 2**25
        assert CTX.multiply(D(i) / 1024, c) >= 1
        t1max = CTX.subtract(CTX.multiply(min(D(i + 1) / 1024, zsplit), c), 1)
        assert t1max < D(2) ** D("-9.49"), i
        jmax = max(jmax, int(CTX.multiply(t1max, D(2**18)).to_integral_value(rounding=decimal.ROUND_FLOOR)))
        Lu = L & (2**128 - 1)
        w(f"  {{0x{Lu & (2**64 - 1):016x}ull, 0x{Lu >> 64:016x}ull, {C}ull, 0ull}},\n")
    w("};\n\n")
    assert jmax == 362
    w(f"#define TF_LOG2U_HI {jmax}\n")
    w("/* {-log(c2_j) units 2^-128 as (lo64, hi64), C2_j, 0} for j = 0 .. TF_LOG2U_HI,\n"
      "   c2_j = C2_j 2^-24, C2_j = ceil(2^42 / (2^18 + j)): t = (1 + t1) c2_j - 1 in [0, 2^-17.97)\n"
      "   for j = floor(2^18 t1) */\n")
    w(f"TF_TABLE_QUALIFIER unsigned long long TF_LOG2U[{jmax + 1}][4] = {{\n")
    for j in range(0, jmax + 1):
        C = -(-(2**42) // (2**18 + j))
        c = CTX.divide(D(C), D(2**24))
        L = fixed(CTX.minus(CTX.ln(c)), 128)
        assert CTX.multiply(1 + D(j) / 2**18, c) >= 1
        assert CTX.subtract(CTX.multiply(1 + D(j + 1) / 2**18, c), 1) < D(2) ** D("-17.97"), j
        Lu = L & (2**128 - 1)
        w(f"  {{0x{Lu & (2**64 - 1):016x}ull, 0x{Lu >> 64:016x}ull, {C}ull, 0ull}},\n")
    w("};\n\n")
    # the paper's reduction: K = 8, L = 1
    w("#define TF_PX_CHALF 511\n#define TF_PX_EHALF 373\n")
    w("/* e^(n/256) in units 2^-124 as {lo64, hi64}; index n + 511 */\n")
    w("TF_TABLE_QUALIFIER unsigned long long TF_PX_C[1023][2] = {\n")
    for n in range(-511, 512):
        v = CTX.exp(CTX.divide(D(n), 256))
        x = fixed(v, 124)
        assert 0 < x < 2**127
        w(f"  {{{u128(x)}}},\n")
    w("};\n")
    w("/* e^(2m) = E 2^e, E in [2^127, 2^128), as {lo64, hi64, e, 0}; index m + 373 */\n")
    w("TF_TABLE_QUALIFIER unsigned long long TF_PX_E[747][4] = {\n")
    for m in range(-373, 374):
        v = CTX.exp(D(2 * m))
        e = int(CTX.log10(v) / CTX.log10(D(2)))  # approximate exponent, corrected below
        while CTX.power(D(2), e) > v:
            e -= 1
        while CTX.power(D(2), e + 1) <= v:
            e += 1
        x = fixed(CTX.multiply(v, CTX.power(D(2), -e)), 127)
        ee = e - 127
        if x == 2**128:
            x, ee = 2**127, ee + 1
        assert 2**127 <= x < 2**128
        w(f"  {{{u128(x)}, 0x{ee & (2**64 - 1):016x}ull, 0ull}},\n")
    w("};\n\n")
    w("/* 2^(j/65536) in units of 2^-127 as {lo64, hi64}; index j + 32768 */\n")
    w("TF_TABLE_QUALIFIER unsigned long long TF_TFIX_TABLE[65537][2] = {\n")
    for v in pow2_table(65536, 32768, 127):
        w(f"  {{{u128(v)}}},\n")
    w("};\n\n")


if __name__ == "__main__":
    main()
