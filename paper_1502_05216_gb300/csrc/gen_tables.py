"""Generate tf_tables.h: the constants of the CUDA twofold exp/log kernels.

Run:  python gen_tables.py > tf_tables.h   (the build checks the file is current)

All values come from Python's decimal module at 120 significant digits; a
value split into doubles is hi = RN(v), lo = RN(v - hi).

  TF_C0     ln2/256 rounded down to 35 significant bits, so that N*C0 is exact
      for |N| < 2^19 (argument reduction x = N ln2/256 + r).
  TF_L0, TF_L1, TF_L2  ln2 = L0 + L1 + L2, L0 with 42 significant bits so that
      n*L0 is exact for |n| < 2^11 (the n ln2 term of the logarithm).
  TF_INV_C  256/ln2 rounded to double.

Fixed-point constants of the integer exp core (unsigned integers, rounded to
nearest, each with its unit):
  TF_TFIX[j]   2^(j/256), units 2^-127, as (lo64, hi64), j = -128 .. 128: the
      table of the reduction x = k ln2 + j ln2/256 + r (a 2^8-step version of
      the paper's tabulated e^c, "Twofold exponent" > "Function pexp0()");
      e^c - 1 of "Function pexpm10()" is TF_TFIX[j] - 2^127, exactly.
  TF_HC_m      1/(m+1)!, the coefficients of H(r) = (e^r - 1)/r = sum r^m/(m+1)!:
      m = 0 .. 4 in units 2^-127 as (lo64, hi64), m = 5 .. 9 in units 2^-72.
  TF_C12FIX    ln2/256 - C0 (> 0), units 2^-148: the tail of the reduction constant.
"""
import decimal
import math
import sys

D = decimal.Decimal
CTX = decimal.Context(prec=120, Emax=99999, Emin=-99999)


def split(v, n=2):
    out = []
    for _ in range(n):
        h = float(v)  # correctly rounded
        out.append(h)
        v = CTX.subtract(v, D(h))
    return out


def trunc_bits(v, bits):
    """v truncated to `bits` significant bits (as a double, exact)."""
    import math
    mant, ex = math.frexp(float(v))
    scaled = CTX.multiply(v, CTX.power(2, bits - ex))
    return float(CTX.multiply(D(int(scaled.to_integral_value(rounding=decimal.ROUND_FLOOR))), CTX.power(2, ex - bits)))


def hexd(x):
    return float.hex(x)


def main(out=sys.stdout):
    ln2 = CTX.ln(D(2))
    c = CTX.divide(ln2, 256)
    C0 = trunc_bits(c, 35)
    L0 = trunc_bits(ln2, 42)
    L1, L2 = split(CTX.subtract(ln2, D(L0)), 2)
    inv_c = float(CTX.divide(256, ln2))
    w = out.write
    w("/* Generated by gen_tables.py -- do not edit.  Constants of the twofold exp/log\n"
      "   kernels, from 120-digit decimal values. */\n")
    w("#pragma once\n\n")
    w("#ifndef TF_TABLE_QUALIFIER\n#define TF_TABLE_QUALIFIER static const\n#endif\n\n")
    w(f"#define TF_TAB_HALF 128       /* table index j = -128 .. 128, step ln2/256 */\n")
    w(f"#define TF_INV_C {hexd(inv_c)}  /* 256/ln2 */\n")
    w(f"#define TF_C0 {hexd(C0)}\n")
    w(f"#define TF_L0 {hexd(L0)}\n#define TF_L1 {hexd(L1)}\n#define TF_L2 {hexd(L2)}\n\n")
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
    c12 = CTX.subtract(c, D(C0))
    assert c12 > 0
    w(f"#define TF_C12FIX {{{u128(fixed(c12, 148))}}}\n\n")
    w("/* 2^(j/256) in units of 2^-127 as {lo64, hi64}; index j + 128 */\n")
    w("TF_TABLE_QUALIFIER unsigned long long TF_TFIX_TABLE[257][2] = {\n")
    for j in range(-128, 129):
        v = CTX.power(D(2), CTX.divide(D(j), 256))
        w(f"  {{{u128(fixed(v, 127))}}},\n")
    w("};\n\n")


if __name__ == "__main__":
    main()
