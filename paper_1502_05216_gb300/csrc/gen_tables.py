"""Generate tf_tables.h: the constants of the CUDA twofold exp/log kernels.

Run:  python gen_tables.py > tf_tables.h   (the build checks the file is current)

All values come from Python's decimal module at 120 significant digits and are
split into doubles hi + lo (+ lo2) with hi = RN(v), lo = RN(v - hi).

  TF_T[j]   = 2^(j/256)        as (hi, lo), j = -128 .. 128
  TF_E1[j]  = 2^(j/256) - 1    as (hi, lo), j = -128 .. 128
      The table of the argument reduction x = k ln2 + j ln2/256 + r (a
      2^8-step version of the paper's tabulated e^c and e^c - 1, section
      "Twofold exponent" > "Function pexp0()" and "Function pexpm10()").
  TF_C0, TF_C1, TF_C2  ln2/256 = C0 + C1 + C2, C0 with 35 significant bits so
      that N*C0 is exact for |N| < 2^18.
  TF_L0, TF_L1, TF_L2  ln2 = L0 + L1 + L2, L0 with 42 significant bits so that
      n*L0 is exact for |n| < 2^11 (the n ln2 term of the logarithm).
  TF_INV_C  256/ln2 rounded to double.
  TF_RF[m]  1/m! as (hi, lo), m = 0 .. 12 (Taylor coefficients of e^r).

Fixed-point constants of the integer exp core (unsigned integers, rounded to
nearest, each with its unit):
  TF_TFIX[j]   2^(j/256), units 2^-127, as (lo64, hi64), j = -128 .. 128
  TF_HC128_m   1/(m+2)!, units 2^-128, m = 0 .. 3 (Horner of (e^r - 1 - r)/r^2)
  TF_HC64_m    1/(m+2)!, units 2^-72, m = 4 .. 8
  TF_C12FIX    ln2/256 - C0, units 2^-148 (the tail of the reduction constant)
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
    C1, C2 = split(CTX.subtract(c, D(C0)), 2)
    L0 = trunc_bits(ln2, 42)
    L1, L2 = split(CTX.subtract(ln2, D(L0)), 2)
    inv_c = float(CTX.divide(256, ln2))
    w = out.write
    w("/* Generated by gen_tables.py -- do not edit.  Constants of the twofold exp/log\n"
      "   kernels, each split as hi + lo doubles from a 120-digit decimal value. */\n")
    w("#pragma once\n\n")
    w("#ifndef TF_TABLE_QUALIFIER\n#define TF_TABLE_QUALIFIER static const\n#endif\n\n")
    w(f"#define TF_TAB_K 8            /* table step ln2 / 2^TF_TAB_K */\n")
    w(f"#define TF_TAB_HALF 128       /* j = -128 .. 128 */\n")
    w(f"#define TF_INV_C {hexd(inv_c)}  /* 256/ln2 */\n")
    w(f"#define TF_C0 {hexd(C0)}\n#define TF_C1 {hexd(C1)}\n#define TF_C2 {hexd(C2)}\n")
    w(f"#define TF_L0 {hexd(L0)}\n#define TF_L1 {hexd(L1)}\n#define TF_L2 {hexd(L2)}\n\n")
    w("/* 1/m! as hi, lo for m = 0 .. 12 */\n")
    f = D(1)
    for m in range(13):
        if m:
            f = CTX.multiply(f, m)
        h, l = split(CTX.divide(1, f))
        w(f"#define TF_RF{m}_HI {hexd(h)}\n#define TF_RF{m}_LO {hexd(l)}\n")
    w("\n")
    def fixed(v, unit_exp):
        """round(v * 2^unit_exp) as a Python int (v a Decimal)."""
        return int(CTX.multiply(v, CTX.power(2, unit_exp)).to_integral_value(rounding=decimal.ROUND_HALF_EVEN))

    def u128(x):
        assert 0 <= x < 2**128
        return f"0x{x & (2**64 - 1):016x}ull, 0x{x >> 64:016x}ull"

    w("/* fixed-point constants of the integer exp core */\n")
    f = D(1)
    for m in range(0, 9):
        fact = D(math.factorial(m + 2))
        v = CTX.divide(1, fact)
        if m <= 3:
            w(f"#define TF_HC128_{m} {{{u128(fixed(v, 128))}}}\n")
        else:
            w(f"#define TF_HC64_{m} 0x{fixed(v, 72):016x}ull\n")
    c12 = CTX.subtract(c, D(C0))
    w(f"#define TF_C12FIX {{{u128(fixed(c12, 148))}}}\n\n")
    w("/* 2^(j/256) in units of 2^-127 as {lo64, hi64}; index j + 128 */\n")
    w("TF_TABLE_QUALIFIER unsigned long long TF_TFIX_TABLE[257][2] = {\n")
    for j in range(-128, 129):
        v = CTX.power(D(2), CTX.divide(D(j), 256))
        w(f"  {{{u128(fixed(v, 127))}}},\n")
    w("};\n\n")
    for name, minus1 in (("TF_T", False), ("TF_E1", True)):
        w(f"/* {'2^(j/256) - 1' if minus1 else '2^(j/256)'} as hi, lo; index j + 128 */\n")
        w(f"TF_TABLE_QUALIFIER double {name}_TABLE[257][2] = {{\n")
        for j in range(-128, 129):
            v = CTX.power(D(2), CTX.divide(D(j), 256))
            if minus1:
                v = CTX.subtract(v, 1)
            h, l = split(v)
            w(f"  {{{hexd(h)}, {hexd(l)}}},\n")
        w("};\n\n")


if __name__ == "__main__":
    main()
