"""CPU oracle for the twofold exp/log library -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA kernels and
their C ABI) never calls it, and the two share no code: this side is plain C in
IEEE binary128 (``tf_oracle.c``) plus an arbitrary-precision ``decimal``
tie-breaker, written from the definition of a twofold function (paper,
"Twofold exponent" > "Method summary"; "Twofold logarithm" > "Newton
inversion"): z0 is f(x0) correctly rounded, z0 + z1 approximates f(x0 + x1).

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle.py`` (decimal evaluations at 60+ digits, closed forms,
series, invariants, arguments whose f lies next to a rounding midpoint, and
planted-mistake checks).
"""
from __future__ import annotations

import ctypes
import decimal
from fractions import Fraction
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")

KINDS = {"texp": 0, "texpm1": 1, "tlog": 2, "tlog1p": 3, "tadd": 4, "tmul": 5}
FL_AMBIG, FL_EXACT = 1, 2

_lib = None
_lock = threading.Lock()


def _compile(out: str, defines=()) -> None:
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
            "-frounding-math", *[f"-D{d}" for d in defines], _SRC, "-o", out, "-lm"]
    # OpenMP when the host compiler has it; the oracle is correct either way.
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)


def build(force: bool = False, defines=(), name: str = "libtforacle.so") -> str:
    """Compile tf_oracle.c into oracle/_build/<name>; returns the path."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, name)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        _compile(out, defines)
    return out


def _bind(path: str):
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.tfo_eval.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp, dp, dp, dp, dp, dp, dp,
                             ctypes.POINTER(ctypes.c_uint)]
    lib.tfo_eval.restype = ctypes.c_int
    lib.tfo_eval2.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, dp, dp, dp, dp, dp, dp, dp, dp,
                              ctypes.POINTER(ctypes.c_uint)]
    lib.tfo_eval2.restype = ctypes.c_int
    lib.tfo_libq.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp]
    lib.tfo_libq.restype = ctypes.c_int
    vp = ctypes.c_void_p
    lib.tfo_chain.argtypes = [ctypes.c_int64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.tfo_chain.restype = ctypes.c_int
    lib.tfo_threads.restype = ctypes.c_int
    lib.tfo_set_threads.argtypes = [ctypes.c_int]
    return lib


def load(path: str | None = None):
    """The oracle library (built on first use)."""
    global _lib
    if path is not None:
        return _bind(path)
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


def threads() -> int:
    return load().tfo_threads()


def set_threads(t: int) -> None:
    load().tfo_set_threads(int(t))


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _as_f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class Result:
    """Per-element oracle answer.

    Z0     f(x0) rounded to nearest double (the required main part),
    Gh+Gl  the ideal z1: F - Z0 with F = f(x0 + x1), to about 106 bits,
    A      |F| rounded to double (scale of the relative error),
    flags  FL_EXACT: the special-value rules fix z1 = Gh exactly.
    """

    def __init__(self, Z0, Gh, Gl, A, flags):
        self.Z0, self.Gh, self.Gl, self.A, self.flags = Z0, Gh, Gl, A, flags


def evaluate(func: str, x0, x1=None, y0=None, y1=None, lib=None, dtype: str = "f64") -> Result:
    """Oracle answer for every element of the twofold function ``func``.
    dtype "f32": float twofolds (unary functions; the float arguments are
    exact in double), Z0 = f(x0) rounded to float."""
    lib = lib or load()
    kind = KINDS[func]
    f32 = dtype == "f32"
    x0, x1, y0, y1 = map(_as_f64, (x0, x1, y0, y1))
    n = x0.shape[0]
    Z0, Gh, Gl, A = (np.empty(n) for _ in range(4))
    fl = np.empty(n, dtype=np.uint32)
    rc = lib.tfo_eval2(kind, int(f32), n, _p(x0), _p(x1), _p(y0), _p(y1), _p(Z0), _p(Gh), _p(Gl), _p(A),
                       fl.ctypes.data_as(ctypes.POINTER(ctypes.c_uint)))
    if rc != 0:
        raise ValueError(f"tfo_eval rejected its arguments ({rc})")
    if func in ("texp", "texpm1", "tlog", "tlog1p"):
        redecide(func, x0, Z0, Gh, fl, f32)
    fl &= ~np.uint32(FL_AMBIG)
    return Result(Z0, Gh, Gl, A, fl)


# Planted mistakes of this Python layer (0 = none), set only by the tests that
# show the pins catch them: 11 shifts the deviation the wrong way when the main
# part is re-decided, 12 re-decides by rounding toward zero.
_PLANT = 0


def redecide(func: str, x0, Z0, Gh, fl, f32: bool = False) -> int:
    """Re-decide, in place, the main part of every element flagged FL_AMBIG
    (f(x0) within 2^-50 of a spacing from a rounding midpoint, where the
    binary128 value cannot be trusted to round correctly): Z0 becomes f(x0)
    evaluated with 80 significant digits in decimal and rounded to nearest
    (double, or float when f32), and the ideal deviation G = F - Z0 moves by
    the opposite amount, so that Z0 + G = F is unchanged.  The old and the new
    Z0 are adjacent (or equal), so Gh - (z - Z0) is exact.  Returns the number
    of main parts that changed."""
    rnd = round_to_float if f32 else round_to_double
    changed = 0
    for i in np.nonzero(fl & FL_AMBIG)[0]:
        v = dec_f(func, float(x0[i]), 80)
        z = _toward_zero(v, f32) if _PLANT == 12 else rnd(v)
        if z != Z0[i]:
            if _PLANT == 11:
                Gh[i] += z - Z0[i]
            else:
                Gh[i] -= z - Z0[i]
            Z0[i] = z
            changed += 1
    return changed


def _toward_zero(v: decimal.Decimal, f32: bool) -> float:
    """The planted wrong rounding (toward zero) of _PLANT == 12."""
    z = round_to_float(v) if f32 else round_to_double(v)
    if np.isfinite(z) and abs(decimal.Decimal(z)) > abs(v):
        z = float(np.nextafter(np.float32(z), np.float32(0))) if f32 else float(np.nextafter(z, 0.0))
    return z


def coupled(res: Result) -> Result:
    """The coupled form of a twofold answer (paper, "Algorithm summary" of the
    exponent and of the logarithm: pexp, pexpm1, plog, plog1p return the
    "coupled" value of f): with F = Z0 + Gh + Gl, the main part becomes RN(F)
    and Gh + Gl the remainder F - RN(F).  Exact rational arithmetic, element by
    element.  Answers fixed by the special-value rules (FL_EXACT), non-finite
    parts and G = 0 (already coupled) are returned unchanged."""
    Z0, Gh, Gl = res.Z0.copy(), res.Gh.copy(), res.Gl.copy()
    for i in range(Z0.size):
        if (res.flags[i] & FL_EXACT) or not (np.isfinite(Z0[i]) and np.isfinite(Gh[i]) and np.isfinite(Gl[i])):
            continue
        if Gh[i] == 0.0 and Gl[i] == 0.0:
            continue
        F = Fraction(float(Z0[i])) + Fraction(float(Gh[i])) + Fraction(float(Gl[i]))
        z = float(F)                     # correctly rounded (integer true division)
        r = F - Fraction(z)
        h = float(r)
        Z0[i], Gh[i], Gl[i] = z, h, float(r - Fraction(h))
    return Result(Z0, Gh, Gl, res.A.copy(), res.flags.copy())


def chain(batch: dict, lib=None):
    """Exact result (binary128) of every chain of a step-major batch (the dict
    of paper_1502_05216_gb300.inputs.chains) and its condition sum K: returns
    (Fh, Fl, K), F = Fh + Fl to about 106 bits; a computation that makes a
    relative error of at most eps per operation is within eps K |F| of F."""
    lib = lib or load()
    n = batch["s0"].shape[0]
    ops = np.ascontiguousarray(batch["ops"], dtype=np.uint8)
    arr = {k: np.ascontiguousarray(batch[k], dtype=np.float64) for k in ("a0", "a1", "s0", "s1")}
    sb = np.ascontiguousarray(batch["step_base"], dtype=np.int64)
    ln = np.ascontiguousarray(batch["length"], dtype=np.int32)
    Fh, Fl, K = np.empty(n), np.empty(n), np.empty(n)
    p = lambda a: a.ctypes.data  # noqa: E731
    rc = lib.tfo_chain(n, p(ops), p(arr["a0"]), p(arr["a1"]), p(sb), p(ln), p(arr["s0"]), p(arr["s1"]),
                       p(Fh), p(Fl), p(K))
    if rc != 0:
        raise ValueError("tfo_chain rejected its arguments")
    return Fh, Fl, K


def libq(func: str, x) -> np.ndarray:
    """glibc binary128 f(x) as (n, 2) hi/lo doubles -- for pinning tests only."""
    x = _as_f64(x)
    out = np.empty((x.shape[0], 2))
    load().tfo_libq(KINDS[func], x.shape[0], _p(x), _p(out))
    return out


# ---------------------------------------------------------------------------------
# Arbitrary-precision decimal evaluation (tie-breaker and independent pin).
# ---------------------------------------------------------------------------------

def dec_f(func: str, x: float, digits: int = 60) -> decimal.Decimal:
    """f(x) for a double x, to about ``digits`` significant digits, in decimal."""
    ctx = decimal.Context(prec=digits + 40, Emax=999999, Emin=-999999)
    d = decimal.Decimal(x)  # exact value of the double
    if func == "texp":
        return ctx.exp(d)
    if func == "texpm1":
        if abs(x) < 1e-3:  # series with exact terms, avoids 1 - 1 cancellation
            term, s, k = d, d, 1
            while True:
                k += 1
                term = ctx.divide(ctx.multiply(term, d), k)
                if term == 0 or abs(term) < abs(s) * decimal.Decimal(10) ** -(digits + 20):
                    return s
                s = ctx.add(s, term)
        return ctx.subtract(ctx.exp(d), 1)
    if func == "tlog":
        return ctx.ln(d)
    if func == "tlog1p":
        return ctx.ln(ctx.add(d, 1))  # 1 + x is exact at this precision
    raise KeyError(func)


def round_to_float(v: decimal.Decimal) -> float:
    """Nearest float (binary32, ties to even, subnormals, overflow at
    2^128 - 2^103) of a decimal value, returned as a Python float."""
    if v.is_nan():
        return float("nan")
    if v.is_infinite():
        return float(v)
    big = decimal.Decimal(2) ** 128 - decimal.Decimal(2) ** 103
    if abs(v) >= big:
        return float("inf") if v > 0 else float("-inf")
    c = np.float32(float(v))
    best = None
    for x in (np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))):
        if not np.isfinite(x):
            continue
        d = abs(decimal.Decimal(float(x)) - v)
        odd = int(np.array(x, dtype=np.float32).view(np.int32)) & 1
        key = (d, odd)
        if best is None or key < best[0]:
            best = (key, float(x))
    return best[1]


def round_to_double(v: decimal.Decimal) -> float:
    """Nearest double (ties to even) of a decimal value; Python's float() of a
    decimal string is correctly rounded, including subnormals and overflow."""
    try:
        return float(v)
    except OverflowError:
        return float("inf") if v > 0 else float("-inf")
