"""Comparison of a twofold result (z0, z1) with the oracle's answer.

err = |z0 + z1 - F| is formed as ((z0 - Z0) + (z1 - Gh)) - Gl.  Whenever the
result is close to the oracle's, z0 - Z0 and z1 - Gh are exact (Sterbenz), so
err is computed to about 2^-53 of itself; when it is far, err is large anyway.

Tolerance (the reading of the accuracy target "z0 + z1 within 2^-100 of
f(x0 + x1)" for a twofold whose main part is fixed):
    err <= 2^-100 |F| + ulp(G)/2 + extra + 2^-1074
with G = F - Z0 the ideal deviation and ulp(G)/2 half the spacing of doubles
at |G|.  z0 = RN(f(x0)) is fixed by x0 alone, so z1, one double, is left to
hold G, which it cannot do more closely than half of its own spacing: for a
twofold whose x1 is far above the ulp scale of the result (exp of |x0| ~ 700
perturbs e^x0 by up to 2^-43.5 relative; log1p of y0 near -1 by up to 2^-23)
that alone exceeds 2^-100 |F|.  So what the method may add to z1's own
rounding is 2^-100 |F|.  For tadd/tmul, ``extra`` bounds the roundings of the
tail terms, which may cancel: tadd 2^-52 (|x1| + |y1|); tmul 2^-52 (|x0 y1| +
|x1 y0|) + |x1 y1| (the dropped second-order term).  Float twofolds use 2^-44,
half a float spacing of G, 2^-149.

The statistics returned include the error beyond half an ulp of G, relative
to |F| ("excess"): what the method adds to z1's own rounding, the quantity the
paper's accuracy thresholds (Analysis > Accuracy) are checked against.
"""
from __future__ import annotations

import numpy as np

# (relative term, unit roundoff of the format, absolute term)
TOL = {"f64": (2.0**-100, 2.0**-53, 2.0**-1074), "f32": (2.0**-44, 2.0**-24, 2.0**-149)}


def half_ulp(G, dtype="f64"):
    """Half the spacing of the format's numbers at |G| (the spacing above |G|,
    which is the larger one at a power of two)."""
    G = np.abs(np.asarray(G, dtype=np.float64))
    with np.errstate(invalid="ignore", over="ignore"):
        if dtype == "f32":
            return np.spacing(G.astype(np.float32)).astype(np.float64) * 0.5
        return np.spacing(G) * 0.5


def allowance(func, args, dtype="f64"):
    """The tail-rounding term ``extra`` of the tolerance for tadd/tmul (else 0)."""
    if func not in ("tadd", "tmul") or args is None:
        return 0.0
    u = 2.0**-52 if dtype == "f64" else 2.0**-23
    x0, x1, y0, y1 = (np.asarray(a, dtype=np.float64) if a is not None else 0.0 for a in args)
    with np.errstate(invalid="ignore", over="ignore"):
        if func == "tadd":
            return u * (np.abs(x1) + np.abs(y1))
        return u * (np.abs(x0 * y1) + np.abs(x1 * y0)) + np.abs(x1 * y1)


def errors(z0, z1, orc):
    """(abs_err, rel_err, mainpart_equal) per element; NaN/Inf handled."""
    z0 = np.asarray(z0, dtype=np.float64)
    z1 = np.asarray(z1, dtype=np.float64)
    with np.errstate(invalid="ignore", over="ignore"):
        d = ((z0 - orc.Z0) + (z1 - orc.Gh)) - orc.Gl
        err = np.abs(d)
        rel = err / np.where(orc.A > 0, orc.A, np.inf)
    same = (z0 == orc.Z0) | (np.isnan(z0) & np.isnan(orc.Z0))
    return err, rel, same


def ulp_distance(a, b):
    """|a - b| in units of doubles between them (0 for equal, NaN pairs 0)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)

    def key(x):
        i = x.view(np.int64)
        return np.where(i < 0, np.int64(-0x8000000000000000) - i, i)

    with np.errstate(over="ignore"):
        d = np.abs(key(a).astype(np.float64) - key(b).astype(np.float64))
    both_nan = np.isnan(a) & np.isnan(b)
    d[both_nan] = 0
    d[np.isnan(a) ^ np.isnan(b)] = np.inf
    return d


def ulp_distance_f32(a, b):
    """|a - b| in units of floats between them (a, b float values)."""
    a = np.asarray(a, dtype=np.float64).astype(np.float32)
    b = np.asarray(b, dtype=np.float64).astype(np.float32)

    def key(x):
        i = x.view(np.int32).astype(np.int64)
        return np.where(i < 0, np.int64(-0x80000000) - i, i)

    d = np.abs(key(a) - key(b)).astype(np.float64)
    both_nan = np.isnan(a) & np.isnan(b)
    d[both_nan] = 0
    d[np.isnan(a) ^ np.isnan(b)] = np.inf
    return d


def check(z0, z1, orc, dtype="f64", mainpart_rate=0.99999, where="", func=None, args=None):
    """Assert the parity bar: z0 == oracle Z0 in >= mainpart_rate of elements and
    within one ulp always; z0 + z1 within the tolerance above always, except for
    elements whose z1 is fixed exactly by the special-value rules (then z1 must
    equal it bitwise, NaN matching NaN).  Returns the statistics: main-part
    mismatches, max / mean of err/|F| (log2), and of the excess over half an
    ulp of G (log2), with the counts of elements whose total error exceeds the
    relative term and whose excess does."""
    rel_tol, ulp_tol, abs_tol = TOL[dtype]
    z0 = np.asarray(z0, dtype=np.float64)
    z1 = np.asarray(z1, dtype=np.float64)
    n = z0.shape[0]
    err, rel, same = errors(z0, z1, orc)
    # z1 fixed by the special-value rules, or an infinite / NaN ideal deviation
    exact = ((orc.flags & 2) != 0) | ~np.isfinite(orc.Gh)
    mism = int(np.count_nonzero(~same))
    ulps = ulp_distance_f32(z0, orc.Z0) if dtype == "f32" else ulp_distance(z0, orc.Z0)
    bad0 = np.nonzero(ulps > 1)[0]
    assert bad0.size == 0, (f"{where}: main part off by >1 ulp at {bad0[:10]}: "
                            f"{_show(bad0, z0, z1, orc, args)}")
    assert mism <= (1.0 - mainpart_rate) * n, f"{where}: {mism} main-part mismatches of {n}"
    # special values: z1 must be the fixed value (NaN matches NaN)
    ex_ok = (z1 == orc.Gh) | (np.isnan(z1) & np.isnan(orc.Gh))
    bad_ex = np.nonzero(exact & ~ex_ok & same)[0]
    assert bad_ex.size == 0, (f"{where}: special-value z1 wrong at {bad_ex[:10]}: "
                              f"{_show(bad_ex, z0, z1, orc, args)}")
    gen = ~exact
    hu = half_ulp(orc.Gh, dtype)
    with np.errstate(invalid="ignore", over="ignore"):
        tol = rel_tol * orc.A + hu + abs_tol + allowance(func, args, dtype)
        ok = err <= tol
    bad = np.nonzero(gen & ~ok)[0]
    if bad.size:
        worst = bad[np.argsort(-(err[bad] / tol[bad]))][:6]
        raise AssertionError(f"{where}: {bad.size} elements beyond tolerance; worst err/tol "
                             f"{err[worst[0]] / tol[worst[0]]:.3g}: {_show(worst, z0, z1, orc, args)}")
    # statistics over results whose z1 is a normal number (|F| 2^-p above the
    # smallest normal), as the paper's accuracy figures exclude subnormal results
    normal_min = 2.0**-969 if dtype == "f64" else 2.0**-102
    fin = gen & (orc.A >= normal_min) & np.isfinite(rel)
    r = rel[fin]
    with np.errstate(invalid="ignore", divide="ignore"):
        # error beyond the representation limit of z1 (what the method itself adds)
        excess = np.maximum(err - hu, 0.0)[fin] / orc.A[fin]

    def lg(v):
        return float(np.log2(v)) if v > 0 else -np.inf

    return {"n": n, "mainpart_mismatch": mism,
            "max_rel_log2": lg(r.max()) if r.size else -np.inf,
            "mean_rel_log2": lg(r.mean()) if r.size else -np.inf,
            "beyond_rel_tol": int(np.count_nonzero(r > rel_tol)),
            "max_excess_rel_log2": lg(excess.max()) if excess.size else -np.inf,
            "mean_excess_rel_log2": lg(excess.mean()) if excess.size else -np.inf,
            "excess_beyond_rel_tol": int(np.count_nonzero(excess > rel_tol)),
            "excess": excess}


def _show(idx, z0, z1, orc, args):
    rows = []
    for i in idx[:6]:
        a = "" if args is None else ", ".join(
            f"{float(np.asarray(x)[i])!r}" for x in args if x is not None)
        rows.append(f"[{i}] args=({a}) z=({z0[i]!r}, {z1[i]!r}) oracle=({orc.Z0[i]!r}, {orc.Gh[i]!r}"
                    f" + {orc.Gl[i]!r}, |F|={orc.A[i]!r})")
    return "; ".join(rows)
