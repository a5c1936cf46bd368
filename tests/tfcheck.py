"""Comparison of a twofold result (z0, z1) with the oracle's answer.

err = |z0 + z1 - F| is formed as ((z0 - Z0) + (z1 - Gh)) - Gl.  Whenever the
result is close to the oracle's, z0 - Z0 and z1 - Gh are exact (Sterbenz), so
err is computed to about 2^-53 of itself; when it is far, err is large anyway.
"""
from __future__ import annotations

import numpy as np

# Tolerances: relative 2^-100 for double twofolds, 2^-44 for float twofolds, plus
# the smallest subnormal (the value of the result is then below the format's
# reach, the paper's "if result is not subnormal" caveat in "Method summary").
TOL = {"f64": (2.0**-100, 2.0**-1074), "f32": (2.0**-44, 2.0**-149)}


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


def check(z0, z1, orc, dtype="f64", mainpart_rate=0.99999, where=""):
    """Assert the parity bar: z0 == oracle Z0 in >= mainpart_rate of elements and
    within one ulp always; z0 + z1 within the relative tolerance always, except
    for elements whose z1 is fixed exactly by the special-value rules (then z1
    must equal it bitwise, NaN matching NaN)."""
    rel_tol, abs_tol = TOL[dtype]
    z0 = np.asarray(z0, dtype=np.float64)
    z1 = np.asarray(z1, dtype=np.float64)
    n = z0.shape[0]
    err, rel, same = errors(z0, z1, orc)
    exact = (orc.flags & 2) != 0
    mism = int(np.count_nonzero(~same))
    ulps = ulp_distance(z0, orc.Z0)
    assert np.all(ulps <= 1), f"{where}: main part off by >1 ulp at {np.nonzero(ulps > 1)[0][:10]}"
    assert mism <= (1.0 - mainpart_rate) * n, f"{where}: {mism} main-part mismatches of {n}"
    # special values: z1 must be the fixed value (NaN matches NaN)
    ex_ok = (z1 == orc.Gh) | (np.isnan(z1) & np.isnan(orc.Gh))
    bad_ex = exact & ~ex_ok & same
    assert not np.any(bad_ex), (f"{where}: special-value z1 wrong at {np.nonzero(bad_ex)[0][:10]}: "
                                f"got {z1[bad_ex][:5]}, want {orc.Gh[bad_ex][:5]}")
    gen = ~exact
    ok = err <= rel_tol * orc.A + abs_tol
    bad = gen & ~ok
    assert not np.any(bad), (f"{where}: {np.count_nonzero(bad)} elements beyond tolerance; worst rel "
                             f"2^{np.log2(np.nanmax(rel[bad])):.1f} at {np.nonzero(bad)[0][:10]}")
    r = rel[gen & (orc.A > 0) & np.isfinite(rel)]
    return {"n": n, "mainpart_mismatch": mism,
            "max_rel_log2": float(np.log2(r.max())) if r.size and r.max() > 0 else -np.inf,
            "mean_rel_log2": float(np.log2(r.mean())) if r.size and r.mean() > 0 else -np.inf}
