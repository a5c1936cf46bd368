"""Seeded synthetic inputs for the twofold exp/log workloads.

This module holds no arithmetic of the twofold method: it only draws argument
arrays.  Both the CUDA path's tests and benchmark and the CPU oracle's tests
take their inputs from here, so the two sides always see identical bits.

Every element is a pure function of (seed, stream, index): a counter-based
generator, SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), applied to the counter
    c = seed * 2**40 + stream * 2**36 + i
as the (c+1)-th output of a SplitMix64 sequence started at state 0, i.e.
    z = (c + 1) * 0x9E3779B97F4A7C15  (mod 2**64)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    z =  z ^ (z >> 31).
A uniform U in [0, 1) is (z >> 11) * 2**-53.  Any single element can therefore
be regenerated on its own, which is how sampled oracle checks at full size work.

A twofold argument is the pair x0 + x1 with x1 = RN(x0 * u * 2**-p), u uniform
in [-1, 1] and p = 53 (double) or 24 (float): a perturbation of at most one ulp
scale, as produced by a preceding twofold operation (paper, "Overview").
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream ids (each draw of an element uses its own stream)
S_MAG, S_SIGN, S_PERT, S_PICK, S_AUX = 0, 1, 2, 3, 4


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """SplitMix64 output for each uint64 counter (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (counter.astype(np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """U in [0, 1) with 53 random bits, elements start .. start+n-1."""
    if not (0 <= seed < 2**24 and 0 <= stream < 16 and 0 <= start and start + n <= 2**36):
        raise ValueError("seed/stream/index out of the generator's counter layout")
    base = (seed << 40) | (stream << 36)
    c = np.arange(start, start + n, dtype=np.uint64) + np.uint64(base)
    return (splitmix64(c) >> np.uint64(11)).astype(np.float64) * 2.0**-53


def _perturb(x0: np.ndarray, seed: int, n: int, start: int, p: int) -> np.ndarray:
    u = 2.0 * uniform(seed, S_PERT, n, start) - 1.0
    with np.errstate(invalid="ignore", over="ignore"):
        return x0 * u * 2.0**-p  # each product is exact up to the final rounding


def _signs(seed: int, n: int, start: int) -> np.ndarray:
    return np.where(uniform(seed, S_SIGN, n, start) < 0.5, -1.0, 1.0)


def _loguniform(lo_exp: float, hi_exp: float, seed: int, n: int, start: int) -> np.ndarray:
    return np.exp2(lo_exp + (hi_exp - lo_exp) * uniform(seed, S_MAG, n, start))


# ---------------------------------------------------------------------------------
# Workloads.  Each returns (x0, x1) as float64 (or float32 for dtype="f32").
# ---------------------------------------------------------------------------------

def texp_uniform(n: int, seed: int = 0, start: int = 0):
    """texp over double, x0 uniform in [-708, 709] (1417 wide), x1 = x0*u*2^-53."""
    x0 = -708.0 + 1417.0 * uniform(seed, S_MAG, n, start)
    return x0, _perturb(x0, seed, n, start, 53)


def exp_args(n: int, seed: int, start: int = 0):
    """texp/texpm1: random sign, |x0| log-uniform in [2^-40, 708]."""
    x0 = _signs(seed, n, start) * _loguniform(-40.0, math.log2(708.0), seed, n, start)
    return x0, _perturb(x0, seed, n, start, 53)


def log_args(n: int, seed: int, start: int = 0):
    """tlog: x0 log-uniform in [2^-1020, 2^1020]."""
    x0 = _loguniform(-1020.0, 1020.0, seed, n, start)
    return x0, _perturb(x0, seed, n, start, 53)


def log1p_args(n: int, seed: int, start: int = 0):
    """tlog1p: half of the elements random sign with |x0| log-uniform in
    [2^-40, 2^-10); the other half x0 = RN(t - 1) with t log-uniform in
    [2^-30, 2^100], which spans -1 + 2^-30 .. 2^100."""
    pick = uniform(seed, S_PICK, n, start) < 0.5
    small = _signs(seed, n, start) * _loguniform(-40.0, -10.0, seed, n, start)
    t = _loguniform(-30.0, 100.0, seed, n, start)
    x0 = np.where(pick, small, t - 1.0)
    return x0, _perturb(x0, seed, n, start, 53)


def arith_args(n: int, seed: int, start: int = 0):
    """tadd/tmul operands: random sign, |x0| log-uniform in [2^-20, 2^20]."""
    x0 = _signs(seed, n, start) * _loguniform(-20.0, 20.0, seed, n, start)
    return x0, _perturb(x0, seed, n, start, 53)


# The double-precision workload of each function: generator and its seed.
WORKLOADS = {
    "texp": (exp_args, 2),
    "texpm1": (exp_args, 3),
    "tlog": (log_args, 4),
    "tlog1p": (log1p_args, 5),
    "tadd": (arith_args, 6),   # second operand: seed 7
    "tmul": (arith_args, 8),   # second operand: seed 9
}


def _workload1(func: str, n: int, start: int):
    gen, seed = WORKLOADS[func]
    x = gen(n, seed, start)
    if func in ("tadd", "tmul"):
        return x + gen(n, seed + 1, start)
    return x


def workload(func: str, n: int, start: int = 0, chunk: int = 1 << 21):
    """(x0, x1[, y0, y1]) of the named function's n-element workload.  Large
    workloads are drawn in chunks on a thread pool (each element depends on its
    index only, so the chunking does not change any value)."""
    if n <= chunk:
        return _workload1(func, n, start)
    from concurrent.futures import ThreadPoolExecutor
    import os
    pieces = [(s, min(chunk, n - s)) for s in range(0, n, chunk)]
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        parts = list(ex.map(lambda p: _workload1(func, p[1], start + p[0]), pieces))
    return tuple(np.concatenate([p[k] for p in parts]) for k in range(len(parts[0])))


# ---------------------------------------------------------------------------------
# Hard cases: arguments near the thresholds where the result overflows, turns
# subnormal or underflows to zero, near 1 for the logarithm and near -1 for
# log1p, x1 = 0 and |x1| = half an ulp of x0, and the IEEE special values.
# The threshold values are properties of the functions (where e^x crosses the
# double range), not of any method of computing them.
# ---------------------------------------------------------------------------------

EXP_OVERFLOW = 709.782712893384      # e^x >= 2^1024 - 2^970 above this
EXP_UNDERFLOW = -745.1332191019412   # e^x rounds to 0 at or below this
EXP_SUBNORMAL = -708.3964185322641   # e^x < 2^-1022 below this

SPECIALS = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, 5e-324, -5e-324,
                     2.2250738585072014e-308, 1.7976931348623157e308, -1.7976931348623157e308])


def _half_ulp(x0: np.ndarray) -> np.ndarray:
    """Half the spacing of doubles above |x0| (exactly representable)."""
    with np.errstate(invalid="ignore", over="ignore"):
        return (np.nextafter(np.abs(x0), np.inf) - np.abs(x0)) * 0.5


def _mix(parts, seed, n, start, x1_scale):
    """Concatenate the generated pieces, cut to n, and draw x1: 10% zero, 5%
    exactly +-half an ulp, else x0*u*2^-x1_scale; the last elements pair the
    special values with each other."""
    x0 = np.concatenate(parts)[:n]
    x1 = _perturb(x0, seed, n, start, x1_scale)
    pick = uniform(seed, S_AUX, n, start)
    sgn = np.where(uniform(seed, S_SIGN, n, start) < 0.5, -1.0, 1.0)
    x1 = np.where(pick < 0.10, 0.0, x1)
    x1 = np.where((pick >= 0.10) & (pick < 0.15), sgn * _half_ulp(x0), x1)
    m = SPECIALS.shape[0]
    k = min(n, m * m)
    if k:
        a = np.repeat(SPECIALS, m)[:k]
        b = np.tile(SPECIALS, m)[:k] * 2.0**-60
        x0[n - k:] = a
        x1[n - k:] = b
    return x0, x1


def hard_cases(func: str, n: int, seed: int = 9, start: int = 0):
    """(x0, x1) hard-case arguments of a unary twofold function."""
    U = lambda s: uniform(seed, s, n, start)  # noqa: E731
    w = 2.0**-10
    if func in ("texp", "texpm1"):
        parts = [
            EXP_OVERFLOW + w * (2 * U(5) - 1),
            EXP_UNDERFLOW + w * (2 * U(6) - 1),
            EXP_SUBNORMAL + w * (2 * U(7) - 1),
            EXP_UNDERFLOW + (EXP_SUBNORMAL - EXP_UNDERFLOW) * U(8),
            _signs(seed, n, start) * np.exp2(-1074 + 1060 * U(9)),   # tiny arguments
            -40.0 + 2 * U(10) - 745 * (U(11) < 0.3),                   # expm1 saturating to -1
        ]
        if func == "texpm1":
            parts[5] = -(np.exp2(5.0 + 5.0 * U(10)))
    elif func == "tlog":
        parts = [
            1.0 + _signs(seed, n, start) * np.exp2(-60 + 40 * U(5)),  # 1 +- 2^-20 and closer
            np.exp2(-1074 + 52 * U(6)),                                  # subnormal y0
            np.exp2(1000 + 24 * U(7) * 0.999),                           # near DBL_MAX
            np.exp2(-1022 + 2044 * U(8)),
            1.0 + np.floor(U(9) * 2**20) * 2.0**-52,                     # 1 + a few ulps
        ]
    elif func == "tlog1p":
        parts = [
            -1.0 + np.exp2(-53 + 52 * U(5)),                             # near -1
            _signs(seed, n, start) * np.exp2(-1074 + 1060 * U(6)),     # tiny, incl. subnormal
            np.exp2(900 + 123 * U(7) * 0.999),                           # huge
            (2 * U(8) - 1) * 0.5 + 0.2,                                  # around the n = 0 band edges
            np.exp2(-20 + 19 * U(9)) * _signs(seed, n, start),
        ]
    else:
        raise KeyError(func)
    k = -(-n // len(parts))
    return _mix([p[:k] for p in parts], seed, n, start, 53)


# ---------------------------------------------------------------------------------
# Batched chains of twofold operations (step-major layout of include/tf.h).
# ---------------------------------------------------------------------------------

OP_ADD, OP_MUL, OP_EXP, OP_LOG = 0, 1, 2, 3
# streams of the chain draws (each draw has its own)
_C_LEN, _C_INIT, _C_OP, _C_OPFIX, _C_MAG, _C_PERT = 10, 11, 12, 13, 14, 15
_LO, _HI = 2.0**-20, 2.0**20
_EXP_MAX = 20.0 * math.log(2.0)                # e^s <= 2^20
_LOG_MIN = math.exp(2.0**-20)                  # log s >= 2^-20


def chains(n_chains: int, seed: int = 8, mean_len: float = 256.0, cap: int = 4096):
    """A batch of independent chains whose ops are drawn uniformly from
    {tadd, tmul, texp, tlog} and whose states stay in [2^-20, 2^20] (positive):

    * length L = min(1 + Geom(p = 1/mean_len), cap) (geometric with that mean);
    * initial state s0 uniform in [1, 2), s1 = s0 u 2^-53;
    * at each step the op is drawn uniformly; an op that would leave the range
      (texp with e^s > 2^20, tlog with log s < 2^-20, tadd with no room above s)
      is redrawn uniformly among the feasible ones;
    * tadd operand a0 log-uniform in [2^-20, 2^20 - s] (positive: no
      cancellation); tmul operand a0 = t / s with t log-uniform in
      [2^-20, 2^20]; a1 = a0 u 2^-53; texp/tlog carry a0 = a1 = 0.

    The host follows each state in plain double only to decide feasibility.
    Chains are numbered longest first; the op stream is step-major.  Returns a
    dict: ops (uint8), a0, a1 (float64), step_base (int64, max_len + 1),
    length (int32), s0, s1 (float64), max_len, mix (count per op)."""
    if n_chains <= 0:
        raise ValueError("n_chains must be positive")
    p = 1.0 / mean_len
    u = uniform(seed, _C_LEN, n_chains)
    L = 1 + np.floor(np.log1p(-u) / math.log1p(-p))
    L = np.minimum(L, cap).astype(np.int64)
    order = np.argsort(-L, kind="stable")       # longest first; ties by index
    L = L[order]
    max_len = int(L[0])
    s0 = 1.0 + uniform(seed, _C_INIT, n_chains)[order]
    s1 = s0 * (2 * uniform(seed, _C_PERT, n_chains)[order] - 1) * 2.0**-53
    active = np.searchsorted(-L, -np.arange(max_len), side="left")  # chains with L > t
    step_base = np.zeros(max_len + 1, dtype=np.int64)
    step_base[1:] = np.cumsum(active)
    total = int(step_base[-1])
    ops = np.empty(total, dtype=np.uint8)
    a0 = np.zeros(total)
    a1 = np.zeros(total)
    s = s0.copy()
    for t in range(max_len):
        m = int(active[t])
        ids = order[:m].astype(np.uint64) * np.uint64(cap) + np.uint64(t)   # per (chain, step) counter
        ids = ids.astype(np.int64)
        st = s[:m]
        U = lambda stream: _uniform_at(seed, stream, ids)  # noqa: E731
        feas = np.stack([st <= _HI - _LO, np.ones(m, bool), st <= _EXP_MAX, st >= _LOG_MIN], axis=1)
        op = np.minimum((U(_C_OP) * 4).astype(np.int64), 3)
        bad = ~feas[np.arange(m), op]
        if bad.any():  # redraw uniformly among the feasible ops
            nf = feas[bad].sum(axis=1)
            pick = np.minimum((U(_C_OPFIX)[bad] * nf).astype(np.int64), nf - 1)
            cum = np.cumsum(feas[bad], axis=1)
            op[bad] = np.argmax(cum > pick[:, None], axis=1)
        mag = U(_C_MAG)
        pert = 2 * U(_C_PERT) - 1
        x = np.zeros(m)
        add = op == OP_ADD
        hi = np.log2(np.maximum(_HI - st[add], _LO))
        x[add] = np.exp2(-20.0 + (hi + 20.0) * mag[add])
        mu = op == OP_MUL
        x[mu] = np.exp2(-20.0 + 40.0 * mag[mu]) / st[mu]
        sl = slice(int(step_base[t]), int(step_base[t + 1]))
        ops[sl] = op
        a0[sl] = x
        a1[sl] = x * pert * 2.0**-53
        with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
            s[:m] = np.where(add, st + x, np.where(mu, st * x, np.where(op == OP_EXP, np.exp(st), np.log(st))))
    mix = np.bincount(ops, minlength=4)
    return {"ops": ops, "a0": a0, "a1": a1, "step_base": step_base, "length": L.astype(np.int32),
            "s0": s0, "s1": s1, "max_len": max_len, "mix": mix}


def _uniform_at(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """U in [0, 1) at arbitrary counter indices (same generator as uniform())."""
    base = np.uint64((seed << 40) | (stream << 36))
    c = idx.astype(np.uint64) + base
    return (splitmix64(c) >> np.uint64(11)).astype(np.float64) * 2.0**-53


# ---------------------------------------------------------------------------------
# Float twofolds (the precision tier): float arguments, x1 = RN_f(x0 u 2^-24).
# ---------------------------------------------------------------------------------

EXPF_OVERFLOW = 88.72283935546875      # e^x rounds to +Inf in float from about here
EXPF_UNDERFLOW = -103.97207708          # e^x rounds to 0 in float below about here
EXPF_SUBNORMAL = -87.33654475           # e^x < 2^-126 below this

SPECIALS_F = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, 2.0**-149, -2.0**-149,
                       2.0**-126, 3.4028234663852886e38, -3.4028234663852886e38], dtype=np.float32)


def _f32(x):
    with np.errstate(over="ignore"):
        return np.asarray(x, dtype=np.float64).astype(np.float32)


def _perturb_f32(x0, seed, n, start):
    u = 2.0 * uniform(seed, S_PERT, n, start) - 1.0
    with np.errstate(invalid="ignore", over="ignore"):
        return _f32(x0.astype(np.float64) * u * 2.0**-24)


def workload_f32(func: str, n: int, start: int = 0):
    """(x0, x1) float32 arrays of a unary function's float workload:
      texp   x0 uniform in [-88, 88] (the double texp workload within float range)
      texpm1 random sign, |x0| log-uniform in [2^-40, 88]
      tlog   x0 log-uniform in [2^-126, 2^127]
      tlog1p half random sign |x0| log-uniform in [2^-40, 2^-10), half x0 = t - 1,
             t log-uniform in [2^-24, 2^100]
    and x1 = RN_f(x0 u 2^-24), u uniform in [-1, 1]."""
    seed = {"texp": 6, "texpm1": 16, "tlog": 7, "tlog1p": 17}[func]
    if func == "texp":
        x0 = _f32(-88.0 + 176.0 * uniform(seed, S_MAG, n, start))
    elif func == "texpm1":
        x0 = _f32(_signs(seed, n, start) * _loguniform(-40.0, math.log2(88.0), seed, n, start))
    elif func == "tlog":
        x0 = _f32(_loguniform(-126.0, 127.0, seed, n, start))
    else:
        pick = uniform(seed, S_PICK, n, start) < 0.5
        small = _signs(seed, n, start) * _loguniform(-40.0, -10.0, seed, n, start)
        t = _loguniform(-24.0, 100.0, seed, n, start)
        x0 = _f32(np.where(pick, small, t - 1.0))
    return x0, _perturb_f32(x0, seed, n, start)


def workload_f32_big(func: str, n: int, start: int = 0, chunk: int = 1 << 21):
    """workload_f32 for large n, drawn in chunks on a thread pool (each element
    depends on its index only, so the values are those of workload_f32)."""
    if n <= chunk:
        return workload_f32(func, n, start)
    from concurrent.futures import ThreadPoolExecutor
    import os
    pieces = [(s, min(chunk, n - s)) for s in range(0, n, chunk)]
    with ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 1)) as ex:
        parts = list(ex.map(lambda p: workload_f32(func, p[1], start + p[0]), pieces))
    return np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts])


def double_of_f32(func: str, x0f: np.ndarray, start: int = 0):
    """The double twofold over the same x0 values as a float workload (the
    precision-tier comparison): x0 exactly, x1 = RN(x0 u 2^-53) with the same u."""
    seed = {"texp": 6, "texpm1": 16, "tlog": 7, "tlog1p": 17}[func]
    x0 = x0f.astype(np.float64)
    return x0, _perturb(x0, seed, x0.shape[0], start, 53)


def _half_ulp_f32(x0):
    with np.errstate(invalid="ignore", over="ignore"):
        a = np.abs(x0.astype(np.float32))
        return ((np.nextafter(a, np.float32(np.inf)) - a) * np.float32(0.5)).astype(np.float32)


def hard_cases_f32(func: str, n: int, seed: int = 19, start: int = 0):
    """Float hard cases: thresholds of overflow/subnormal/underflow, tiny
    arguments, log near 1 and of subnormals, log1p near -1; x1 = 0 (10%),
    exactly +-half an ulp (5%), the IEEE specials paired at the end."""
    U = lambda s: uniform(seed, s, n, start)  # noqa: E731
    w = 2.0**-6
    if func in ("texp", "texpm1"):
        parts = [EXPF_OVERFLOW + w * (2 * U(5) - 1), EXPF_UNDERFLOW + w * (2 * U(6) - 1),
                 EXPF_SUBNORMAL + w * (2 * U(7) - 1),
                 EXPF_UNDERFLOW + (EXPF_SUBNORMAL - EXPF_UNDERFLOW) * U(8),
                 _signs(seed, n, start) * np.exp2(-149 + 140 * U(9)),
                 -(np.exp2(3.0 + 4.0 * U(10)))]
    elif func == "tlog":
        parts = [1.0 + _signs(seed, n, start) * np.exp2(-24 + 20 * U(5)), np.exp2(-149 + 23 * U(6)),
                 np.exp2(100 + 28 * U(7)), np.exp2(-126 + 253 * U(8))]
    else:
        parts = [-1.0 + np.exp2(-24 + 22 * U(5)), _signs(seed, n, start) * np.exp2(-149 + 140 * U(6)),
                 np.exp2(60 + 68 * U(7)), -0.5 + 0.25 * U(8)]
    k = -(-n // len(parts))
    x0 = _f32(np.concatenate([np.asarray(p)[:k] for p in parts])[:n])
    x1 = _perturb_f32(x0, seed, n, start)
    pick = U(4)
    sgn = np.where(U(1) < 0.5, -1.0, 1.0).astype(np.float32)
    x1 = np.where(pick < 0.10, np.float32(0.0), x1).astype(np.float32)
    x1 = np.where((pick >= 0.10) & (pick < 0.15), sgn * _half_ulp_f32(x0), x1).astype(np.float32)
    m = SPECIALS_F.shape[0]
    k = min(n, m * m)
    if k:
        x0[n - k:] = np.repeat(SPECIALS_F, m)[:k]
        x1[n - k:] = (np.tile(SPECIALS_F, m)[:k].astype(np.float64) * 2.0**-30).astype(np.float32)
    return x0, x1
