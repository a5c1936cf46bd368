"""Deterministic edge cases of the double logarithms (tlog, tlog1p) against the oracle.

The kernels reduce y = 2^n z by a reciprocal table (i = round(1024 z) in the
general core) and place the fixed-point sum by cases: units 2^-116 for n != 0,
2^-128 off the table's centre for n = 0, and relative to d = z - 1 at the centre
for n = 0 (switching at |d| = 2^-22 and, for the right shift of d c, at |d| =
2^-60).  tlog's sign-free core takes i = floor(1024 z) and j = floor(2^18 t1)
with tables rounded up, serves n = 0 outside [1 - 2^-10, 1 + 2^-22), and places
its n = 0 sum in units 2^-136 in cell 1024.  These inputs sit on every such
boundary:

* z on both sides of every table cell boundary (i +- 1/2)/1024, at several n;
* z on both sides of the sign-free core's cells i/1024 and of its second
  table's cells t1 = j 2^-18 (z = (1 + j 2^-18)/c_i), and of 1 - 2^-10,
  1 + 2^-22;
* exact powers of two (d = 0) over the whole exponent range;
* 1 +- 2^-k and their neighbours for every k (d crosses the placement switches);
* tlog1p: +-2^-k down to the subnormals, the edges of the n = 0 band, cell
  boundaries of 1 + y0 inside the band, and 1 + y0 inexact with n != 0 (the
  low part of 1 + y0 enters the sum).

x1 is zero for a third of the elements and y0 u 2^-53 (u uniform in (-1, 1))
otherwise.  Expectations are those of the other parity tests: z0 correctly
rounded, z0 + z1 within 2^-100 relative.
"""
import numpy as np
import pytest

import oracle
import tfcheck
from paper_1502_05216_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SPLIT_Z = 1.0 + 0x6a09e00000000 / 2.0**52  # the kernels' y = 2^n z split: z >= this is halved


@pytest.fixture(scope="module")
def tf():
    import torch
    from paper_1502_05216_gb300 import build, tf as tfmod
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    build.build()
    tfmod.load()
    return tfmod


def _around(v):
    v = np.asarray(v, dtype=np.float64)
    return np.concatenate([v, np.nextafter(v, -np.inf), np.nextafter(v, np.inf)])


def _with_x1(x0, seed):
    u = 2 * I.uniform(seed, 1, x0.size) - 1
    x1 = x0 * u * 2.0**-53
    x1[::3] = 0.0
    return x0, x1


def tlog_edges():
    cells = np.array([(i + h) / 1024 for i in range(724, 1449) for h in (-0.5, 0.5)])
    up = [i / 1024 for i in range(724, 1449)]
    for i in range(724, 1449, 9):
        ci = -(-(2**34) // i) / 2.0**24  # the sign-free core's c_i
        up += [(1 + j * 2.0**-18) / ci for j in (1, 2, 77, 200, 300, 362)]
    up += [1 - 2.0**-10, 1 - 2.0**-11, 1 + 2.0**-22, 1 + 2.0**-21, 1 + 2.0**-18]
    z = _around(np.concatenate([cells, up, [SPLIT_Z, SPLIT_Z / 2, 1.0]]))
    z = z[(z >= SPLIT_Z / 2) & (z < SPLIT_Z)]
    ys = [z * 2.0**k for k in (0, 1, -1, 7, -7, 300, -300, 1000, -1000)]
    ys.append(np.exp2(np.arange(-1074, 1024, dtype=np.float64)))      # powers of two
    k = np.arange(1, 60, dtype=np.float64)
    near1 = _around(np.concatenate([1.0 + 2.0**-k, 1.0 - 2.0**-k]))
    ys += [near1 * 2.0**s for s in (0, 1, -1, 20, -20)]
    x0 = np.concatenate(ys)
    return _with_x1(x0[np.isfinite(x0) & (x0 > 0)], 31)


def tlog1p_edges():
    k = np.arange(1, 1075, dtype=np.float64)
    tiny = np.concatenate([2.0**-k, -(2.0**-k)])
    band = _around([SPLIT_Z - 1, SPLIT_Z / 2 - 1, np.sqrt(2.0) - 1, np.sqrt(0.5) - 1])
    cells = _around(np.array([(i + h) / 1024 - 1 for i in range(724, 1449) for h in (-0.5, 0.5)]))
    # 1 + y0 inexact with n != 0: y0 = 2^m (1 + j 2^-40) and -1 + 2^-m (1 + j 2^-40)
    j = np.arange(1, 40, dtype=np.float64)
    m = np.arange(1, 60, dtype=np.float64)
    big = (2.0**m[:, None] * (1 + j[None, :] * 2.0**-40)).ravel()
    near_m1 = (-1.0 + 2.0**-m[:, None] * (1 + j[None, :] * 2.0**-40)).ravel()
    x0 = np.concatenate([tiny, band, cells, big, near_m1])
    return _with_x1(x0[np.isfinite(x0) & (x0 > -1)], 32)


@pytest.mark.parametrize("func,gen", [("tlog", tlog_edges), ("tlog1p", tlog1p_edges)])
def test_log_edges(tf, func, gen):
    import torch
    x0, x1 = gen()
    dev = [torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0") for a in (x0, x1)]
    z0, z1 = tf.FUNCS[func](*dev)
    torch.cuda.synchronize()
    orc = oracle.evaluate(func, x0, x1)
    st = tfcheck.check(z0.cpu().numpy(), z1.cpu().numpy(), orc, "f64", 0.9999, f"{func} edges", func, (x0, x1))
    assert st["mainpart_mismatch"] == 0, st
