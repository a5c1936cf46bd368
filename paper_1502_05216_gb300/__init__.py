"""Twofold exp/log on GB300: z0 + z1 = f(x0 + x1) for f in exp, expm1, log,
log1p (plus twofold add and multiply), evaluated elementwise by hand-written
sm_103a CUDA kernels behind a C ABI (include/tf.h).

The Python layer only marshals arguments (see ``tf.py``); the library is built
in-tree by ``build.py``.
"""
from .tf import (TwofoldError, call_host, load, tadd, texp, texpm1, tlog, tlog1p,  # noqa: F401
                 tmul)
