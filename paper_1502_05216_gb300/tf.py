"""Python binding of libtf.so (argument marshalling only).

Every function takes float64 tensors on a CUDA device and enqueues the kernel
on the current torch stream (or the given one); all the arithmetic happens in
the CUDA kernels behind the C ABI of include/tf.h.  There is no CPU fallback:
without the built library or a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lib = None
_lock = threading.Lock()

UNARY = ("texp", "texpm1", "tlog", "tlog1p")
BINARY = ("tadd", "tmul")
# Coupled results (p...) and twofold results of coupled arguments (t...p).
COUPLED = ("pexp", "pexpm1", "plog", "plog1p", "texpp", "texpm1p", "tlogp", "tlog1pp")
# the same function computed another way (the paper's own exp reduction)
VARIANTS = ("texp_tables", "tlog_newton_fp64", "tlog1p_newton_fp64")


class TwofoldError(RuntimeError):
    pass


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libtf.so (it must have been built: paper_1502_05216_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or _build.LIB
        if not os.path.exists(p):
            raise TwofoldError(f"{p} is missing: build it with python -m paper_1502_05216_gb300.build")
        lib = ctypes.CDLL(p)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        for name in UNARY:
            f = getattr(lib, "tf_" + name)
            f.argtypes = [vp, vp, vp, vp, i64, vp]
            f.restype = i32
        for name in UNARY:
            f = getattr(lib, "tf_" + name + "f")
            f.argtypes = [vp, vp, vp, vp, i64, vp]
            f.restype = i32
        for name in COUPLED + VARIANTS:
            f = getattr(lib, "tf_" + name)
            f.argtypes = [vp, vp, vp, vp, i64, vp]
            f.restype = i32
        for name in BINARY:
            f = getattr(lib, "tf_" + name)
            f.argtypes = [vp, vp, vp, vp, vp, vp, i64, vp]
            f.restype = i32
        lib.tf_chain.argtypes = [vp, vp, vp, vp, vp, vp, vp, i64, ctypes.c_int32, vp, i32, i32, i32, vp]
        lib.tf_chain.restype = i32
        lib.tf_chain_noalloc.argtypes = [vp, vp, vp, vp, vp, vp, vp, i64, ctypes.c_int32, i32, i32, i32, vp]
        lib.tf_chain_noalloc.restype = i32
        lib.tf_chain_step.argtypes = [i32, vp, i64, i64, vp, vp, vp, vp, vp]
        lib.tf_chain_step.restype = i32
        lib.tf_strerror.argtypes = [i32]
        lib.tf_strerror.restype = ctypes.c_char_p
        lib.tf_version.restype = i32
        if path is None:
            _lib = lib
        return lib


def _check(rc: int, name: str):
    if rc != 0:
        raise TwofoldError(f"tf_{name}: {load().tf_strerror(rc).decode()} (code {rc})")


def _ptr(t, name, n, device, dtype=None):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    dtype = dtype or torch.float64
    if t.dtype != dtype or not t.is_cuda or t.device != device:
        raise TypeError(f"{name} must be a {dtype} CUDA tensor on {device}")
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be contiguous with {n} elements")
    return t.data_ptr()


def _stream(stream, device):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return s.cuda_stream


def _unary(name, x0, x1=None, out=None, stream=None):
    import torch
    n = x0.numel()
    dev = x0.device
    if out is None:
        out = (torch.empty_like(x0), torch.empty_like(x0))
    args = (_ptr(x0, "x0", n, dev), _ptr(x1, "x1", n, dev), _ptr(out[0], "z0", n, dev),
            _ptr(out[1], "z1", n, dev))
    with torch.cuda.device(dev):
        _check(getattr(load(), "tf_" + name)(*args, n, _stream(stream, dev)), name)
    return out


def _unary_f(name, x0, x1=None, out=None, stream=None):
    import torch
    n = x0.numel()
    dev = x0.device
    if out is None:
        out = (torch.empty_like(x0), torch.empty_like(x0))
    f32 = torch.float32
    args = (_ptr(x0, "x0", n, dev, f32), _ptr(x1, "x1", n, dev, f32), _ptr(out[0], "z0", n, dev, f32),
            _ptr(out[1], "z1", n, dev, f32))
    with torch.cuda.device(dev):
        _check(getattr(load(), "tf_" + name + "f")(*args, n, _stream(stream, dev)), name + "f")
    return out


def _binary(name, x0, x1, y0, y1, out=None, stream=None):
    import torch
    n = x0.numel()
    dev = x0.device
    if out is None:
        out = (torch.empty_like(x0), torch.empty_like(x0))
    args = (_ptr(x0, "x0", n, dev), _ptr(x1, "x1", n, dev), _ptr(y0, "y0", n, dev), _ptr(y1, "y1", n, dev),
            _ptr(out[0], "z0", n, dev), _ptr(out[1], "z1", n, dev))
    with torch.cuda.device(dev):
        _check(getattr(load(), "tf_" + name)(*args, n, _stream(stream, dev)), name)
    return out


def texp(x0, x1=None, out=None, stream=None):
    """(z0, z1) with z0 + z1 = e^(x0 + x1), z0 = RN(e^x0)."""
    return _unary("texp", x0, x1, out, stream)


def texpm1(x0, x1=None, out=None, stream=None):
    """(z0, z1) with z0 + z1 = e^(x0 + x1) - 1, z0 = RN(e^x0 - 1)."""
    return _unary("texpm1", x0, x1, out, stream)


def tlog(y0, y1=None, out=None, stream=None):
    """(z0, z1) with z0 + z1 = log(y0 + y1), z0 = RN(log y0)."""
    return _unary("tlog", y0, y1, out, stream)


def tlog1p(y0, y1=None, out=None, stream=None):
    """(z0, z1) with z0 + z1 = log(1 + y0 + y1), z0 = RN(log1p y0)."""
    return _unary("tlog1p", y0, y1, out, stream)


def tadd(x0, x1, y0, y1, out=None, stream=None):
    """(z0, z1) with z0 = x0 + y0 (plain) and z0 + z1 = (x0 + x1) + (y0 + y1)."""
    return _binary("tadd", x0, x1, y0, y1, out, stream)


def tmul(x0, x1, y0, y1, out=None, stream=None):
    """(z0, z1) with z0 = x0 * y0 (plain) and z0 + z1 = (x0 + x1)(y0 + y1)."""
    return _binary("tmul", x0, x1, y0, y1, out, stream)


def texpf(x0, x1=None, out=None, stream=None):
    """Float twofolds: (z0, z1) float32 with z0 + z1 = e^(x0 + x1), z0 = RN_f(e^x0)."""
    return _unary_f("texp", x0, x1, out, stream)


def texpm1f(x0, x1=None, out=None, stream=None):
    """Float twofolds: z0 + z1 = e^(x0 + x1) - 1."""
    return _unary_f("texpm1", x0, x1, out, stream)


def tlogf(y0, y1=None, out=None, stream=None):
    """Float twofolds: z0 + z1 = log(y0 + y1)."""
    return _unary_f("tlog", y0, y1, out, stream)


def tlog1pf(y0, y1=None, out=None, stream=None):
    """Float twofolds: z0 + z1 = log(1 + y0 + y1)."""
    return _unary_f("tlog1p", y0, y1, out, stream)


FUNCS_F = {"texp": texpf, "texpm1": texpm1f, "tlog": tlogf, "tlog1p": tlog1pf}


def pexp(x0, x1=None, out=None, stream=None):
    """Coupled (z0, z1): z0 + z1 = e^(x0 + x1) with z0 = RN(z0 + z1)."""
    return _unary("pexp", x0, x1, out, stream)


def pexpm1(x0, x1=None, out=None, stream=None):
    """Coupled (z0, z1): z0 + z1 = e^(x0 + x1) - 1 with z0 = RN(z0 + z1)."""
    return _unary("pexpm1", x0, x1, out, stream)


def plog(y0, y1=None, out=None, stream=None):
    """Coupled (z0, z1): z0 + z1 = log(y0 + y1) with z0 = RN(z0 + z1)."""
    return _unary("plog", y0, y1, out, stream)


def plog1p(y0, y1=None, out=None, stream=None):
    """Coupled (z0, z1): z0 + z1 = log(1 + y0 + y1) with z0 = RN(z0 + z1)."""
    return _unary("plog1p", y0, y1, out, stream)


def texpp(x0, x1=None, out=None, stream=None):
    """As texp for a coupled argument (no renormalising path for a loose x1)."""
    return _unary("texpp", x0, x1, out, stream)


def texpm1p(x0, x1=None, out=None, stream=None):
    """As texpm1 for a coupled argument."""
    return _unary("texpm1p", x0, x1, out, stream)


def tlogp(y0, y1=None, out=None, stream=None):
    """As tlog for a coupled argument."""
    return _unary("tlogp", y0, y1, out, stream)


def tlog1pp(y0, y1=None, out=None, stream=None):
    """As tlog1p for a coupled argument."""
    return _unary("tlog1pp", y0, y1, out, stream)


def texp_tables(x0, x1=None, out=None, stream=None):
    """texp computed with the paper's own table reduction (A/B variant)."""
    return _unary("texp_tables", x0, x1, out, stream)


def tlog_newton_fp64(y0, y1=None, out=None, stream=None):
    """tlog with its Newton step in binary64 (A/B variant)."""
    return _unary("tlog_newton_fp64", y0, y1, out, stream)


def tlog1p_newton_fp64(y0, y1=None, out=None, stream=None):
    """tlog1p with its Newton step in binary64 (A/B variant)."""
    return _unary("tlog1p_newton_fp64", y0, y1, out, stream)


# the A/B variants and the function each computes
VARIANT_FUNCS = {"texp_tables": (texp_tables, "texp"), "tlog_newton_fp64": (tlog_newton_fp64, "tlog"),
                 "tlog1p_newton_fp64": (tlog1p_newton_fp64, "tlog1p")}


FUNCS_C = {"pexp": pexp, "pexpm1": pexpm1, "plog": plog, "plog1p": plog1p,
           "texpp": texpp, "texpm1p": texpm1p, "tlogp": tlogp, "tlog1pp": tlog1pp}
# the twofold function each one is built on
BASE_OF = {"pexp": "texp", "pexpm1": "texpm1", "plog": "tlog", "plog1p": "tlog1p",
           "texpp": "texp", "texpm1p": "texpm1", "tlogp": "tlog", "tlog1pp": "tlog1p"}


# operation codes of the chain entry points (TF_OP_* in include/tf.h)
OP_ADD, OP_MUL, OP_EXP, OP_LOG = 0, 1, 2, 3
CHAIN_WORKSPACE = 256  # TF_CHAIN_WORKSPACE


def _dptr(t, name, dtype, device):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_cuda or t.device != device:
        raise TypeError(f"{name} must be a {dtype} CUDA tensor on {device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def chain(ops, a0, a1, step_base, length, s0, s1, max_len, workspace, threads=128, blocks=0, group=0,
          stream=None):
    """tf_chain: run every chain of a step-major batch to its end in one
    persistent launch; s0/s1 (float64) are updated in place.  ops uint8,
    step_base int64, length int32, workspace a uint8 tensor of
    CHAIN_WORKSPACE bytes; group = chains per warp (1 .. 32), 0 = by length."""
    import torch
    dev = s0.device
    n = s0.numel()
    if s1.numel() != n or length.numel() != n or step_base.numel() != int(max_len) + 1:
        raise ValueError("s0, s1, length must have one entry per chain; step_base max_len + 1")
    if workspace.numel() * workspace.element_size() < CHAIN_WORKSPACE:
        raise ValueError(f"workspace must hold {CHAIN_WORKSPACE} bytes")
    args = (_dptr(ops, "ops", torch.uint8, dev), _dptr(a0, "a0", torch.float64, dev),
            _dptr(a1, "a1", torch.float64, dev), _dptr(step_base, "step_base", torch.int64, dev),
            _dptr(length, "length", torch.int32, dev), _dptr(s0, "s0", torch.float64, dev),
            _dptr(s1, "s1", torch.float64, dev))
    if not workspace.is_cuda or workspace.device != dev:
        raise TypeError(f"workspace must be on {dev}")
    with torch.cuda.device(dev):
        _check(load().tf_chain(*args, n, int(max_len), workspace.data_ptr(), int(threads), int(blocks),
                               int(group), _stream(stream, dev)), "chain")


def chain_noalloc(ops, a0, a1, step_base, length, s0, s1, max_len, threads=128, blocks=0, group=0,
                  stream=None):
    """tf_chain_noalloc: as chain() but with the library's static scratch in
    place of a workspace, for callers that cannot allocate device memory (see
    include/tf.h); calls must not overlap on the GPU."""
    import torch
    dev = s0.device
    n = s0.numel()
    if s1.numel() != n or length.numel() != n or step_base.numel() != int(max_len) + 1:
        raise ValueError("s0, s1, length must have one entry per chain; step_base max_len + 1")
    args = (_dptr(ops, "ops", torch.uint8, dev), _dptr(a0, "a0", torch.float64, dev),
            _dptr(a1, "a1", torch.float64, dev), _dptr(step_base, "step_base", torch.int64, dev),
            _dptr(length, "length", torch.int32, dev), _dptr(s0, "s0", torch.float64, dev),
            _dptr(s1, "s1", torch.float64, dev))
    # the library finds the static scratch of the current device: make s0's
    # device current for the call
    with torch.cuda.device(dev):
        _check(load().tf_chain_noalloc(*args, n, int(max_len), int(threads), int(blocks), int(group),
                                       _stream(stream, dev)), "chain_noalloc")


def chain_step(op, idx, step_base_t, a0, a1, s0, s1, stream=None):
    """tf_chain_step: one operation kind at one step for the chains in idx (int32)."""
    import torch
    dev = s0.device
    args = (_dptr(idx, "idx", torch.int32, dev), idx.numel(), int(step_base_t),
            _dptr(a0, "a0", torch.float64, dev), _dptr(a1, "a1", torch.float64, dev),
            _dptr(s0, "s0", torch.float64, dev), _dptr(s1, "s1", torch.float64, dev))
    with torch.cuda.device(dev):
        _check(load().tf_chain_step(int(op), *args, _stream(stream, dev)), "chain_step")


FUNCS = {"texp": texp, "texpm1": texpm1, "tlog": tlog, "tlog1p": tlog1p, "tadd": tadd, "tmul": tmul}


class HostPipeline:
    """End-to-end evaluation on host arrays: the arrays are cut into chunks, and
    each chunk's host-to-device copy, kernel and device-to-host copy are
    enqueued on one of ``depth`` streams in turn, so the copy engines of one
    chunk overlap the kernels of the others.  Device staging buffers are
    allocated once per pipeline and reused.  Host arrays should be pinned
    (``torch.empty(..., pin_memory=True)``) for the copies to be asynchronous."""

    def __init__(self, device="cuda", chunk: int = 1 << 22, depth: int = 3):
        import torch
        self.device = torch.device(device)
        self.chunk = int(chunk)
        self.depth = int(depth)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(self.depth)]
        self.bufs = [[torch.empty(self.chunk, dtype=torch.float64, device=self.device) for _ in range(6)]
                     for _ in range(self.depth)]
        self.launches = 0

    def run(self, name, *host_arrays, out=None):
        """z0 + z1 = name(*host_arrays) into the pinned host pair ``out`` (allocated
        when None).  Returns ``out`` after the last copy has landed."""
        import torch
        h = [None if a is None else (a if isinstance(a, torch.Tensor) else torch.from_numpy(a))
             for a in host_arrays]
        n = h[0].numel()
        if out is None:
            out = (torch.empty(n, dtype=torch.float64, pin_memory=True),
                   torch.empty(n, dtype=torch.float64, pin_memory=True))
        cur = torch.cuda.current_stream(self.device)
        for st in self.streams:
            st.wait_stream(cur)
        for c, s in enumerate(range(0, n, self.chunk)):
            e = min(n, s + self.chunk)
            m = e - s
            slot = c % self.depth
            st = self.streams[slot]
            b = self.bufs[slot]
            with torch.cuda.stream(st):
                dargs = []
                for k, a in enumerate(h):
                    if a is None:
                        dargs.append(None)
                    else:
                        b[k][:m].copy_(a[s:e], non_blocking=True)
                        dargs.append(b[k][:m])
                FUNCS[name](*dargs, out=(b[4][:m], b[5][:m]), stream=st)
                self.launches += 1
                out[0][s:e].copy_(b[4][:m], non_blocking=True)
                out[1][s:e].copy_(b[5][:m], non_blocking=True)
        for st in self.streams:
            st.synchronize()
        return out


_pipes = {}


def _pinned_ptr(t, name, n):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float64 or not t.is_pinned():
        raise TypeError(f"{name} must be a pinned float64 CPU tensor for the zero-copy call")
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be contiguous with {n} elements")
    return t.data_ptr()


def call_host_zero_copy(name, *host_arrays, out=None, device="cuda", stream=None):
    """End-to-end call on pinned host arrays without staging copies: the kernel
    itself loads the arguments from pinned host memory and stores (z0, z1)
    there, over the GPU's link to host memory (pinned host memory is
    addressable from the device under unified addressing).  Returns ``out``
    after the kernel has finished."""
    import torch
    dev = torch.device(device)
    h = list(host_arrays)
    n = h[0].numel()
    if out is None:
        out = (torch.empty(n, dtype=torch.float64, pin_memory=True),
               torch.empty(n, dtype=torch.float64, pin_memory=True))
    names = ("x0", "x1") if len(h) == 2 else ("x0", "x1", "y0", "y1")
    args = [_pinned_ptr(a, nm, n) for a, nm in zip(h, names)] + [_pinned_ptr(out[0], "z0", n),
                                                                 _pinned_ptr(out[1], "z1", n)]
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    with torch.cuda.device(dev):
        _check(getattr(load(), "tf_" + name)(*args, n, st.cuda_stream), name)
    st.synchronize()
    return out


def call_host(name, *host_arrays, out=None, device="cuda", mode="zero-copy"):
    """End-to-end call on host arrays.  mode "zero-copy" (pinned float64 CPU
    tensors): call_host_zero_copy.  mode "pipeline" (numpy or CPU tensors,
    pinned for speed): copy in, run, copy (z0, z1) back, pipelined over chunks
    and streams (HostPipeline).  Returns CPU tensors (pinned when allocated here)."""
    import torch
    dev = torch.device(device)
    if mode == "zero-copy":
        return call_host_zero_copy(name, *host_arrays, out=out, device=dev)
    key = (dev.type, dev.index if dev.index is not None else torch.cuda.current_device())
    if key not in _pipes:
        _pipes[key] = HostPipeline(dev)
    return _pipes[key].run(name, *host_arrays, out=out)
