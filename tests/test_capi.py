"""The C ABI library without a GPU: it builds, loads, exports every entry point
that include/tf.h declares, and rejects bad arguments before touching CUDA."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tf.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tf_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1502_05216_gb300 import build, tf
    build.build()
    return tf.load()


def test_header_declares_the_entry_points():
    names = declared()
    for f in ("tf_texp", "tf_texpm1", "tf_tlog", "tf_tlog1p", "tf_tadd", "tf_tmul", "tf_strerror",
              "tf_texpf", "tf_texpm1f", "tf_tlogf", "tf_tlog1pf", "tf_chain", "tf_chain_step"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared():
        assert hasattr(lib, name), f"{name} declared in tf.h but not exported"


def test_tables_are_current():
    from paper_1502_05216_gb300 import build
    build.check_tables()


def test_error_codes_before_any_launch(lib):
    """Argument checks return before any CUDA call, so they run here."""
    good = ctypes.c_void_p(1 << 20)        # 16-byte aligned, never dereferenced
    odd = ctypes.c_void_p((1 << 20) + 4)  # not 8-byte aligned
    for name in ("tf_texp", "tf_texpm1", "tf_tlog", "tf_tlog1p"):
        f = getattr(lib, name)
        assert f(good, good, good, good, 0, None) == 0                 # n == 0: no-op
        assert f(good, good, good, good, -1, None) == 2                # TF_ERR_SIZE
        assert f(None, good, good, good, 5, None) == 1                 # TF_ERR_NULL
        assert f(good, good, None, good, 5, None) == 1
        assert f(good, good, good, None, 5, None) == 1
        assert f(odd, good, good, good, 5, None) == 3                  # TF_ERR_ALIGN
        assert f(good, odd, good, good, 5, None) == 3
    odd2 = ctypes.c_void_p((1 << 20) + 2)  # not 4-byte aligned
    for name in ("tf_texpf", "tf_texpm1f", "tf_tlogf", "tf_tlog1pf"):
        f = getattr(lib, name)
        assert f(good, good, good, good, 0, None) == 0
        assert f(good, good, good, good, -1, None) == 2
        assert f(None, good, good, good, 5, None) == 1
        assert f(odd2, good, good, good, 5, None) == 3
        assert f(good, good, good, odd2, 5, None) == 3
    for name in ("tf_tadd", "tf_tmul"):
        f = getattr(lib, name)
        assert f(good, good, good, good, good, good, 0, None) == 0
        assert f(good, good, good, good, good, good, -3, None) == 2
        assert f(good, good, None, good, good, good, 3, None) == 1
        assert f(good, good, good, odd, good, good, 3, None) == 3
    # chains: sizes, block size and op code are checked first
    # (tf.load() declared the argument types of every entry point)
    g7 = [good] * 7
    assert lib.tf_chain(*g7, 0, 5, good, 128, 0, 0, None) == 0      # no chains: no-op
    assert lib.tf_chain(*g7, -1, 5, good, 128, 0, 0, None) == 2     # TF_ERR_SIZE
    assert lib.tf_chain(*g7, 10, -1, good, 128, 0, 0, None) == 2
    assert lib.tf_chain(*g7, 10, 5, good, 33, 0, 0, None) == 6      # TF_ERR_ARG: not a warp multiple
    assert lib.tf_chain(*g7, 10, 5, good, 2048, 0, 0, None) == 6
    assert lib.tf_chain(*g7, 10, 5, good, 128, 0, 33, None) == 6    # TF_ERR_ARG: group
    assert lib.tf_chain(*g7, 10, 5, None, 128, 0, 0, None) == 1     # no workspace
    assert lib.tf_chain(*g7, 10, 5, odd, 128, 0, 0, None) == 3
    assert lib.tf_chain_step(7, good, 5, 0, good, good, good, good, None) == 6
    assert lib.tf_chain_step(0, good, 0, 0, good, good, good, good, None) == 0
    assert lib.tf_chain_step(1, good, -2, 0, good, good, good, good, None) == 2
    assert lib.tf_chain_step(2, None, 5, 0, good, good, good, good, None) == 1
    assert lib.tf_strerror(2).decode() == "n is negative or too large"
    assert lib.tf_strerror(12345).decode() == "unknown error code"
    assert lib.tf_version() >> 16 == 1


def test_binding_has_no_cpu_fallback():
    """The Python binding refuses CPU tensors instead of computing on the host."""
    import torch
    from paper_1502_05216_gb300 import tf
    x = torch.zeros(4, dtype=torch.float64)
    with pytest.raises(TypeError):
        tf.texp(x, x)


def test_failed_cuda_call_is_never_ok(lib):
    """With no usable CUDA device, calls whose arguments pass the checks reach
    the CUDA runtime, which fails; the entry points must report that failure
    (TF_ERR_NODEVICE or TF_ERR_LAUNCH), also when called a second time (the
    runtime clears a non-sticky error when it is read).  Runs only where no
    CUDA device is visible: the pointers are fake, and nothing may be launched
    on them."""
    import torch
    if torch.cuda.is_available() or torch.cuda.device_count() > 0:
        pytest.skip("a CUDA device is visible: the fake pointers must not reach a launch")
    good = ctypes.c_void_p(1 << 20)
    g7 = [good] * 7
    for _ in range(2):
        assert lib.tf_chain(*g7, 10, 5, good, 128, 0, 0, None) in (4, 5)
        assert lib.tf_chain(*g7, 10, 5, good, 128, 64, 0, None) in (4, 5)
        assert lib.tf_chain_noalloc(*g7, 10, 5, 128, 0, 0, None) in (4, 5)
        assert lib.tf_texp(good, good, good, good, 5, None) in (4, 5)
        assert lib.tf_chain_step(0, good, 5, 0, good, good, good, good, None) in (4, 5)
