"""tf_chain_noalloc against tf_chain, through the C ABI (GPU).

tf_chain_noalloc serves callers that cannot allocate device memory -- code
running where a host framework owns all of the device's memory (its own pool
or a hard cap), or on a latency-critical path that cannot afford cudaMalloc,
which may synchronize the whole device.  Instead of a caller-provided
workspace it keeps its work-queue counter in a static device array inside the
library.  Two calls in a row must each give exactly tf_chain's result: the
second call sees the counter the first one left behind, so this also checks
that every call clears it.  Bitwise equality is stricter than the 2^-97 K |F|
bound of the chain tests, which the result is also checked against.

This file is collected last so that a run that stops at the first failure
has already run every other test; it also passes when run on its own.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1502_05216_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1502_05216_gb300 import build, tf
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    build.build()
    return tf.load()


def _device_batch(batch):
    import torch
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()  # noqa: E731
    return {"ops": t(batch["ops"], np.uint8), "a0": t(batch["a0"], np.float64), "a1": t(batch["a1"], np.float64),
            "sb": t(batch["step_base"], np.int64), "len": t(batch["length"], np.int32),
            "s0": t(batch["s0"], np.float64), "s1": t(batch["s1"], np.float64)}


def _run(lib, d, batch, noalloc):
    import torch
    s0, s1 = d["s0"].clone(), d["s1"].clone()
    n, max_len = s0.numel(), int(batch["max_len"])
    p = [ctypes.c_void_p(x.data_ptr()) for x in (d["ops"], d["a0"], d["a1"], d["sb"], d["len"], s0, s1)]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if noalloc:
        rc = lib.tf_chain_noalloc(*p, n, max_len, 128, 0, 0, stream)
    else:
        ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
        rc = lib.tf_chain(*p, n, max_len, ctypes.c_void_p(ws.data_ptr()), 128, 0, 0, stream)
    assert rc == 0, lib.tf_strerror(rc).decode()
    torch.cuda.synchronize()
    return s0.cpu().numpy(), s1.cpu().numpy()


def test_noalloc_equals_workspace_entry_point_twice(lib):
    batches = [I.chains(6000, seed=51, mean_len=48.0, cap=400), I.chains(9000, seed=52, mean_len=32.0, cap=300)]
    for k, batch in enumerate(batches):  # two calls in a row on the static scratch
        d = _device_batch(batch)
        ref = _run(lib, d, batch, noalloc=False)
        got = _run(lib, d, batch, noalloc=True)
        assert np.array_equal(ref[0].view(np.int64), got[0].view(np.int64)), f"call {k + 1}: z0"
        assert np.array_equal(ref[1].view(np.int64), got[1].view(np.int64)), f"call {k + 1}: z1"
        Fh, Fl, K = oracle.chain(batch)
        err = np.abs((got[0] - Fh) + (got[1] - Fl))
        assert np.all(err <= 2.0**-97 * K * np.abs(Fh) + 2.0**-1060), f"call {k + 1}: beyond 2^-97 K |F|"


def test_noalloc_binding_equals_chain(lib):
    """The Python binding tf.chain_noalloc (which makes the tensors' device
    current for the call) against tf.chain, bit for bit, twice."""
    import torch
    from paper_1502_05216_gb300 import tf
    batch = I.chains(3000, seed=53, mean_len=40.0, cap=200)
    d = _device_batch(batch)
    ws = torch.zeros(tf.CHAIN_WORKSPACE, dtype=torch.uint8, device="cuda:0")
    for k in range(2):
        r0, r1 = d["s0"].clone(), d["s1"].clone()
        g0, g1 = d["s0"].clone(), d["s1"].clone()
        common = (d["ops"], d["a0"], d["a1"], d["sb"], d["len"])
        tf.chain(*common, r0, r1, int(batch["max_len"]), ws)
        tf.chain_noalloc(*common, g0, g1, int(batch["max_len"]))
        torch.cuda.synchronize()
        assert torch.equal(r0.view(torch.int64), g0.view(torch.int64)), f"call {k + 1}: z0"
        assert torch.equal(r1.view(torch.int64), g1.view(torch.int64)), f"call {k + 1}: z1"


def test_noalloc_rejects_bad_arguments(lib):
    # The pointers below are fake: every case must be rejected by the argument
    # checks, which come before any device access (the scratch lookup, the
    # memset and the launch), or return early with nothing to do.
    good = ctypes.c_void_p(1 << 20)
    g7 = [good] * 7
    assert lib.tf_chain_noalloc(*g7, (1 << 40) + 1, 5, 128, 0, 0, None) == 2  # beyond the maximum: TF_ERR_SIZE
    assert lib.tf_chain_noalloc(*g7, -1, 5, 128, 0, 0, None) == 2
    assert lib.tf_chain_noalloc(*g7, 10, 5, 48, 0, 0, None) == 6             # TF_ERR_ARG: block size
    assert lib.tf_chain_noalloc(*g7, 10, 5, 128, 0, 33, None) == 6           # TF_ERR_ARG: group
    assert lib.tf_chain_noalloc(*g7, 0, 5, 128, 0, 0, None) == 0             # nothing to do
