"""taser_run_host_static: the whole detector for callers that cannot allocate device
memory, whose scratch is a static device array inside the library.

This file is collected last (by name), so a failure here stops an -x run only after every
other test has run.  Each test stands alone: it builds the library if needed and makes
its own inputs.
"""
import ctypes
import os

import numpy as np
import pytest
import torch

from synth import make_jed, make_mimo


@pytest.fixture(scope="module")
def taser():
    from paper_1609_01797_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    import paper_1609_01797_gb300 as T
    return T


def test_static_scratch_rejects_batches_beyond_its_size(taser):
    """Needs no GPU: the size check comes before any device work."""
    from paper_1609_01797_gb300._native import STATIC_SCRATCH_BYTES, lib
    per = taser.host_workspace_bytes("mimo_qpsk", 1000, 128, 16) / 1000
    too_many = int(STATIC_SCRATCH_BYTES / per) + 100
    st = lib().taser_run_host_static(1, too_many, 128, 16, ctypes.c_void_p(16), ctypes.c_void_p(16), 0.5, 20, 1,
                                     0, ctypes.c_void_p(16), None, None)
    assert st == 1
    assert b"split the batch" in lib().taser_last_error()


def _inputs(kind, n, seed):
    if kind == "jed_bpsk":
        w = make_jed(n, 16, 32, np.linspace(0, 12, n), seed=seed)
        return w["Y"], None, 32
    w = make_mimo(n, 128, 16, np.linspace(0, 20, n), "qpsk", seed=seed)
    return w["H"], w["y"], 16


@pytest.mark.gpu
@pytest.mark.parametrize("kind,precision,t_max", [("mimo_qpsk", "bf16_tc", 20), ("jed_bpsk", "fp32", 20)])
def test_static_scratch_matches_workspace_entry_point(taser, kind, precision, t_max):
    """Two calls in a row through the C ABI give the decisions and flags of taser_run_host
    with a caller-allocated workspace (same kernels, so identical results)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = 1500
    for call, seed in enumerate((31, 32)):
        X, y, M = _inputs(kind, n, seed)
        N = taser.problem_size(kind, M)
        Xh = torch.from_numpy(X).pin_memory()
        yh = torch.from_numpy(y).pin_memory() if y is not None else None
        s_static = torch.full((n, N - 1), 7, dtype=torch.int8).pin_memory()
        f_static = torch.full((n,), -1, dtype=torch.int32).pin_memory()
        taser.run_host_static(kind, Xh, yh, 0.5, t_max, precision, s_static, flags=f_static)
        torch.cuda.synchronize()
        ws = torch.empty(taser.host_workspace_bytes(kind, n, X.shape[1], M), device="cuda", dtype=torch.uint8)
        s_ref = torch.empty((n, N - 1), dtype=torch.int8).pin_memory()
        f_ref = torch.empty((n,), dtype=torch.int32).pin_memory()
        taser.run_host(kind, Xh, yh, 0.5, t_max, precision, ws, s_ref, flags=f_ref)
        torch.cuda.synchronize()
        assert torch.all(s_static.abs() == 1), call
        np.testing.assert_array_equal(s_static.numpy(), s_ref.numpy())
        np.testing.assert_array_equal(f_static.numpy(), f_ref.numpy())


@pytest.mark.gpu
def test_static_scratch_largest_batch_that_fits(taser):
    """The largest QPSK 128x16 batch whose scratch fits the static array, so the last
    chunk's buffers (decisions and flags) end at the array's end: the same decisions and
    flags as taser_run_host with a caller-allocated workspace of that size."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01797_gb300._native import STATIC_SCRATCH_BYTES
    lo, hi = 1, 1 << 16
    while lo < hi:                       # largest n with host_workspace_bytes(n) <= the array
        mid = (lo + hi + 1) // 2
        if taser.host_workspace_bytes("mimo_qpsk", mid, 128, 16) <= STATIC_SCRATCH_BYTES:
            lo = mid
        else:
            hi = mid - 1
    n = lo
    assert taser.host_workspace_bytes("mimo_qpsk", n + 1, 128, 16) > STATIC_SCRATCH_BYTES
    X, y, M = _inputs("mimo_qpsk", n, 33)
    Xh, yh = torch.from_numpy(X).pin_memory(), torch.from_numpy(y).pin_memory()
    s_static = torch.full((n, 32), 7, dtype=torch.int8).pin_memory()
    f_static = torch.full((n,), -1, dtype=torch.int32).pin_memory()
    taser.run_host_static("mimo_qpsk", Xh, yh, 0.5, 20, "bf16_tc", s_static, flags=f_static)
    torch.cuda.synchronize()
    ws = torch.empty(taser.host_workspace_bytes("mimo_qpsk", n, 128, 16), device="cuda", dtype=torch.uint8)
    s_ref = torch.empty((n, 32), dtype=torch.int8).pin_memory()
    f_ref = torch.empty((n,), dtype=torch.int32).pin_memory()
    taser.run_host("mimo_qpsk", Xh, yh, 0.5, 20, "bf16_tc", ws, s_ref, flags=f_ref)
    torch.cuda.synchronize()
    assert torch.all(s_static.abs() == 1)
    np.testing.assert_array_equal(s_static.numpy(), s_ref.numpy())
    np.testing.assert_array_equal(f_static.numpy(), f_ref.numpy())
