"""Positive control of the bounds-checked build (libtaser_debug.so): an index that fails its
check is counted, the record names its source, and the access it guards is skipped.

Runs only in a session that loads the debug library (TASER_LIBRARY=debug, which
test_gpu_debug_build.py starts); the release library is never given the invalid item.
The invalid item's offset (-1) names memory inside the pool's own allocation (64 floats
of headroom sit before T_pool[0]), so even an access that escaped the check would stay
in bounds.
"""
import os

import numpy as np
import pytest
import torch

from synth import make_mimo

pytestmark = [
    pytest.mark.gpu,
    pytest.mark.skipif(os.environ.get("TASER_LIBRARY") != "debug",
                       reason="needs the bounds-checked library (TASER_LIBRARY=debug)"),
]

FLAG_BAD_ITEM = 1 << 4


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_01797_gb300 as taser
    return taser


def test_counters_start_clean(T):
    rep = T.debug_report()
    assert rep["fails"] == 0, rep


def test_negative_item_offset_is_counted_and_skipped(T):
    N, t_max = 9, 10                                      # BPSK 32x8
    w = make_mimo(2, 32, 8, 10.0, "bpsk", seed=5)
    out = T.build_T("mimo_bpsk", torch.from_numpy(w["H"]).cuda(), torch.from_numpy(w["y"]).cuda(), 0.5)
    s_dense, _, _ = T.detect(out["T_tilde"], out["D"], out["tau"], t_max, "fp32", want_L=False)
    big = torch.zeros(64 + 2 * N * N, dtype=torch.float32, device="cuda")
    big[64:] = out["T_tilde"].reshape(-1)
    T_pool = big[64:]
    D_pool = out["D"].reshape(-1).contiguous()
    items = T.make_items([N, N], [t_max, t_max], [0, -1], [0, N], [0, N - 1])
    items_d = torch.from_numpy(items.view(np.uint8).copy()).cuda()
    s = torch.zeros(2 * (N - 1), dtype=torch.int8, device="cuda")
    flags = torch.zeros(2, dtype=torch.int32, device="cuda")
    ws = torch.empty(T.uneven_workspace_bytes(2), dtype=torch.uint8, device="cuda")
    assert T.debug_report()["fails"] == 0
    T.detect_uneven(items_d, T_pool, D_pool, out["tau"], s, ws, precision="fp32", flags=flags)
    torch.cuda.synchronize()
    rep = T.debug_report()
    assert rep["fails"] >= 1, rep
    assert rep["first"]["source"] == "uneven.cu", rep
    assert rep["first"]["index"] == 0xffffffff, rep       # the low 32 bits of -1
    fl = flags.cpu().numpy().astype(np.uint32)
    assert fl[1] & FLAG_BAD_ITEM and not fl[0] & FLAG_BAD_ITEM
    s = s.cpu().numpy()
    assert np.array_equal(s[:N - 1], s_dense[0].cpu().numpy())   # the valid item is detected
    assert not s[N - 1:].any()                                     # the invalid one is skipped
    assert T.debug_report()["fails"] == 0                          # reading cleared the counters


FLAG_TIMEOUT = 1 << 7


def test_withheld_staging_copy_times_out_and_is_flagged(T):
    """A TMA staging copy that never arrives: the bounded wait expires (about a second), the
    instance is flagged TASER_FLAG_TIMEOUT and its T~ and D stay unwritten, while the other
    instances are built as usual.  The copy is withheld, never issued, so nothing faults."""
    n, B, U = 8, 128, 16
    w = make_mimo(n, B, U, 8.0, "qpsk", seed=9)
    H, y = torch.from_numpy(w["H"]).cuda(), torch.from_numpy(w["y"]).cuda()
    ref = T.build_T("mimo_qpsk", H, y, 0.5)
    torch.cuda.synchronize()
    out = {k: torch.full_like(v, 7.0) if v.dtype == torch.float32 else torch.zeros_like(v) for k, v in ref.items()}
    T.debug_drop_copy(3, 2)
    try:
        T.build_T("mimo_qpsk", H, y, 0.5, out=out, with_tau=False)
        torch.cuda.synchronize()
    finally:
        T.debug_drop_copy(-1, 0)
    fl = out["flags"].cpu().numpy().astype(np.uint32)
    assert fl[3] == FLAG_TIMEOUT, fl
    assert (np.delete(fl, 3) == 0).all(), fl
    Tt, D = out["T_tilde"].cpu().numpy(), out["D"].cpu().numpy()
    assert (Tt[3] == 7.0).all() and (D[3] == 7.0).all()
    keep = [i for i in range(n) if i != 3]
    assert np.array_equal(Tt[keep], ref["T_tilde"].cpu().numpy()[keep])
    assert np.array_equal(D[keep], ref["D"].cpu().numpy()[keep])
    # with the injection off the same call builds every instance again
    T.build_T("mimo_qpsk", H, y, 0.5, out=out, with_tau=False)
    torch.cuda.synchronize()
    assert (out["flags"].cpu().numpy() == 0).all()
    assert np.array_equal(out["T_tilde"].cpu().numpy(), ref["T_tilde"].cpu().numpy())
    assert T.debug_report()["fails"] == 0
