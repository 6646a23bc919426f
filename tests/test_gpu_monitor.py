"""Objective monitoring on the GPU (taser_detect_monitored): the trace f(L~(t)) =
Tr(L~ T~ L~^T), t = 0..t_max, and the ascent flag, against f evaluated in FP64 by the
oracle on the path's own iterates L~(t) (taser_detect run for t = 1..t_max; the kernels
are deterministic, so these are the monitored call's iterates), and, for FP32, against
the FP64 oracle's trajectory.

Prop. 1 (Sec. III-E) guarantees descent only for a small enough step (alpha < 1/2 with
the Lipschitz constant 2||T~||_2 of tril(2 L~ T~)); at alpha = 0.95 a few percent of
random BPSK 32x16 instances have an iteration in which f rises, by up to several percent.

Tolerances: the trace within 1e-5 (FP32) or 1e-4 (tensor cores, BF16 split monitor
product) of max_t |f| per instance.  Flags (ascent_tol 1e-5 FP32, 1e-4 tensor cores): a
rise above 1e-3 of the path's own iterates must be flagged, a rise below 1e-6 (FP32) or
1e-5 (tensor cores) must not be; the band between is left free.
"""
import numpy as np
import pytest
import torch

from oracle import taser_oracle as O
from synth import make_jed, make_mimo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_01797_gb300 as taser
    return taser


def oracle_trace(Tt, D, tau, t_max, mode):
    _, _, Ls = O.taser(Tt, D, tau, t_max, lnn_mode=mode, history=True)
    f = np.stack([O.objective(L, Tt) for L in Ls], axis=1)          # [n, t_max + 1]
    rise = ((f[:, 1:] - f[:, :-1]) / np.abs(f[:, :-1])).max(axis=1)
    return f, rise


def setup(kind, n, B, M, snr, seed, alpha):
    if kind.startswith("jed"):
        w = make_jed(n, B, M, snr, seed=seed)
        X, y = w["Y"], None
    else:
        w = make_mimo(n, B, M, snr, kind.split("_")[1], seed=seed)
        X, y = w["H"], w["y"]
    r = O.detect(kind, X, y, alpha, 1)
    Tt = r["T_tilde"].astype(np.float32)
    D = r["D"].astype(np.float32)
    tau = O.step_size(Tt.astype(np.float64), alpha).astype(np.float32)
    return Tt, D, tau


def dev(*a):
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in a]


def own_trace(T, dT, dD, dtau, Tt, D, t_max, precision, mode):
    """f in FP64 on the path's own iterates: L~(0) = D and L~(t) from taser_detect(t)."""
    Tt64 = Tt.astype(np.float64)
    f = [O.objective(np.einsum("ni,ij->nij", D.astype(np.float64), np.eye(D.shape[1])), Tt64)]
    for t in range(1, t_max + 1):
        _, L, _ = T.detect(dT, dD, dtau, t, precision, lnn_mode=mode)
        f.append(O.objective(L.cpu().numpy().astype(np.float64), Tt64))
    f = np.stack(f, axis=1)
    rise = ((f[:, 1:] - f[:, :-1]) / np.abs(f[:, :-1])).max(axis=1)
    return f, rise


@pytest.mark.parametrize("kind,B,M,precision,mode", [
    ("mimo_bpsk", 32, 16, "fp32", "fixed"), ("mimo_bpsk", 32, 16, "fp32", "literal"),
    ("mimo_qpsk", 128, 16, "fp32", "fixed"), ("mimo_qpsk", 256, 32, "fp32", "fixed"),
    ("jed_bpsk", 16, 32, "fp32", "fixed"), ("mimo_bpsk", 32, 4, "bf16_tc", "fixed"),
    ("mimo_bpsk", 32, 16, "bf16_tc", "fixed"), ("mimo_bpsk", 48, 32, "fp16_tc", "fixed"),
    ("mimo_qpsk", 128, 16, "bf16_tc", "fixed"), ("mimo_qpsk", 64, 12, "bf16_tc", "literal"),
    ("jed_bpsk", 16, 32, "bf16_tc", "fixed")])
def test_objective_trace_and_ascent_flag(T, kind, B, M, precision, mode):
    n, t_max, alpha = 3000, 20, 0.95
    snr = np.linspace(0.0, 12.0 if kind.startswith("jed") else 15.0, n)
    Tt, D, tau = setup(kind, n, B, M, snr, seed=60 + M, alpha=alpha)
    tc = precision != "fp32" and Tt.shape[1] >= 10
    tol = 1e-4 if tc else 1e-5
    dT, dD, dtau = dev(Tt, D, tau)
    s, L, flags, obj = T.detect_monitored(dT, dD, dtau, t_max, precision, ascent_tol=tol, lnn_mode=mode)
    s_ref, L_ref, f_ref = T.detect(dT, dD, dtau, t_max, precision, lnn_mode=mode)
    torch.cuda.synchronize()
    # the monitored call changes nothing else
    assert torch.equal(s, s_ref) and torch.equal(L, L_ref)
    fl = flags.cpu().numpy().astype(np.uint32)
    np.testing.assert_array_equal(fl & ~np.uint32(T.FLAG_ASCENT), f_ref.cpu().numpy().astype(np.uint32))
    f = obj.cpu().numpy()
    f_own, rise = own_trace(T, dT, dD, dtau, Tt, D, t_max, precision, mode)
    scale = np.abs(f_own).max(axis=1)
    err = (np.abs(f - f_own).max(axis=1) / scale).max()
    assert err <= (1e-4 if tc else 1e-5), err
    if not tc:
        f_o, rise_o = oracle_trace(Tt.astype(np.float64), D.astype(np.float64), tau.astype(np.float64), t_max, mode)
        assert (np.abs(f - f_o).max(axis=1) / scale).max() <= 1e-5
    flagged = (fl & T.FLAG_ASCENT) != 0
    must = rise > 1e-3
    must_not = rise < (1e-5 if tc else 1e-6)
    assert flagged[must].all(), (np.nonzero(must & ~flagged)[0][:5], rise[must & ~flagged][:5])
    assert not flagged[must_not].any(), (np.nonzero(must_not & flagged)[0][:5])
    if kind == "mimo_bpsk" and M == 16:
        assert must.sum() >= 20          # the case has real ascents to catch


@pytest.mark.parametrize("precision", ["fp32", "bf16_tc"])
def test_no_ascent_below_half(T, precision):
    """alpha = 0.45 < 1/2: the oracle's objective never rises; the FP32 path flags nothing,
    and the tensor-core path flags nothing whose own iterates do not rise by 1e-5."""
    n, t_max = 3000, 20
    Tt, D, tau = setup("mimo_bpsk", n, 32, 16, np.linspace(0.0, 15.0, n), seed=71, alpha=0.45)
    _, rise_o = oracle_trace(Tt.astype(np.float64), D.astype(np.float64), tau.astype(np.float64), t_max, "fixed")
    assert (rise_o <= 0).all()
    dT, dD, dtau = dev(Tt, D, tau)
    tc = precision != "fp32"
    _, _, flags, _ = T.detect_monitored(dT, dD, dtau, t_max, precision, ascent_tol=1e-4 if tc else 1e-5,
                                        want_L=False)
    torch.cuda.synchronize()
    flagged = (flags.cpu().numpy().astype(np.uint32) & T.FLAG_ASCENT) != 0
    if tc:
        _, rise = own_trace(T, dT, dD, dtau, Tt, D, t_max, precision, "fixed")
        assert not flagged[rise < 1e-5].any()
    else:
        assert not flagged.any()
