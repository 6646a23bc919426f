"""TASER_FIXED14 (the 14-bit datapath of Sec. IV-D) on the GPU against the integer
fixed-point oracle: bit-exact L~ codes, decisions and flags (integer work), at sizes
spanning every bucket, ragged batches, saturation, non-finite input, the uneven path and
the full-size QPSK 128x16 workload (sampled)."""
import numpy as np
import pytest
import torch

from oracle import taser_fixed_oracle as F
from oracle import taser_oracle as O
from synth import make_mimo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_01797_gb300 as taser
    return taser


def oracle_inputs(N, n, seed, snr=6.0, const="bpsk"):
    U = N - 1 if const == "bpsk" else (N - 1) // 2
    w = make_mimo(n, max(2 * U, 4), U, snr, const, seed=seed)
    r = O.detect("mimo_" + const, w["H"], w["y"], 0.5, 1)
    return r["T_tilde"].astype(np.float32), r["D"].astype(np.float32), r["tau"].astype(np.float32)


def dev(*a):
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in a]


def check_exact(T, Tt, D, tau, t_max):
    s, L, flags = T.detect(*dev(Tt, D, tau), t_max, "fixed14")
    torch.cuda.synchronize()
    ref = F.taser_fixed(Tt, D, tau, t_max)
    np.testing.assert_array_equal(L.cpu().numpy(), ref["L_real"].astype(np.float32))
    np.testing.assert_array_equal(s.cpu().numpy(), ref["s_hat"])
    np.testing.assert_array_equal(flags.cpu().numpy().astype(np.uint32), ref["flags"])
    return ref


@pytest.mark.parametrize("N", [2, 3, 5, 9, 10, 16, 17, 18, 31, 33, 34, 50, 64, 65])
@pytest.mark.parametrize("t_max", [1, 20])
def test_fixed14_bit_exact(T, N, t_max):
    n = 67 if N > 33 else 131                        # several blocks and a ragged tail
    Tt, D, tau = oracle_inputs(N, n, seed=5000 + N)
    check_exact(T, Tt, D, tau, t_max)


def test_fixed14_qpsk_and_low_snr(T):
    Tt, D, tau = oracle_inputs(33, 150, seed=5101, snr=0.0, const="qpsk")
    check_exact(T, Tt, D, tau, 20)


def test_fixed14_saturation_and_nonfinite(T):
    Tt, D, tau = oracle_inputs(17, 64, seed=5202)
    D = D.copy()
    D[::3, -1] = 300.0                                 # L~_NN register out of range
    D[1::3, 4] = 40.0                                  # a diagonal PE out of range
    Tt = Tt.copy()
    Tt[2, 3, 5] = np.nan
    ref = check_exact(T, Tt, D, tau, 10)
    assert np.all(ref["flags"][::3] & F.FLAG_SATURATED) and ref["flags"][2] & F.FLAG_SATURATED


def test_fixed14_zero_column(T):
    Tt, D, tau = oracle_inputs(9, 40, seed=5303)
    Tt = Tt.copy()
    D = D.copy()
    Tt[5, 2, :] = 0.0
    Tt[5, :, 2] = 0.0
    D[5, 2] = 0.0                                      # column 2 starts and stays at zero
    ref = check_exact(T, Tt, D, tau, 5)
    assert ref["flags"][5] & F.FLAG_ZERO_COLUMN


def test_fixed14_rejects_literal_mode(T):
    Tt, D, tau = oracle_inputs(9, 4, seed=1)
    with pytest.raises(Exception, match="FIXED14"):
        T.detect(*dev(Tt, D, tau), 5, "fixed14", "literal")


def test_fixed14_uneven_equals_dense(T):
    rng = np.random.default_rng(3)
    per, items = {}, []
    for N in (5, 17, 33, 65):
        per[N] = oracle_inputs(N, 60, seed=5400 + N)
        items += [(N, int(rng.choice([3, 20])), k) for k in range(60)]
    items = [items[i] for i in rng.permutation(len(items))]
    Ns = np.array([i[0] for i in items])
    tm = np.array([i[1] for i in items])
    t_off = np.concatenate([[0], np.cumsum(Ns * Ns)[:-1]])
    d_off = np.concatenate([[0], np.cumsum(Ns)[:-1]])
    s_off = np.concatenate([[0], np.cumsum(Ns - 1)[:-1]])
    Tp = np.concatenate([per[N][0][k].ravel() for N, _, k in items])
    Dp = np.concatenate([per[N][1][k] for N, _, k in items])
    tau = np.array([per[N][2][k] for N, _, k in items], dtype=np.float32)
    it = T.make_items(Ns, tm, t_off, d_off, s_off, t_off)
    s = torch.zeros(int((Ns - 1).sum()), dtype=torch.int8, device="cuda")
    L = torch.zeros(int((Ns * Ns).sum()), dtype=torch.float32, device="cuda")
    flags = torch.zeros(len(items), dtype=torch.int32, device="cuda")
    ws = torch.empty(T.uneven_workspace_bytes(len(items)), dtype=torch.uint8, device="cuda")
    T.detect_uneven(torch.from_numpy(it.view(np.uint8).copy()).cuda(), *dev(Tp, Dp, tau), s, ws,
                    precision="fixed14", L_pool=L, flags=flags)
    torch.cuda.synchronize()
    s, L, flags = s.cpu().numpy(), L.cpu().numpy(), flags.cpu().numpy().astype(np.uint32)
    for i, (N, t, k) in enumerate(items):
        Tt, D, ta = per[N]
        ref = F.taser_fixed(Tt[k:k + 1], D[k:k + 1], ta[k:k + 1], t)
        np.testing.assert_array_equal(s[s_off[i]:s_off[i] + N - 1], ref["s_hat"][0])
        np.testing.assert_array_equal(L[t_off[i]:t_off[i] + N * N].reshape(N, N), ref["L_real"][0].astype(np.float32))
        assert flags[i] == ref["flags"][0]


def test_fixed14_full_size_qpsk_128x16_sampled(T):
    """The benchmark's workload shape (65,536 QPSK 128x16 instances, t_max = 20) through the
    device build_T + step size + fixed-point detect; 96 sampled instances are recomputed by
    the oracle from the same device-built T~, D, tau."""
    n = 65536
    w = make_mimo(n, 128, 16, np.arange(n) % 11 * 2.0, "qpsk", seed=1)
    out = T.build_T("mimo_qpsk", *dev(w["H"], w["y"]), alpha=0.5)
    s, L, flags = T.detect(out["T_tilde"], out["D"], out["tau"], 20, "fixed14")
    torch.cuda.synchronize()
    idx = np.random.default_rng(0).choice(n, 96, replace=False)
    Tt = out["T_tilde"][idx].cpu().numpy()
    D = out["D"][idx].cpu().numpy()
    tau = out["tau"][idx].cpu().numpy()
    ref = F.taser_fixed(Tt, D, tau, 20)
    np.testing.assert_array_equal(L[idx].cpu().numpy(), ref["L_real"].astype(np.float32))
    np.testing.assert_array_equal(s[idx].cpu().numpy(), ref["s_hat"])
    np.testing.assert_array_equal(flags[idx].cpu().numpy().astype(np.uint32), ref["flags"])


def test_fixed14_loss_against_fp32(T):
    """Sec. V-A: the 14-bit design loses little against floating point.  65,536 16x16 BPSK
    instances per SNR: the fixed-point VER stays within 15% (about 0.2 dB on this slope)
    of the FP32 VER plus counting noise."""
    for snr in (8.0, 11.0):
        n = 65536
        w = make_mimo(n, 16, 16, snr, "bpsk", seed=int(snr))
        out = T.build_T("mimo_bpsk", *dev(w["H"], w["y"]), alpha=0.5)
        truth = torch.from_numpy(w["bits_re"]).cuda()
        ver = {}
        for p in ("fp32", "fixed14"):
            s, _, _ = T.detect(out["T_tilde"], out["D"], out["tau"], 10, p, want_L=False)
            ver[p] = (s != truth).any(dim=1).float().mean().item()
        assert ver["fixed14"] <= 1.15 * ver["fp32"] + 4 * np.sqrt(ver["fp32"] / n), (snr, ver)
