"""Parity at the full sizes of the workload configurations, in the launch configurations the
benchmark uses: every instance where the oracle is cheap (BPSK 32x8, 1,024 instances),
sampled instances against the oracle elsewhere, and properties that hold at any size on
all instances (lower-triangular L~, column norms D, decisions +-1, BER near the oracle's).

Tolerances as in test_gpu_parity: FP32 1e-5 relative Frobenius on L~ (decisions identical
beyond 1e-3 of the row norm), tensor cores 3e-2 (beyond 5e-2)."""
import numpy as np
import pytest
import torch

from oracle import taser_oracle as O
from synth import make_jed, make_mimo, make_uneven

pytestmark = pytest.mark.gpu
ALPHA = 0.5


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_01797_gb300 as taser
    return taser


def dev(*a):
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in a]


def rel_frob(A, B):
    return np.linalg.norm(A - B, axis=(1, 2)) / np.linalg.norm(B, axis=(1, 2))


def confident(L, margin):
    row = L[:, -1, :]
    return np.abs(row[:, :-1]) > margin * np.linalg.norm(row, axis=1, keepdims=True)


def test_bpsk_32x8_all_1024_instances(T):
    """BPSK 32x8 (N = 9), 1,024 instances at 10 dB, t_max = 10, seed 0: every instance of
    the FP32 path against the FP64 oracle, end to end from H and y."""
    w = make_mimo(1024, 32, 8, 10.0, "bpsk", seed=0)
    r = O.detect("mimo_bpsk", w["H"], w["y"], ALPHA, 10)
    out = T.build_T("mimo_bpsk", *dev(w["H"], w["y"]), alpha=ALPHA)
    s, L, flags = T.detect(out["T_tilde"], out["D"], out["tau"], 10, "fp32", flags=out["flags"])
    torch.cuda.synchronize()
    L = L.cpu().numpy().astype(np.float64)
    assert rel_frob(L, r["L"]).max() <= 1e-5
    m = confident(r["L"], 1e-3)
    np.testing.assert_array_equal(s.cpu().numpy()[m], r["s_hat"][m])
    assert int((s.cpu().numpy() != w["bits_re"]).sum()) == int((r["s_hat"] != w["bits_re"]).sum())
    assert not np.any(flags.cpu().numpy())


@pytest.mark.parametrize("K", [16, 32])
@pytest.mark.parametrize("precision", ["fp32", "bf16_tc"])
def test_jed_bpsk_131072_sampled(T, K, precision):
    """SIMO JED BPSK, B = 16, K = 16 and 32 slots (pilot first), 131,072 instances, SNR
    0..12 dB, t_max = 20: 128 sampled instances against the oracle, properties on all."""
    n = 131072
    snr = np.tile(np.arange(0.0, 13.0, 2.0), n // 7 + 1)[:n]
    w = make_jed(n, 16, K, snr, seed=2000 + K)
    out = T.build_T("jed_bpsk", *dev(w["Y"]), None, alpha=ALPHA)
    s, L, flags = T.detect(out["T_tilde"], out["D"], out["tau"], 20, precision, flags=out["flags"])
    torch.cuda.synchronize()
    idx = np.random.default_rng(K).choice(n, 128, replace=False)
    r = O.detect("jed_bpsk", w["Y"][idx], None, ALPHA, 20)
    Ls = L[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.float64)
    assert rel_frob(Ls, r["L"]).max() <= (1e-5 if precision == "fp32" else 3e-2)
    m = confident(r["L"], 1e-3 if precision == "fp32" else 5e-2)
    np.testing.assert_array_equal(s.cpu().numpy()[idx][m], r["s_hat"][m])
    assert torch.all(torch.triu(L, 1) == 0)
    # column norms D (the last column holds L~_NN = D_N)
    assert torch.allclose(torch.linalg.vector_norm(L, dim=1), out["D"], rtol=1e-4)
    s = s.cpu().numpy()
    assert np.all(np.abs(s) == 1)
    truth = w["s"][:, 1:]
    # bit errors on the sample agree with the oracle's up to its unconfident entries
    assert abs(int((s[idx] != truth[idx]).sum()) - int((r["s_hat"] != truth[idx]).sum())) <= int((~m).sum())
    assert np.mean(s != truth) < 0.1


@pytest.mark.parametrize("precision", ["fp32", "bf16_tc"])
def test_uneven_200000_sampled(T, precision):
    """The uneven batch of the benchmark (200,000 QPSK items, (B, U) in {(32,4), (64,8),
    (128,16), (256,32)}, t_max 10 or 20) through one detect_uneven call: 160 sampled items
    (40 per size) against the oracle run on the same device-built T~, D, tau."""
    n = 200000
    w = make_uneven(n, seed=3)
    shapes = w["shapes"]
    Ns = np.array([2 * u + 1 for _, u in shapes])[w["shape_idx"]]
    tm = w["t_max"]
    t_off = np.zeros(n, np.int64)
    d_off = np.zeros(n, np.int64)
    T_parts, D_parts, tau = [], [], torch.empty(n, device="cuda")
    host = {}
    t_base = d_base = 0
    for si, ps in enumerate(w["per_shape"]):
        N_ = 2 * shapes[si][1] + 1
        out = T.build_T("mimo_qpsk", *dev(ps["H"], ps["y"]), alpha=ALPHA)
        sel = ps["items"]
        t_off[sel] = t_base + np.arange(len(sel)) * N_ * N_
        d_off[sel] = d_base + np.arange(len(sel)) * N_
        t_base += len(sel) * N_ * N_
        d_base += len(sel) * N_
        T_parts.append(out["T_tilde"].reshape(-1))
        D_parts.append(out["D"].reshape(-1))
        tau[torch.from_numpy(sel).cuda()] = out["tau"]
        pick = np.random.default_rng(si).choice(len(sel), 40, replace=False)
        host[si] = (sel[pick], out["T_tilde"][pick].cpu().numpy(), out["D"][pick].cpu().numpy(),
                    out["tau"][pick].cpu().numpy())
    s_off = np.concatenate([[0], np.cumsum(Ns - 1)[:-1]])
    l_off = np.concatenate([[0], np.cumsum(Ns * Ns)[:-1]])
    items = torch.from_numpy(T.make_items(Ns, tm, t_off, d_off, s_off, l_off).view(np.uint8).copy()).cuda()
    s_pool = torch.empty(int((Ns - 1).sum()), dtype=torch.int8, device="cuda")
    L_pool = torch.empty(int((Ns * Ns).sum()), dtype=torch.float32, device="cuda")
    flags = torch.zeros(n, dtype=torch.int32, device="cuda")
    ws = torch.empty(T.uneven_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    T.detect_uneven(items, torch.cat(T_parts), torch.cat(D_parts), tau, s_pool, ws, precision=precision,
                    L_pool=L_pool, flags=flags)
    torch.cuda.synchronize()
    s_pool, L_pool = s_pool.cpu().numpy(), L_pool.cpu().numpy()
    assert np.all(np.abs(s_pool) == 1)
    for si, (sel, Tt, D, ta) in host.items():
        N_ = 2 * shapes[si][1] + 1
        for t in (10, 20):
            k = tm[sel] == t
            if not k.any():
                continue
            Lo, _ = O.taser(Tt[k].astype(np.float64), D[k].astype(np.float64), ta[k].astype(np.float64), t)
            Lg = np.stack([L_pool[l_off[i]:l_off[i] + N_ * N_].reshape(N_, N_) for i in sel[k]]).astype(np.float64)
            assert rel_frob(Lg, Lo).max() <= (1e-5 if precision == "fp32" else 3e-2), (N_, t)
            m = confident(Lo, 1e-3 if precision == "fp32" else 5e-2)
            sg = np.stack([s_pool[s_off[i]:s_off[i] + N_ - 1] for i in sel[k]])
            np.testing.assert_array_equal(sg[m], O.decisions(Lo)[m])


def test_unfolded_training_batch_8192(T):
    """Unfolded TASER training at its batch size (8,192 fresh QPSK 128x16 instances, SNR
    uniform in [4, 14] dB, t_max = 10, checkpoints every 4 iterations): the per-instance
    dloss/dtau_t of 64 sampled instances equal the FP64 reverse mode, and the batch
    gradient dloss/dalpha_t equals the FP64 sum of the GPU's per-instance terms."""
    n, t_max, c = 8192, 10, 4
    w = make_mimo(n, 128, 16, np.random.default_rng(5).uniform(4, 14, n), "qpsk", seed=8192)
    out = T.build_T("mimo_qpsk", *dev(w["H"], w["y"]), alpha=ALPHA)
    inv = 1.0 / out["spec_norm"]
    alpha = torch.full((t_max,), 0.5, device="cuda")
    soft, _, ckpt = T.unfolded_forward(out["T_tilde"], out["D"], inv, alpha, c)
    truth = torch.from_numpy(np.concatenate([w["bits_re"], w["bits_im"]], 1).astype(np.float32)).cuda()
    g_soft = 2.0 * (soft - truth) / soft.numel()
    grad_tau, grad_alpha = T.unfolded_backward(out["T_tilde"], out["D"], inv, alpha, c, ckpt, g_soft)
    torch.cuda.synchronize()
    assert torch.isfinite(grad_tau).all() and torch.isfinite(grad_alpha).all()
    idx = np.random.default_rng(1).choice(n, 64, replace=False)
    ti = torch.from_numpy(idx).cuda()
    Tt = out["T_tilde"][ti].cpu().numpy().astype(np.float64)
    D = out["D"][ti].cpu().numpy().astype(np.float64)
    tau_t = (0.5 * inv[ti]).cpu().numpy().astype(np.float64)[:, None].repeat(t_max, axis=1)
    _, Ls = O.unfolded_forward(Tt, D, tau_t)
    g_o = O.unfolded_backward(Tt, D, tau_t, Ls, g_soft[ti].cpu().numpy().astype(np.float64))
    g = grad_tau[ti].cpu().numpy().astype(np.float64)
    scale = np.abs(g_o).max(axis=1, keepdims=True) + 1e-30
    assert (np.abs(g - g_o) / scale).max() <= 2e-3
    ga = (grad_tau.double() * inv.double()[:, None]).sum(dim=0).cpu().numpy()
    np.testing.assert_allclose(grad_alpha.cpu().numpy(), ga, rtol=1e-5, atol=1e-7 * np.abs(ga).max())
