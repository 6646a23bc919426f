"""Unfolded TASER on the GPU (learnable per-iteration steps): forward, checkpoints and the
hand-written adjoint against the FP64 oracle (whose adjoint is pinned by finite
differences and the dot-product test on the CPU).

Tolerances: soft outputs and checkpoints within 1e-5 (FP32 iterations, as for the
detector); dloss/dalpha_t within 1e-5 relative of the FP64 sum of the GPU's own
per-instance gradients; dloss/dtau_t within 1e-3 of the largest entry per instance.  The
adjoint walks t_max steps in reverse, and each step multiplies the adjoint by the prox
Jacobian, whose column factor D_k / ||V_.k|| reaches about 2 when a column of V has
shrunk to half of D_k (common on these channels: the smallest ratio per instance has a
median of 0.5 to 0.7), and by I - 2 tau T~ (norm up to 1 + 2 alpha).  A rounding error of
2^-24 made at a late step therefore reaches the early tau_t amplified by up to ~2^t, while
the early entries are not the largest.  Measured against the FP64 reverse mode over 5,632
instances of these five configurations: median 2e-7 to 6e-6, 99th percentile up to 2.5e-4, max
7.4e-4 (QPSK 32x4, t_max = 10) of the per-instance largest entry.
"""
import numpy as np
import pytest
import torch

from oracle import taser_oracle as O
from synth import make_mimo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_01797_gb300 as taser
    return taser


def setup(n, B, U, const, t_max, seed):
    w = make_mimo(n, B, U, np.linspace(2.0, 14.0, n), const, seed=seed)
    kind = "mimo_" + const
    r = O.detect(kind, w["H"], w["y"], 0.5, 1)
    Tt = r["T_tilde"].astype(np.float32)
    D = r["D"].astype(np.float32)
    inv = (1.0 / O.spectral_norm(r["T_tilde"])).astype(np.float32)
    rng = np.random.default_rng(seed)
    alpha = rng.uniform(0.3, 0.7, size=t_max).astype(np.float32)
    truth = w["bits_re"] if const == "bpsk" else np.concatenate([w["bits_re"], w["bits_im"]], 1)
    return Tt, D, inv, alpha, truth.astype(np.float64)


def dev(*a):
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in a]


CASES = [(96, 32, 4, "qpsk", 10, 4), (64, 16, 16, "bpsk", 7, 3), (128, 128, 16, "qpsk", 10, 4),
         (40, 24, 8, "qpsk", 20, 5), (33, 12, 5, "bpsk", 5, 5)]


@pytest.mark.parametrize("n,B,U,const,t_max,c", CASES)
def test_unfolded_forward_and_checkpoints(T, n, B, U, const, t_max, c):
    Tt, D, inv, alpha, _ = setup(n, B, U, const, t_max, seed=U)
    tau_t = alpha[None, :].astype(np.float64) * inv[:, None].astype(np.float64)
    L, Ls = O.unfolded_forward(Tt.astype(np.float64), D.astype(np.float64), tau_t)
    soft_o = O.soft_output(L, D.astype(np.float64))
    soft, s_hat, ckpt = T.unfolded_forward(*dev(Tt, D, inv, alpha), c)
    torch.cuda.synchronize()
    assert np.abs(soft.cpu().numpy() - soft_o).max() <= 1e-5
    np.testing.assert_array_equal(s_hat.cpu().numpy(), np.where(L[:, -1, :-1] >= 0, 1, -1)[:, :])
    ck = ckpt.cpu().numpy().astype(np.float64)
    for k in range(ck.shape[1]):
        ref = Ls[k * c]
        err = np.linalg.norm(ck[:, k] - ref, axis=(1, 2)) / np.linalg.norm(ref, axis=(1, 2))
        assert err.max() <= 1e-5, (k, err.max())


@pytest.mark.parametrize("n,B,U,const,t_max,c", CASES)
def test_unfolded_backward_matches_oracle(T, n, B, U, const, t_max, c):
    Tt, D, inv, alpha, truth = setup(n, B, U, const, t_max, seed=100 + U)
    dT, dD, dinv, dalpha = dev(Tt, D, inv, alpha)
    soft, _, ckpt = T.unfolded_forward(dT, dD, dinv, dalpha, c)
    x = soft.cpu().numpy().astype(np.float64)
    g_soft = (2.0 * (x - truth) / x.size).astype(np.float32)       # MSE loss gradient
    grad_tau, grad_alpha = T.unfolded_backward(dT, dD, dinv, dalpha, c, ckpt, dev(g_soft)[0])
    torch.cuda.synchronize()
    tau_t = alpha[None, :].astype(np.float64) * inv[:, None].astype(np.float64)
    _, Ls = O.unfolded_forward(Tt.astype(np.float64), D.astype(np.float64), tau_t)
    g_o = O.unfolded_backward(Tt.astype(np.float64), D.astype(np.float64), tau_t, Ls, g_soft.astype(np.float64))
    g = grad_tau.cpu().numpy().astype(np.float64)
    scale = np.abs(g_o).max(axis=1, keepdims=True) + 1e-30
    assert (np.abs(g - g_o) / scale).max() <= 1e-3, (np.abs(g - g_o) / scale).max()
    ga = (g * inv[:, None].astype(np.float64)).sum(axis=0)
    np.testing.assert_allclose(grad_alpha.cpu().numpy(), ga, rtol=1e-5, atol=1e-7 * np.abs(ga).max())


def test_checkpoint_spacing_does_not_change_the_gradient(T):
    Tt, D, inv, alpha, truth = setup(72, 64, 8, "qpsk", 12, seed=5)
    dT, dD, dinv, dalpha = dev(Tt, D, inv, alpha)
    g_soft = dev((np.random.default_rng(1).standard_normal((72, 16)) * 1e-3).astype(np.float32))[0]
    ref = None
    for c in (1, 3, 4, 12):
        soft, _, ckpt = T.unfolded_forward(dT, dD, dinv, dalpha, c)
        gt, _ = T.unfolded_backward(dT, dD, dinv, dalpha, c, ckpt, g_soft)
        torch.cuda.synchronize()
        if ref is None:
            ref = gt.clone()
        assert torch.equal(gt, ref), c


def test_wide_checkpoint_spacing_at_n33(T):
    """At N = 33 the packed shared-memory iterates admit c up to 92 (c + 2 iterates of 612
    floats for a one-warp block); every spacing gives the same gradient bit for bit, and
    c = 93 is rejected on the host before any launch."""
    t_max = 21
    Tt, D, inv, alpha, truth = setup(40, 128, 16, "qpsk", t_max, seed=9)
    dT, dD, dinv, dalpha = dev(Tt, D, inv, alpha)
    g_soft = dev((np.random.default_rng(2).standard_normal((40, 32)) * 1e-3).astype(np.float32))[0]
    ref = None
    for c in (1, 5, 20, 21):
        soft, _, ckpt = T.unfolded_forward(dT, dD, dinv, dalpha, c)
        gt, _ = T.unfolded_backward(dT, dD, dinv, dalpha, c, ckpt, g_soft)
        torch.cuda.synchronize()
        if ref is None:
            ref = gt.clone()
        assert torch.equal(gt, ref), c
    Tt2, D2, inv2, alpha2, _ = setup(8, 128, 16, "qpsk", 93, seed=3)
    a2 = dev(Tt2, D2, inv2, alpha2)
    soft, _, ckpt = T.unfolded_forward(*a2, 93)
    with pytest.raises(Exception, match="shared memory"):
        T.unfolded_backward(*a2, 93, ckpt, torch.zeros_like(soft))


def test_unfolded_training_lowers_the_loss(T):
    """A few Adam steps on alpha_t with fresh seeded QPSK 128x16 batches (N = 33,
    t_max = 10, c = 4) lower the MSE between the soft last row and the symbols."""
    t_max, c = 10, 4
    alpha = torch.full((t_max,), 0.5, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([alpha], lr=0.05)
    losses = []
    for step in range(12):
        w = make_mimo(1024, 128, 16, np.random.default_rng(step).uniform(4, 14, 1024), "qpsk", seed=700 + step)
        out = T.build_T("mimo_qpsk", *dev(w["H"], w["y"]), alpha=0.5)
        inv = 1.0 / out["spec_norm"]
        truth = dev(np.concatenate([w["bits_re"], w["bits_im"]], 1).astype(np.float32))[0]
        soft = T.UnfoldedTASER.apply(alpha, out["T_tilde"], out["D"], inv, c)
        loss = torch.mean((soft - truth) ** 2)
        opt.zero_grad()
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert alpha.grad is not None and torch.isfinite(alpha.grad).all()
    assert np.mean(losses[-3:]) < losses[0]


def test_alpha_gradient_matches_gpu_central_differences():
    """d loss / d alpha_t of the GPU adjoint at N = 9 (QPSK 32x4, FP32 kernels) against
    central differences of the loss taken in FP64 on the host from two GPU forward calls
    per t (alpha_t +- h, h = 1e-3 alpha_t).  Averaging over 8,192 instances brings the
    rounding noise of the FP32 soft outputs in the loss to about 1e-9, so the differences
    carry about 1e-6 absolute error; the truncation error is O(h^2)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_01797_gb300 as taser
    n, t_max, c = 8192, 6, 3
    Tt, D, inv, _, truth = setup(n, 32, 4, "qpsk", t_max, seed=77)
    alpha = np.array([0.55, 0.35, 0.62, 0.48, 0.41, 0.58], dtype=np.float32)
    dT, dD, dinv = dev(Tt, D, inv)

    def loss(a):
        soft, _, _ = taser.unfolded_forward(dT, dD, dinv, dev(a.astype(np.float32))[0], c, want_ckpt=False)
        x = soft.cpu().numpy().astype(np.float64)
        return np.mean((x - truth) ** 2), x

    _, x = loss(alpha)
    g_soft = (2.0 * (x - truth) / x.size).astype(np.float32)
    soft, _, ckpt = taser.unfolded_forward(dT, dD, dinv, dev(alpha)[0], c)
    _, g_alpha = taser.unfolded_backward(dT, dD, dinv, dev(alpha)[0], c, ckpt, dev(g_soft)[0])
    g = g_alpha.cpu().numpy().astype(np.float64)
    fd = np.zeros(t_max)
    for t in range(t_max):
        h = 1e-3 * alpha[t]
        ap, am = alpha.astype(np.float64).copy(), alpha.astype(np.float64).copy()
        ap[t] += h
        am[t] -= h
        # the steps actually used are the FP32-rounded ones
        hp = np.float32(ap[t]) - np.float32(alpha[t])
        hm = np.float32(alpha[t]) - np.float32(am[t])
        fd[t] = (loss(ap)[0] - loss(am)[0]) / (float(hp) + float(hm))
    assert np.abs(g - fd).max() <= 2e-3 * np.abs(fd).max() + 1e-7, (g, fd)


# Tensor-core unfolded TASER (BF16/FP16 products, FP32 master iterates and prox), bucket 32.
TC_CASES = [(96, 128, 16, "qpsk", 10, 4, "bf16_tc"), (64, 24, 12, "qpsk", 7, 3, "bf16_tc"),
            (80, 40, 20, "bpsk", 10, 4, "fp16_tc"), (48, 64, 32, "bpsk", 12, 5, "bf16_tc"),
            (40, 128, 16, "qpsk", 20, 5, "fp16_tc")]


@pytest.mark.parametrize("n,B,U,const,t_max,c,precision", TC_CASES)
def test_unfolded_tensor_core_forward(T, n, B, U, const, t_max, c, precision):
    """Soft outputs within 1e-2 and checkpoints within the detector's tensor-core tolerance
    (3e-2 relative Frobenius) of the FP64 oracle; decisions equal wherever |x_k| exceeds
    5e-2 ||x||."""
    Tt, D, inv, alpha, _ = setup(n, B, U, const, t_max, seed=200 + U)
    tau_t = alpha[None, :].astype(np.float64) * inv[:, None].astype(np.float64)
    L, Ls = O.unfolded_forward(Tt.astype(np.float64), D.astype(np.float64), tau_t)
    soft_o = O.soft_output(L, D.astype(np.float64))
    soft, s_hat, ckpt = T.unfolded_forward(*dev(Tt, D, inv, alpha), c, precision=precision)
    torch.cuda.synchronize()
    assert np.abs(soft.cpu().numpy() - soft_o).max() <= 1e-2
    conf = np.abs(soft_o) > 5e-2 * np.linalg.norm(soft_o, axis=1, keepdims=True)
    np.testing.assert_array_equal(s_hat.cpu().numpy()[conf], np.where(soft_o >= 0, 1, -1)[conf])
    ck = ckpt.cpu().numpy().astype(np.float64)
    for k in range(ck.shape[1]):
        ref = Ls[k * c]
        err = np.linalg.norm(ck[:, k] - ref, axis=(1, 2)) / np.linalg.norm(ref, axis=(1, 2))
        assert err.max() <= 3e-2, (k, err.max())


@pytest.mark.parametrize("n,B,U,const,t_max,c,precision", TC_CASES)
def test_unfolded_tensor_core_backward(T, n, B, U, const, t_max, c, precision):
    """dloss/dtau_t of the tensor-core adjoint against the FP64 reverse mode (on the FP64
    forward): the adjoint differentiates the tensor-core forward, whose products carry
    about 2^-8 relative error, so the entries agree to 5e-2 of the batch's largest entry
    (not of each instance's: where an instance has converged to an exact sign pattern its
    FP64 gradient is ~1e-13 and the tensor-core iterates' rounding noise, ~1e-7, is all
    that remains), and dloss/dalpha_t, the sum over the batch, to 5e-2 of its largest entry."""
    Tt, D, inv, alpha, truth = setup(n, B, U, const, t_max, seed=300 + U)
    dT, dD, dinv, dalpha = dev(Tt, D, inv, alpha)
    soft, _, ckpt = T.unfolded_forward(dT, dD, dinv, dalpha, c, precision=precision)
    x = soft.cpu().numpy().astype(np.float64)
    g_soft = (2.0 * (x - truth) / x.size).astype(np.float32)
    grad_tau, grad_alpha = T.unfolded_backward(dT, dD, dinv, dalpha, c, ckpt, dev(g_soft)[0], precision=precision)
    torch.cuda.synchronize()
    tau_t = alpha[None, :].astype(np.float64) * inv[:, None].astype(np.float64)
    _, Ls = O.unfolded_forward(Tt.astype(np.float64), D.astype(np.float64), tau_t)
    g_o = O.unfolded_backward(Tt.astype(np.float64), D.astype(np.float64), tau_t, Ls, g_soft.astype(np.float64))
    g = grad_tau.cpu().numpy().astype(np.float64)
    assert np.abs(g - g_o).max() <= 5e-2 * np.abs(g_o).max(), np.abs(g - g_o).max() / np.abs(g_o).max()
    ga = (g * inv[:, None].astype(np.float64)).sum(axis=0)
    ga_o = (g_o * inv[:, None].astype(np.float64)).sum(axis=0)
    assert np.abs(ga - ga_o).max() <= 5e-2 * np.abs(ga_o).max(), (ga, ga_o)
    np.testing.assert_allclose(grad_alpha.cpu().numpy(), ga, rtol=1e-5, atol=1e-7 * np.abs(ga).max())


def test_unfolded_tensor_core_checkpoint_spacing_and_small_n(T):
    """Every checkpoint spacing gives the same tensor-core gradient bit for bit; below the
    tensor-core bucket (N <= 17) the tensor-core precisions run the FP32 kernels."""
    Tt, D, inv, alpha, truth = setup(50, 128, 16, "qpsk", 12, seed=7)
    dT, dD, dinv, dalpha = dev(Tt, D, inv, alpha)
    g_soft = dev((np.random.default_rng(3).standard_normal((50, 32)) * 1e-3).astype(np.float32))[0]
    ref = None
    for c in (1, 3, 4, 12):
        soft, _, ckpt = T.unfolded_forward(dT, dD, dinv, dalpha, c, precision="bf16_tc")
        gt, _ = T.unfolded_backward(dT, dD, dinv, dalpha, c, ckpt, g_soft, precision="bf16_tc")
        torch.cuda.synchronize()
        if ref is None:
            ref = gt.clone()
        assert torch.equal(gt, ref), c
    Tt, D, inv, alpha, _ = setup(30, 32, 8, "qpsk", 6, seed=8)        # N = 17
    a = dev(Tt, D, inv, alpha)
    s32, _, _ = T.unfolded_forward(*a, 3, precision="fp32")
    stc, _, _ = T.unfolded_forward(*a, 3, precision="bf16_tc")
    assert torch.equal(s32, stc)


def test_unfolded_tensor_core_training_lowers_the_loss(T):
    t_max, c = 10, 4
    alpha = torch.full((t_max,), 0.5, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([alpha], lr=0.05)
    losses = []
    for step in range(12):
        w = make_mimo(1024, 128, 16, np.random.default_rng(step).uniform(4, 14, 1024), "qpsk", seed=800 + step)
        out = T.build_T("mimo_qpsk", *dev(w["H"], w["y"]), alpha=0.5)
        truth = dev(np.concatenate([w["bits_re"], w["bits_im"]], 1).astype(np.float32))[0]
        soft = T.UnfoldedTASER.apply(alpha, out["T_tilde"], out["D"], 1.0 / out["spec_norm"], c, "bf16_tc")
        loss = torch.mean((soft - truth) ** 2)
        opt.zero_grad()
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert torch.isfinite(alpha.grad).all()
    assert np.mean(losses[-3:]) < losses[0]
