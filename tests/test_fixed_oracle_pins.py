"""Pins of the fixed-point oracle (oracle/taser_fixed_oracle.py) against facts that do not
come from the oracle itself: exact integer rounding of the inverse square-root LUT
(Sec. IV-D), exact rational arithmetic for the rounding and normalisation steps, the FP64
oracle (itself pinned in test_oracle_pins.py) reached by the same datapath at wide
formats, invariants of the prox, and the paper's statement that the 14-bit designs lose
little against floating point (Sec. V-A)."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import taser_fixed_oracle as F
from oracle import taser_oracle as O
from synth import make_jed, make_mimo

# Same bit layout as the paper's datapath (8 / 7 / 5 fraction bits: alignment shifts of 1
# and 2 bits), 26-30 fraction bits elsewhere and a 2^22-entry LUT.
WIDE = dict(bits=40, frac_l=24, frac_last=23, frac_lnn=21, frac_t=26, lut_index_bits=22, lut_frac=30)


def inputs(kind, n, B, M, snr, seed, alpha=0.5):
    if kind == "jed_bpsk":
        w = make_jed(n, B, M, snr, seed=seed)
        r = O.detect(kind, w["Y"], None, alpha, 1)
    else:
        w = make_mimo(n, B, M, snr, kind[5:], seed=seed)
        r = O.detect(kind, w["H"], w["y"], alpha, 1)
    return r["T_tilde"].astype(np.float32), r["D"].astype(np.float32), r["tau"].astype(np.float32), w


def test_lut_entries_are_exactly_rounded():
    """LUT[i] = round(2^13 / sqrt((i + 1/2) / 512)) = round(2^18 / sqrt(2i + 1)): e is that
    integer iff (2e - 1)^2 (2i + 1) <= 2^38 < (2e + 1)^2 (2i + 1) (exact integers)."""
    lut = F.inverse_sqrt_lut()
    assert lut.shape == (2048,)
    assert np.all(lut[:512] == 0)
    for i in range(512, 2048):
        e = int(lut[i])
        assert (2 * e - 1) ** 2 * (2 * i + 1) <= 2 ** 38 < (2 * e + 1) ** 2 * (2 * i + 1), i
    body = lut[512:]
    assert body.max() <= 8192 and body.min() > 4096           # 1/sqrt(m), m in [1, 4), 13 fraction bits
    assert np.all(np.diff(body) <= 0)
    assert body.max() < 2 ** 14                                 # 14-bit words


def test_lut_index_normalisation_is_exact():
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.integers(1, 2 ** 40, 400), np.arange(1, 300), [2 ** k for k in range(40)],
                         [2 ** k - 1 for k in range(1, 40)]]).astype(np.int64)
    idx, s = F.lut_index_and_shift(xs)
    for x, i, e in zip(xs.tolist(), idx.tolist(), s.tolist()):
        assert e % 2 == 0 and 2 ** e <= x < 2 ** (e + 2)
        assert i == (x << 9) >> e                               # floor(512 x / 2^e)
        assert 512 <= i < 2048


def test_round_shift_is_round_half_up():
    rng = np.random.default_rng(1)
    a = np.concatenate([rng.integers(-2 ** 40, 2 ** 40, 500), np.arange(-40, 41)]).astype(np.int64)
    for k in (1, 2, 5, 12, 13):
        got = F.round_shift(a, k)
        for x, g in zip(a.tolist(), got.tolist()):
            q = Fraction(x, 2 ** k) + Fraction(1, 2)
            assert g == q.numerator // q.denominator            # floor(x / 2^k + 1/2)


def test_saturation_and_quantisation():
    v, sat = F.saturate(np.array([-9000, -8192, 0, 8191, 8192]), 14)
    assert v.tolist() == [-8192, -8192, 0, 8191, 8191] and sat.tolist() == [True, False, False, False, True]
    q, sat = F.quantize(np.array([0.5 / 256, -0.5 / 256, 1.0, 40.0, np.nan]), 8, 14, np.int64)
    assert q.tolist() == [1, 0, 256, 8191, 0] and sat.tolist() == [False, False, False, True, True]


@pytest.mark.parametrize("kind,B,M,t_max", [("mimo_bpsk", 12, 8, 7), ("mimo_qpsk", 24, 4, 5),
                                            ("jed_bpsk", 12, 7, 6)])
def test_wide_formats_reach_the_fp64_oracle(kind, B, M, t_max):
    """The same integer datapath with wide words converges to Algorithm 1 in FP64: a wrong
    alignment shift, sign, product order, triangle or prox axis would not."""
    Tt, D, tau, _ = inputs(kind, 5, B, M, 6.0, seed=B + M)
    Lo, _ = O.taser(Tt.astype(np.float64), D.astype(np.float64), tau.astype(np.float64), t_max)
    # FP64 oracle on the FP32 product 2 tau T~ the fixed-point inputs are quantised from.
    two_tau = (tau + tau).astype(np.float32)
    That = (two_tau[:, None, None] * Tt).astype(np.float32).astype(np.float64)
    Lo2, _ = O.taser(That, D.astype(np.float64), np.full(len(tau), 0.5), t_max)
    assert np.abs(Lo2 - Lo).max() <= 1e-5 * np.abs(Lo).max()
    fx = F.taser_fixed(Tt, D, tau, t_max, WIDE)
    err = np.abs(fx["L_real"] - Lo2).max() / np.abs(Lo2).max()
    assert err <= 1e-6, err
    np.testing.assert_array_equal(fx["s_hat"], O.decisions(Lo2))
    assert not np.any(fx["flags"] & F.FLAG_SATURATED)


def test_paper_formats_invariants():
    Tt, D, tau, _ = inputs("mimo_bpsk", 40, 16, 16, 8.0, seed=9)
    fx = F.taser_fixed(Tt, D, tau, 10)
    L, d = fx["L"], fx["d"]
    N = L.shape[1]
    assert np.all(np.triu(L, 1) == 0)
    np.testing.assert_array_equal(L[:, -1, -1], d[:, -1])          # the constant L~_NN register
    assert np.all(np.abs(L) < 2 ** 13)
    # column norms restored to D within the LUT's bin (2^-10 relative) and the 2^-8 grid
    norms = np.linalg.norm(fx["L_real"][:, :, : N - 1], axis=1)
    np.testing.assert_allclose(norms, D[:, : N - 1], rtol=3e-3)
    np.testing.assert_array_equal(fx["s_hat"], np.where(L[:, -1, :-1] >= 0, 1, -1))
    assert not np.any(fx["flags"] & F.FLAG_SATURATED)


def test_out_of_range_inputs_are_flagged():
    Tt, D, tau, _ = inputs("mimo_bpsk", 6, 16, 8, 8.0, seed=4)
    D2 = D.copy()
    D2[:, -1] = 300.0                                              # beyond the 5-fraction-bit register
    fx = F.taser_fixed(Tt, D2, tau, 3)
    assert np.all(fx["flags"] & F.FLAG_SATURATED)
    with pytest.raises(ValueError):
        F.taser_fixed(Tt, D, tau, 0)


def test_fixed_point_loss_is_small():
    """Sec. V-A: the 14-bit design costs little against floating point (under 0.2 dB at 1% VER
    for 16x16).  On 4,000 16x16 BPSK instances at 9 dB: the fixed-point VER stays within the
    statistical reach of a 0.2 dB loss of the FP64 VER, and the decisions agree on almost all
    instances."""
    n, t_max = 4000, 10
    w = make_mimo(n, 16, 16, 9.0, "bpsk", seed=77)
    r = O.detect("mimo_bpsk", w["H"], w["y"], 0.5, t_max)
    fx = F.taser_fixed(r["T_tilde"].astype(np.float32), r["D"].astype(np.float32), r["tau"].astype(np.float32),
                       t_max)
    truth = np.asarray(w["bits_re"])
    ver_float = np.mean(np.any(r["s_hat"] != truth, axis=1))
    ver_fixed = np.mean(np.any(fx["s_hat"] != truth, axis=1))
    assert 0.005 < ver_float < 0.2
    assert ver_fixed <= 1.5 * ver_float + 5.0 / n, (ver_fixed, ver_float)
    agree = np.mean(np.all(fx["s_hat"] == r["s_hat"], axis=1))
    assert agree >= 0.97, agree
