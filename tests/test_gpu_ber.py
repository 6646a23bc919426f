"""Equal BER at every SNR point (Sec. V-A simulation setup) on a reduced instance count:
the GPU paths and the FP64 oracle detect identical seeded instances, and each path's bit
error rate must lie inside the oracle's Clopper-Pearson 95% interval at every point.
Decisions must agree wherever the oracle's |L~_N,k| exceeds the path's margin, and L~
must stay within the path's tolerance of FP64 (1e-5 FP32, 3e-2 tensor cores).

QPSK 128x16 (N = 33), t_max = 20, SNR 0..20 dB; SIMO JED BPSK B = 16, K = 16 and 32,
t_max = 20, SNR 0..12 dB.  The full-size counts (65,536 and 131,072 per point) run in
``bench.py --workload ber``.
"""
import numpy as np
import pytest
import torch
from scipy.stats import beta

from oracle import taser_oracle as O
from synth import make_jed, make_mimo

pytestmark = pytest.mark.gpu

ALPHA, T_MAX = 0.5, 20


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_01797_gb300 as taser
    return taser


def clopper_pearson(k, n):
    lo = 0.0 if k == 0 else float(beta.ppf(0.025, k, n - k + 1))
    hi = 1.0 if k == n else float(beta.ppf(0.975, k + 1, n - k))
    return lo, hi


def inputs(kind, B, M, snr, n, seed):
    if kind == "mimo_qpsk":
        w = make_mimo(n, B, M, snr, "qpsk", seed=seed)
        return w["H"], w["y"], np.concatenate([w["bits_re"], w["bits_im"]], axis=1)
    w = make_jed(n, B, M, snr, seed=seed)
    return w["Y"], None, w["s"][:, 1:]


@pytest.mark.parametrize("kind,B,M,snrs,n", [
    ("mimo_qpsk", 128, 16, np.arange(0.0, 21.0, 2.0), 2048),
    ("jed_bpsk", 16, 16, np.arange(0.0, 13.0, 2.0), 1024),
    ("jed_bpsk", 16, 32, np.arange(0.0, 13.0, 2.0), 1024)])
def test_ber_inside_the_oracle_interval_at_every_snr(T, kind, B, M, snrs, n):
    for si, snr in enumerate(snrs):
        X, y, truth = inputs(kind, B, M, float(snr), n, seed=5000 + 100 * M + si)
        r = O.detect(kind, X, y, ALPHA, T_MAX)
        nbits = truth.size
        lo, hi = clopper_pearson(int((r["s_hat"] != truth).sum()), nbits)
        row = r["L"][:, -1, :]
        rown = np.linalg.norm(row, axis=1)
        nrm = np.linalg.norm(r["L"], axis=(1, 2))
        Xd = torch.from_numpy(X).cuda()
        yd = torch.from_numpy(y).cuda() if y is not None else None
        out = T.build_T(kind, Xd, yd, alpha=ALPHA)
        for precision, tol, margin in (("fp32", 1e-5, 1e-3), ("bf16_tc", 3e-2, 5e-2), ("fp16_tc", 3e-2, 5e-2)):
            s, L, _ = T.detect(out["T_tilde"], out["D"], out["tau"], T_MAX, precision)
            s = s.cpu().numpy()
            ber = (s != truth).sum() / nbits
            assert lo <= ber <= hi, (precision, float(snr), ber, lo, hi)
            conf = np.abs(row[:, :-1]) > margin * rown[:, None]
            np.testing.assert_array_equal(s[conf], r["s_hat"][conf])
            err = np.linalg.norm(L.cpu().numpy().astype(np.float64) - r["L"], axis=(1, 2)) / nrm
            assert err.max() <= tol, (precision, float(snr), err.max())
