"""Uneven batches (taser_detect_uneven): problems of different N and t_max in one
stream-ordered, graph-capturable call fed by a size-bucketed work queue.

Each item's result must equal (bitwise) the dense taser_detect on the same inputs, since
the same per-instance code runs in both, and agree with the FP64 oracle within the FP32
(1e-5) or tensor-core (3e-2) tolerances of the detector tests.
"""
import numpy as np
import pytest
import torch

from oracle import taser_oracle as O
from synth import make_mimo

pytestmark = pytest.mark.gpu

NS = (2, 5, 9, 12, 17, 24, 33, 40, 65)
TMAX = (1, 5, 10, 20)


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_01797_gb300 as taser
    return taser


@pytest.fixture(scope="module")
def batch(T):
    """~1,600 items, shuffled over N and t_max, with oracle-built T~, D, tau (fp32)."""
    rng = np.random.default_rng(11)
    per = {}
    for N in NS:
        U = N - 1
        w = make_mimo(180, max(2 * U, 4), U, rng.uniform(0, 15, 180), "bpsk", seed=300 + N)
        r = O.detect("mimo_bpsk", w["H"], w["y"], 0.5, 1)
        per[N] = (r["T_tilde"].astype(np.float32), r["D"].astype(np.float32), r["tau"].astype(np.float32))
    items = [(N, int(rng.choice(TMAX)), k) for N in NS for k in range(180)]
    order = rng.permutation(len(items))
    items = [items[i] for i in order]
    Ns = np.array([it[0] for it in items])
    tm = np.array([it[1] for it in items])
    t_sizes, d_sizes, s_sizes = Ns * Ns, Ns, Ns - 1
    t_off = np.concatenate([[0], np.cumsum(t_sizes)[:-1]])
    d_off = np.concatenate([[0], np.cumsum(d_sizes)[:-1]])
    s_off = np.concatenate([[0], np.cumsum(s_sizes)[:-1]])
    Tp = np.concatenate([per[N][0][k].ravel() for N, _, k in items]).astype(np.float32)
    Dp = np.concatenate([per[N][1][k] for N, _, k in items]).astype(np.float32)
    tau = np.array([per[N][2][k] for N, _, k in items], dtype=np.float32)
    return {"items": items, "N": Ns, "t_max": tm, "t_off": t_off, "d_off": d_off, "s_off": s_off,
            "T_pool": Tp, "D_pool": Dp, "tau": tau, "per": per, "n_s": int(s_sizes.sum()), "n_t": int(t_sizes.sum())}


def run_uneven(T, b, precision, lnn_mode="fixed", items_np=None, tune=None):
    it = items_np if items_np is not None else T.make_items(b["N"], b["t_max"], b["t_off"], b["d_off"], b["s_off"],
                                                            b["t_off"])
    n = len(it)
    items = torch.from_numpy(it.view(np.uint8).copy()).cuda()
    Tp, Dp, tau = (torch.from_numpy(x).cuda() for x in (b["T_pool"], b["D_pool"], b["tau"]))
    s = torch.zeros(b["n_s"], dtype=torch.int8, device="cuda")
    L = torch.zeros(b["n_t"], dtype=torch.float32, device="cuda")
    flags = torch.zeros(n, dtype=torch.int32, device="cuda")
    ws = torch.empty(T.uneven_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    T.detect_uneven(items, Tp, Dp, tau, s, ws, precision=precision, lnn_mode=lnn_mode, L_pool=L, flags=flags,
                    tune=tune)
    torch.cuda.synchronize()
    return s.cpu().numpy(), L.cpu().numpy(), flags.cpu().numpy().astype(np.uint32)


@pytest.mark.parametrize("precision", ["fp32", "bf16_tc"])
def test_uneven_equals_dense_per_group(T, batch, precision):
    s, L, _ = run_uneven(T, batch, precision)
    b = batch
    groups = {}
    for i, (N, tm, k) in enumerate(b["items"]):
        groups.setdefault((N, tm), []).append((i, k))
    for (N, tm), members in groups.items():
        ks = [k for _, k in members]
        Tt, D, tau = b["per"][N]
        sd, Ld, _ = T.detect(*[torch.from_numpy(np.ascontiguousarray(x[ks])).cuda() for x in (Tt, D, tau)], tm,
                             precision)
        sd, Ld = sd.cpu().numpy(), Ld.cpu().numpy()
        for row, (i, _) in enumerate(members):
            so = b["s_off"][i]
            to = b["t_off"][i]
            np.testing.assert_array_equal(s[so:so + N - 1], sd[row])
            np.testing.assert_array_equal(L[to:to + N * N].reshape(N, N), Ld[row])


def test_uneven_matches_oracle(T, batch):
    s, L, _ = run_uneven(T, batch, "fp32")
    b = batch
    for i, (N, tm, k) in enumerate(b["items"][:400]):
        Tt, D, tau = b["per"][N]
        Lo, _ = O.taser(Tt[k:k + 1].astype(np.float64), D[k:k + 1].astype(np.float64),
                        tau[k:k + 1].astype(np.float64), tm)
        Lg = L[b["t_off"][i]:b["t_off"][i] + N * N].reshape(1, N, N).astype(np.float64)
        err = np.linalg.norm(Lg - Lo) / np.linalg.norm(Lo)
        assert err <= 1e-5, (i, N, tm, err)


def test_uneven_literal_mode_and_bad_items(T, batch):
    b = dict(batch)
    it = T.make_items(b["N"], b["t_max"], b["t_off"], b["d_off"], b["s_off"], b["t_off"])
    it["N"][3] = 70          # out of range
    it["t_max"][7] = 0       # out of range
    s, L, flags = run_uneven(T, b, "fp32", lnn_mode="literal", items_np=it)
    assert flags[3] & 16 and flags[7] & 16
    ok = np.ones(len(it), bool)
    ok[[3, 7]] = False
    assert not np.any(flags[ok] & 16)
    so = b["s_off"][3]
    assert np.all(s[so:so + b["N"][3] - 1] == 0)             # skipped item left untouched
    i = 11
    N, tm, k = b["items"][i]
    Tt, D, tau = b["per"][N]
    Lo, _ = O.taser(Tt[k:k + 1].astype(np.float64), D[k:k + 1].astype(np.float64), tau[k:k + 1].astype(np.float64),
                    tm, "literal")
    np.testing.assert_array_equal(s[b["s_off"][i]:b["s_off"][i] + N - 1][None, :] == 1,
                                  O.decisions(Lo, "literal") == 1)


def test_uneven_in_a_cuda_graph(T, batch):
    b = batch
    it = T.make_items(b["N"], b["t_max"], b["t_off"], b["d_off"], b["s_off"], b["t_off"])
    n = len(it)
    items = torch.from_numpy(it.view(np.uint8).copy()).cuda()
    Tp, Dp, tau = (torch.from_numpy(x).cuda() for x in (b["T_pool"], b["D_pool"], b["tau"]))
    s = torch.zeros(b["n_s"], dtype=torch.int8, device="cuda")
    L = torch.zeros(b["n_t"], dtype=torch.float32, device="cuda")
    ws = torch.empty(T.uneven_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        T.detect_uneven(items, Tp, Dp, tau, s, ws, precision="bf16_tc", L_pool=L)   # warm-up before capture
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    ref_s, ref_L = s.clone(), L.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        T.detect_uneven(items, Tp, Dp, tau, s, ws, precision="bf16_tc", L_pool=L)
    for _ in range(2):
        s.zero_()
        L.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(s, ref_s) and torch.equal(L, ref_L)


def test_autotuned_launch_gives_the_same_results(T, batch):
    from paper_1609_01797_gb300.autotune import tune_uneven
    b = batch
    it = T.make_items(b["N"], b["t_max"], b["t_off"], b["d_off"], b["s_off"])
    n = len(it)
    items = torch.from_numpy(it.view(np.uint8).copy()).cuda()
    Tp, Dp, tau = (torch.from_numpy(x).cuda() for x in (b["T_pool"], b["D_pool"], b["tau"]))
    s = torch.zeros(b["n_s"], dtype=torch.int8, device="cuda")
    ws = torch.empty(T.uneven_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    tune, report = tune_uneven(items, Tp, Dp, tau, s, ws, precision="bf16_tc", blocks_candidates=(1, 0),
                               pop_candidates=(1, 2), repeats=2)
    assert report["tuned_ms"] <= report["default_ms"] * 1.0001
    s_def, _, _ = run_uneven(T, b, "bf16_tc")
    s_tuned, _, _ = run_uneven(T, b, "bf16_tc", tune=tune)
    np.testing.assert_array_equal(s_def, s_tuned)
