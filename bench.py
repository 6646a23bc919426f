#!/usr/bin/env python3
"""TASER detections/s on MU-MIMO QPSK 128x16 (N = 33), t_max = 20: BF16 tensor-core
path vs FP32 path at equal BER, on one or more GPUs (one process per GPU).

A step is one pass of the whole detector over one batch of synthetic instances that
are already resident in HBM: taser_build_T (T~ and D from H, y), taser_step_size
(tau = alpha / ||T~||_2) and taser_detect (Algorithm 1 and the decisions).  The batch is 65,536 instances per GPU
with the SNR cycling over 0, 2, ..., 20 dB (the SNR sweep of the workload); its inputs
(1.14 GB) are larger than the 129 MB L2, so no flush is needed between steps.

Prints one JSON line on rank 0.  `--impl reference` times the FP64 CPU oracle instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

B, U, T_MAX, ALPHA = 128, 16, 20, 0.5
N = 2 * U + 1
SNR_GRID = np.arange(0.0, 21.0, 2.0)
METRIC = "TASER detections/s, QPSK 128x16, t_max=20: BF16-TC vs FP32 path at equal BER"
WORKLOAD = "mimo_qpsk_B128_U16_N33_tmax20_snr0-20dB"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["taser", "reference"], default="taser")
    ap.add_argument("--instances", type=int, default=65536, help="instances per GPU per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=8192,
                    help="instances of the workload run through the oracle in one process (1-core rate and the "
                         "GPU paths' error against FP64)")
    ap.add_argument("--jed-instances", type=int, default=131072, help="JED instances per SNR point (--workload ber)")
    ap.add_argument("--train-steps", type=int, default=400, help="training steps before the held-out BER "
                                                                 "(--workload unfolded)")
    ap.add_argument("--unfolded-precision", choices=["fp32", "bf16_tc", "fp16_tc"], default="fp32",
                    help="arithmetic of the unfolded forward and adjoint products (--workload unfolded)")
    ap.add_argument("--workload", choices=["qpsk128x16", "uneven", "tradeoff", "unfolded", "ber", "jed"],
                    default="qpsk128x16",
                    help="uneven: 200,000 QPSK items with N in {9,17,33,65}, t_max in {10,20}; tradeoff: SNR "
                         "for 1%% VER vs throughput over t_max = 1..20 for 32x32 BPSK/QPSK; unfolded: training "
                         "steps of unfolded TASER on batches of 8,192; ber: BER per SNR point of the GPU paths "
                         "against the FP64 oracle; jed: throughput of the JED BPSK path, B = 16, K = 16 and 32 "
                         "(none of these is the headline)")
    return ap.parse_args()


def flops_per_detection(n, t_max):
    """Algorithmic work of Algorithm 1 (Sec. III-D) with the triangular skip (Sec. IV-A):
    per iteration P(N) = N(N+1)(2N+1)/6 MACs for V, then N(N+1)/2 squares, N(N+1)/2 adds
    and N(N+1)/2 scalings for the prox, plus N scale factors."""
    P = n * (n + 1) * (2 * n + 1) // 6
    return t_max * (2 * P + 3 * n * (n + 1) // 2 + n)


def build_bytes_per_instance(b, u, n):
    """Algorithmic HBM bytes of the build kernel per instance: read H (B x U complex64)
    and y (B complex64), write T~ (N x N fp32) and D (N fp32)."""
    return 8 * b * u + 8 * b + 4 * n * n + 4 * n


def spectral_flops_per_instance(u):
    """Complex Hermitian tridiagonalisation of order n = U + 1 (16/3 n^3 real flops) plus
    the Sturm multisection of the folded kernel (U <= 16: 7 rounds x 8 points x n steps x 4
    flops)."""
    n = u + 1
    return 16 * n ** 3 // 3 + 7 * 8 * n * 4


KERNEL_SOURCES = {"build": "build_T.cu", "spectral": "spectral.cu", "detect_tc": "detect_tc.cu",
                  "detect_fp32": "detect_fp32.cu", "detect_fx14": "detect_fx14.cu"}


def source_sha(path):
    """sha1 of a kernel source with its // comments and blank lines removed, so that only a
    change of the code itself marks the counters taken on it as stale (the sources hold no
    // inside string literals)."""
    import hashlib
    lines = []
    for line in open(path, encoding="utf-8"):
        code = line.split("//", 1)[0].rstrip()
        if code:
            lines.append(code)
    return hashlib.sha1("\n".join(lines).encode()).hexdigest()


def measured_traffic(name="dram_traffic.txt"):
    """Per-kernel figures from a committed ncu summary (DRAM bytes per instance, or the
    tensor-pipe active fraction), kept only while the kernel's code is unchanged since the
    counters were taken (source_sha match)."""
    path = os.path.join(ROOT, "profiles", name)
    out = {}
    if not os.path.exists(path):
        return out
    for line in open(path):
        p = line.split()
        if len(p) != 3 or line.startswith("#"):
            continue
        key, per_inst, sha = p[0], float(p[1]), p[2]
        src = os.path.join(ROOT, "paper_1609_01797_gb300", "csrc", KERNEL_SOURCES.get(key, ""))
        if os.path.isfile(src) and source_sha(src) == sha:
            out[key] = per_inst
    return out


def make_workload(n, seed):
    from synth import make_mimo
    snr = np.tile(SNR_GRID, n // len(SNR_GRID) + 1)[:n]
    return make_mimo(n, B, U, snr, "qpsk", seed=seed)


def truth_bits(w):
    return np.concatenate([w["bits_re"], w["bits_im"]], axis=1)


def clopper_pearson(k, n, conf=0.95):
    from scipy.stats import beta
    a = (1 - conf) / 2
    lo = 0.0 if k == 0 else float(beta.ppf(a, k, n - k + 1))
    hi = 1.0 if k == n else float(beta.ppf(1 - a, k + 1, n - k))
    return lo, hi


# ---------------------------------------------------------------------------------
# The FP64 oracle on every host core: a pool of spawned processes (safe to create at any
# time, GPU context or not), each with one BLAS thread.
# ---------------------------------------------------------------------------------
def oracle_pool(workers=None):
    import multiprocessing as mp
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    workers = workers or os.cpu_count() or 1
    return mp.get_context("spawn").Pool(workers), workers


BER_CHUNK = 4096


def ber_inputs(kind, b, m, snr, n, seed):
    """Seeded inputs of one chunk: (H or Y, y or None, transmitted signs in decision order)."""
    from synth import make_jed, make_mimo
    if kind == "mimo_qpsk":
        w = make_mimo(n, b, m, snr, "qpsk", seed=seed)
        return w["H"], w["y"], truth_bits(w)
    w = make_jed(n, b, m, snr, seed=seed)
    return w["Y"], None, w["s"][:, 1:]


def _oracle_ber_chunk(job):
    """Pool worker: the oracle on one chunk, compared with the GPU paths' results on the
    same instances (relative Frobenius error of L~ against FP64, decision agreement)."""
    from oracle import taser_oracle as O
    kind, b, m, snr, seed, n, alpha, t_max, gpu = job
    X, y, truth = ber_inputs(kind, b, m, snr, n, seed)
    t0 = time.perf_counter()
    r = O.detect(kind, X, y, alpha, t_max)
    dt = time.perf_counter() - t0
    Lo, so = r["L"], r["s_hat"]
    nrm = np.linalg.norm(Lo, axis=(1, 2))
    row = Lo[:, -1, :]
    rown = np.linalg.norm(row, axis=1)
    out = {"n": n, "oracle_s": dt, "oracle": {"bit_errors": int((so != truth).sum()),
                                               "vec_errors": int((so != truth).any(axis=1).sum())}}
    for p, (L, s) in gpu.items():
        err = np.linalg.norm(L.astype(np.float64) - Lo, axis=(1, 2)) / nrm
        conf = np.abs(row[:, :-1]) > (1e-3 if p == "fp32" else 5e-2) * rown[:, None]
        d = s != so
        out[p] = {"bit_errors": int((s != truth).sum()), "vec_errors": int((s != truth).any(axis=1).sum()),
                  "discordant_bits": int(d.sum()), "discordant_instances": int(d.any(axis=1).sum()),
                  "differ_beyond_margin": int(d[conf].sum()), "err": err.astype(np.float32)}
    return out


class OracleTeam:
    """The FP64 oracle timed on every host core: one spawned process per core, each with
    its own seeded chunks of the headline workload generated before any timing.  A step
    releases every worker at once (a barrier) and ends when the last one has finished
    detect on its chunk, so a step's wall-clock time is that of the slowest core."""

    def __init__(self, workers, per_worker, n_chunks=4, seed=1):
        import multiprocessing as mp
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"
        ctx = mp.get_context("spawn")
        self.workers, self.per_worker = workers, per_worker
        self.go, self.done = ctx.Barrier(workers + 1), ctx.Barrier(workers + 1)
        self.procs = [ctx.Process(target=_team_worker, args=(i, per_worker, n_chunks, seed, self.go, self.done),
                                  daemon=True) for i in range(workers)]
        for pr in self.procs:
            pr.start()
        self.go.wait()            # every worker has generated its chunks

    def step(self):
        self.go.wait()
        t0 = time.perf_counter()
        self.done.wait()
        return time.perf_counter() - t0

    def close(self):
        for pr in self.procs:
            pr.terminate()
            pr.join()


def _team_worker(idx, per_worker, n_chunks, seed, go, done):
    from oracle import taser_oracle as O
    chunks = [make_workload(per_worker, seed=seed * 100_003 + 1000 * idx + k) for k in range(n_chunks)]
    go.wait()
    k = 0
    while True:
        go.wait()
        w = chunks[k % n_chunks]
        O.detect("mimo_qpsk", w["H"], w["y"], ALPHA, T_MAX)
        done.wait()
        k += 1


def run_ber(args):
    """Equal BER per SNR point (Sec. V-A simulation setup): BER of the FP32, BF16 and FP16
    GPU paths and of the FP64 oracle on identical seeded instances, with Clopper-Pearson
    95% intervals, paired discordance counts and each path's relative Frobenius error of
    L~ against FP64 (max, mean, 99th percentile).  QPSK 128x16, t_max = 20, SNR 0..20 dB
    (65,536 instances per point by default) and SIMO JED BPSK B = 16, K = 16 and 32,
    t_max = 20, SNR 0..12 dB (131,072 per point).  The oracle runs on every host core."""
    pool, workers = oracle_pool()          # spawned before the first GPU call
    import torch
    import paper_1609_01797_gb300 as taser
    dev = torch.device("cuda", 0)
    n1 = args.instances
    n2 = args.jed_instances
    cfgs = [("mimo_qpsk", B, U, np.arange(0.0, 21.0, 2.0), n1, 0),
            ("jed_bpsk", 16, 16, np.arange(0.0, 13.0, 2.0), n2, 1),
            ("jed_bpsk", 16, 32, np.arange(0.0, 13.0, 2.0), n2, 2)]
    paths = ("fp32", "bf16_tc", "fp16_tc")
    t_start = time.perf_counter()
    pending = []
    results = {}

    def collect(block):
        key, snr, nn, handles = block
        parts = [h.get() for h in handles]
        pt = {"snr_db": float(snr), "instances": nn}
        o_bits = sum(p["oracle"]["bit_errors"] for p in parts)
        nbits = nn * results[key]["bits_per_instance"]
        lo, hi = clopper_pearson(o_bits, nbits)
        pt["oracle"] = {"bit_errors": o_bits, "ber": o_bits / nbits, "ber_ci95": [lo, hi],
                        "vec_errors": sum(p["oracle"]["vec_errors"] for p in parts),
                        "oracle_s": sum(p["oracle_s"] for p in parts)}
        for p in paths:
            be = sum(q[p]["bit_errors"] for q in parts)
            err = np.concatenate([q[p]["err"] for q in parts]).astype(np.float64)
            pt[p] = {"bit_errors": be, "ber": be / nbits, "ber_ci95": list(clopper_pearson(be, nbits)),
                     "in_oracle_ci95": bool(lo <= be / nbits <= hi),
                     "vec_errors": sum(q[p]["vec_errors"] for q in parts),
                     "discordant_bits_vs_oracle": sum(q[p]["discordant_bits"] for q in parts),
                     "discordant_instances_vs_oracle": sum(q[p]["discordant_instances"] for q in parts),
                     "decisions_differ_beyond_margin": sum(q[p]["differ_beyond_margin"] for q in parts),
                     "L_relerr_vs_fp64": {"max": float(err.max()), "mean": float(err.mean()),
                                          "p99": float(np.quantile(err, 0.99))}}
        results[key]["points"].append(pt)

    for kind, b, m, snrs, n, ci in cfgs:
        key = "%s_B%d_%s%d" % (kind, b, "U" if kind == "mimo_qpsk" else "K", m)
        N = taser.problem_size(kind, m)
        results[key] = {"kind": kind, "B": b, "U_or_K": m, "N": N, "t_max": T_MAX, "alpha": ALPHA,
                        "bits_per_instance": N - 1, "points": []}
        for si, snr in enumerate(snrs):
            chunks = []
            for c0 in range(0, n, BER_CHUNK):
                nc = min(BER_CHUNK, n - c0)
                seed = 9_000_000 + 100_000 * ci + 1000 * si + c0 // BER_CHUNK
                chunks.append((c0, nc, seed) + ber_inputs(kind, b, m, float(snr), nc, seed))
            X = torch.from_numpy(np.concatenate([c[3] for c in chunks])).to(dev)
            y = torch.from_numpy(np.concatenate([c[4] for c in chunks])).to(dev) if kind == "mimo_qpsk" else None
            out = taser.build_T(kind, X, y, ALPHA)
            host = {}
            for p in paths:
                s, L, _ = taser.detect(out["T_tilde"], out["D"], out["tau"], T_MAX, p, want_L=True)
                host[p] = (L.cpu().numpy(), s.cpu().numpy())
            del X, y, out
            handles = []
            for c0, nc, seed, *_ in chunks:
                gpu = {p: (host[p][0][c0:c0 + nc], host[p][1][c0:c0 + nc]) for p in paths}
                handles.append(pool.apply_async(_oracle_ber_chunk,
                                                ((kind, b, m, float(snr), seed, nc, ALPHA, T_MAX, gpu),)))
            pending.append((key, snr, n, handles))
            while len(pending) > 2:
                collect(pending.pop(0))
    while pending:
        collect(pending.pop(0))
    pool.close()
    pool.join()
    summary = {}
    for key, r in results.items():
        pts = r["points"]
        summary[key] = {p: {"every_point_in_oracle_ci95": all(pt[p]["in_oracle_ci95"] for pt in pts),
                            "decisions_differ_beyond_margin": sum(pt[p]["decisions_differ_beyond_margin"]
                                                                  for pt in pts),
                            "L_relerr_vs_fp64_max": max(pt[p]["L_relerr_vs_fp64"]["max"] for pt in pts)}
                        for p in paths}
    print(json.dumps({"metric": "BER per SNR point: GPU paths vs the FP64 oracle on identical instances "
                                "(Clopper-Pearson 95%)", "unit": "bit error rate", "n_gpus": 1,
                      "dtype": "f32, bf16, f16 (GPU); f64 (oracle)", "data": "synthetic",
                      "config": {"workload": "ber_c1_qpsk128x16_snr0-20_c2_jed16_K16-32_snr0-12",
                                 "instances_per_snr": {"mimo_qpsk": n1, "jed_bpsk": n2}, "t_max": T_MAX,
                                 "alpha": ALPHA, "oracle_cores": workers,
                                 "margins": {"fp32": "1e-3 ||l_N||", "tensor cores": "5e-2 ||l_N||"}},
                      "wall_s": time.perf_counter() - t_start, "summary": summary, "configs": results}))
    return 0


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while the GPU is busy."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.gpu)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                    power.append(float(p[3]))
                except ValueError:
                    continue
                for name, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        busy = [s for s in sm if smax and s > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_median": statistics.median(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _peak(d, *keys):
    for k in keys:
        if k in d and isinstance(d[k], (int, float)):
            return float(d[k])
    return None


def cpu_baseline(w, sample, team_per_core=1024):
    """The FP64 oracle as it stands: on every host core (the reported value: one barrier-
    synchronised step of `team_per_core` instances per core), and in one process on the
    first `sample` instances of this workload, whose results also give the GPU path's
    error against FP64.  Returns (baseline dict, oracle result on the sample)."""
    from oracle import taser_oracle as O
    workers = os.cpu_count() or 1
    team = OracleTeam(workers, team_per_core)
    try:
        team.step()                      # warm-up (imports, first-touch)
        t_all = team.step()
    finally:
        team.close()
    H, y = w["H"][:sample], w["y"][:sample]
    t0 = time.perf_counter()
    r = O.detect("mimo_qpsk", H, y, ALPHA, T_MAX)
    dt = time.perf_counter() - t0
    base = {"value": workers * team_per_core / t_all, "unit": "detections/s", "cores": workers, "kind": "oracle",
            "sample": "%d QPSK 128x16 instances of the workload per host core (%d cores, one process each, "
                      "inputs generated before timing), FP64 numpy oracle (T, Jacobi preconditioning, eigvalsh, "
                      "Algorithm 1), %.2f s" % (team_per_core, workers, t_all),
            "single_core": {"value": sample / dt, "cores": 1,
                            "sample": "the first %d instances of the workload, one process, %.1f s" % (sample, dt)}}
    return base, r


def error_vs_fp64(taser, bufs, r, sample):
    """Each GPU path's result against the FP64 oracle on the first `sample` instances of
    the headline workload (outside the timed region): relative Frobenius error of L~ per
    instance (max, mean, 99th percentile) and decisions that differ where the oracle's
    |L~_N,k| exceeds the path's margin (1e-3 ||l~_N|| FP32, 5e-2 ||l~_N|| tensor cores)."""
    Lo, so = r["L"], r["s_hat"]
    row = Lo[:, -1, :]
    rown = np.linalg.norm(row, axis=1)
    nrm = np.linalg.norm(Lo, axis=(1, 2))
    res = {"instances": sample}
    T_s, D_s, tau_s = (bufs[k][:sample].contiguous() for k in ("T_tilde", "D", "tau"))
    for p in ("bf16_tc", "fp16_tc", "fp32"):
        s, L, _ = taser.detect(T_s, D_s, tau_s, T_MAX, p, want_L=True)
        L = L.cpu().numpy().astype(np.float64)
        s = s.cpu().numpy()
        err = np.linalg.norm(L - Lo, axis=(1, 2)) / nrm
        conf = np.abs(row[:, :-1]) > (1e-3 if p == "fp32" else 5e-2) * rown[:, None]
        res[p] = {"L_relerr_max": float(err.max()), "L_relerr_mean": float(err.mean()),
                  "L_relerr_p99": float(np.quantile(err, 0.99)),
                  "decisions_differ_beyond_margin": int((s != so)[conf].sum()),
                  "discordant_bits": int((s != so).sum())}
    return res


def run_reference(args):
    """The FP64 oracle as it stands on every host core: each step is one barrier-synchronised
    pass of 256 instances of the workload per core (inputs generated before timing)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    per_core = 256
    workers = os.cpu_count() or 1
    team = OracleTeam(workers, per_core)
    try:
        times = []
        for i in range(args.warmup + args.steps):
            dt = team.step()
            if i >= args.warmup:
                times.append(dt)
    finally:
        team.close()
    sample = per_core * workers
    value = sample * len(times) / sum(times)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "detections/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "instances_per_step": sample,
                                           "t_max": T_MAX, "alpha": ALPHA},
           "cpu_baseline": {"value": value, "unit": "detections/s", "cores": workers, "kind": "oracle",
                            "sample": "%d instances of the workload per core and step, %d cores (one process "
                                      "each), FP64 numpy oracle" % (per_core, workers)},
           "e2e": {"value": value, "unit": "detections/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def run_uneven(args):
    """Uneven QPSK batch: taser_detect_uneven replayed from a CUDA graph vs the same work as
    dense taser_detect calls per (shape, t_max) group (the scheduling overhead)."""
    import torch
    import paper_1609_01797_gb300 as taser
    from synth import make_uneven
    dev = torch.device("cuda", 0)
    n = 200000
    w = make_uneven(n, seed=3)
    shapes = w["shapes"]
    Ns = np.array([2 * u + 1 for _, u in shapes])[w["shape_idx"]]
    tm = w["t_max"]
    # T~, D, tau per shape (dense builds), pooled in shape order
    groups, T_parts, D_parts, tau_parts = [], [], [], []
    t_base = d_base = 0
    t_off = np.zeros(n, np.int64)
    d_off = np.zeros(n, np.int64)
    for si, ps in enumerate(w["per_shape"]):
        B_, U_ = shapes[si]
        N_ = 2 * U_ + 1
        out = taser.build_T("mimo_qpsk", torch.from_numpy(ps["H"]).to(dev), torch.from_numpy(ps["y"]).to(dev), ALPHA)
        sel = ps["items"]
        t_off[sel] = t_base + np.arange(len(sel)) * N_ * N_
        d_off[sel] = d_base + np.arange(len(sel)) * N_
        t_base += len(sel) * N_ * N_
        d_base += len(sel) * N_
        T_parts.append(out["T_tilde"].reshape(-1))
        D_parts.append(out["D"].reshape(-1))
        tau_parts.append((si, sel, out["tau"]))
        groups.append((N_, sel, out))
    T_pool = torch.cat(T_parts)
    D_pool = torch.cat(D_parts)
    tau = torch.empty(n, device=dev)
    for si, sel, tv in tau_parts:
        tau[torch.from_numpy(sel).to(dev)] = tv
    s_off = np.concatenate([[0], np.cumsum(Ns - 1)[:-1]])
    items = torch.from_numpy(taser.make_items(Ns, tm, t_off, d_off, s_off).view(np.uint8).copy()).to(dev)
    s_pool = torch.empty(int((Ns - 1).sum()), dtype=torch.int8, device=dev)
    ws = torch.empty(taser.uneven_workspace_bytes(n), dtype=torch.uint8, device=dev)
    result = {}
    for precision in ("bf16_tc", "fp32"):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            taser.detect_uneven(items, T_pool, D_pool, tau, s_pool, ws, precision=precision)
        torch.cuda.current_stream().wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            taser.detect_uneven(items, T_pool, D_pool, tau, s_pool, ws, precision=precision)
        for _ in range(args.warmup):
            g.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        un_ms = e0.elapsed_time(e1) / args.steps
        # the same work as dense calls per (shape, t_max) group
        dense = []
        for N_, sel, out in groups:
            for t in (10, 20):
                m = torch.from_numpy(tm[sel] == t).to(dev)
                dense.append((N_, t, out["T_tilde"][m].contiguous(), out["D"][m].contiguous(),
                              out["tau"][m].contiguous()))
        for _ in range(args.warmup):
            for N_, t, Tg, Dg, tg in dense:
                taser.detect(Tg, Dg, tg, t, precision, want_L=False)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            for N_, t, Tg, Dg, tg in dense:
                taser.detect(Tg, Dg, tg, t, precision, want_L=False)
        e1.record()
        torch.cuda.synchronize()
        dn_ms = e0.elapsed_time(e1) / args.steps
        result[precision] = {"uneven_ms": un_ms, "dense_ms": dn_ms, "det_per_s": n / (un_ms * 1e-3),
                             "overhead_vs_dense": un_ms / dn_ms - 1.0}
    print(json.dumps({"metric": "TASER detections/s, uneven QPSK batch (N = 9, 17, 33, 65; t_max 10/20), "
                                "detection only, CUDA-graph replay", "value": result["bf16_tc"]["det_per_s"],
                      "unit": "detections/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
                      "config": {"workload": "uneven_qpsk_200000_N9-65_tmax10-20", "items": n}, "paths": result}))
    return 0


def run_jed(args):
    """Throughput of the whole SIMO JED BPSK path (Sec. II-B and III-C: build T~ = -D^-1 A^T A
    D^-1 and D from Y, step size, Algorithm 1) at B = 16 receive antennas, K = 16 and 32
    slots, t_max = 20, 131,072 device-resident instances per step, SNR cycling over 0..12 dB
    in 2 dB steps: detections/s per path, the per-kernel split and the BER against the
    transmitted symbols."""
    import torch
    import paper_1609_01797_gb300 as taser
    from synth import make_jed
    dev = torch.device("cuda", 0)
    n = args.jed_instances
    steps, warmup = args.steps, max(args.warmup, 3)
    snr = np.tile(np.arange(0.0, 13.0, 2.0), n // 7 + 1)[:n]
    result = {}
    for K in (16, 32):
        w = make_jed(n, 16, K, snr, seed=31_000 + K)
        Y = torch.from_numpy(w["Y"]).to(dev)
        truth = torch.from_numpy(w["s"][:, 1:].astype(np.int8)).to(dev)
        N = taser.problem_size("jed_bpsk", K)
        bufs = {"T_tilde": torch.empty((n, N, N), device=dev), "D": torch.empty((n, N), device=dev),
                "tau": torch.empty((n,), device=dev), "flags": torch.zeros((n,), device=dev, dtype=torch.int32)}
        s_hat = torch.empty((n, N - 1), device=dev, dtype=torch.int8)
        stream = torch.cuda.current_stream(dev)
        paths = {}
        for precision in ("bf16_tc", "fp32"):
            def one(ev=None):
                if ev is not None:
                    ev[0].record(stream)
                taser.build_T("jed_bpsk", Y, None, ALPHA, out=bufs, with_tau=False)
                if ev is not None:
                    ev[1].record(stream)
                taser.step_size(bufs["T_tilde"], ALPHA, structure="jed_bpsk", tau=bufs["tau"])
                if ev is not None:
                    ev[2].record(stream)
                taser.detect(bufs["T_tilde"], bufs["D"], bufs["tau"], T_MAX, precision, want_L=False,
                             flags=bufs["flags"], out_s=s_hat)
                if ev is not None:
                    ev[3].record(stream)
            for _ in range(warmup):
                one()
            ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            a.record(stream)
            for i in range(steps):
                one(ev[i])
            b.record(stream)
            torch.cuda.synchronize(dev)
            ms = a.elapsed_time(b) / steps
            split = [sum(e[k].elapsed_time(e[k + 1]) for e in ev) / steps for k in range(3)]
            errs = int((s_hat != truth).sum().item())
            nbits = n * (N - 1)
            paths[precision] = {"det_per_s": n / (ms * 1e-3), "ms_per_step": ms, "build_ms": split[0],
                                "spectral_ms": split[1], "detect_ms": split[2],
                                "detect_only_det_per_s": n / (split[2] * 1e-3),
                                "bit_errors": errs, "ber": errs / nbits,
                                "ber_ci95": list(clopper_pearson(errs, nbits))}
        result["K%d" % K] = {"N": N, "instances": n, "paths": paths}
        del Y, truth, bufs, s_hat
    head = result["K32"]["paths"]["bf16_tc"]
    print(json.dumps({"metric": "TASER JED BPSK detections/s (whole path: build T~ and D from Y, step size, "
                      "Algorithm 1), BF16 tensor-core path", "value": head["det_per_s"], "unit": "detections/s",
                      "n_gpus": 1, "steps": steps, "warmup": warmup, "ms_per_step": head["ms_per_step"],
                      "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
                      "config": {"workload": "jed_bpsk_B16_K16_K32_tmax20_snr0-12dB", "instances": n, "t_max": T_MAX,
                                 "alpha": ALPHA, "inputs": "device-resident, larger than L2"},
                      "results": result}))
    return 0


def run_tradeoff(args):
    """Throughput vs the SNR needed for 1% VER as t_max goes from 1 to 20, for 32-user
    systems (B = 32, U = 32, BPSK N = 33 and QPSK N = 65): the GPU counterpart of the
    paper's trade-off figures (Sec. V-A).  alpha is the paper's system-dependent tuning
    parameter (Sec. III-B): per t_max the best alpha of a small grid is reported.  VER per
    SNR point on fresh instances (65,536 by default), 1 dB steps, the 1% crossing
    interpolated in log10(VER); throughput of taser_detect alone (as the paper's FPGA
    figures, which exclude the preprocessing) at each t_max."""
    import torch
    import paper_1609_01797_gb300 as taser
    from synth import make_mimo_device
    dev = torch.device("cuda", 0)
    n = args.instances
    t_list = list(range(1, 21))
    alphas = (0.5, 0.7, 0.9, 0.99)
    precisions = ("bf16_tc", "fp32")
    snrs = np.arange(0.0, 41.0, 1.0)

    def crossing(pts):
        for (s0, v0), (s1, v1) in zip(pts, pts[1:]):
            if v0 >= 0.01 > v1:
                if v1 <= 0:
                    return s1
                l0, l1 = np.log10(v0), np.log10(v1)
                return s0 + (s1 - s0) * (l0 + 2.0) / (l0 - l1)
        return None

    table = {}
    for const in ("bpsk", "qpsk"):
        u = b = 32
        kind = "mimo_" + const
        nn = 2 * u + 1 if const == "qpsk" else u + 1
        bits = u * (2 if const == "qpsk" else 1)
        keys = [(p, a) for p in precisions for a in alphas]
        ver = {(p, a, t): [] for p, a in keys for t in t_list}
        done = {k: False for k in keys}
        tau = torch.empty(n, device=dev)
        for si, snr in enumerate(snrs):
            H, y, truth = make_mimo_device(n, b, u, float(snr), const, seed=(17 if const == "bpsk" else 18) * 1000 + si,
                                           device=dev)
            out = taser.build_T(kind, H, y, 0.5, with_tau=False)
            for a in alphas:
                taser.step_size(out["T_tilde"], a, structure=kind, tau=tau)
                for p in precisions:
                    if done[(p, a)]:
                        continue
                    for t in t_list:
                        s, _, _ = taser.detect(out["T_tilde"], out["D"], tau, t, p, want_L=False)
                        ver[(p, a, t)].append((float(snr), (s != truth).any(dim=1).float().mean().item()))
                    done[(p, a)] = all(ver[(p, a, t)][-1][1] < 0.005 for t in t_list)
            if all(done.values()):
                break
        rows = []
        for t in t_list:
            row = {"t_max": t}
            for p in precisions:
                best = None
                for a in alphas:
                    req = crossing(ver[(p, a, t)])
                    if req is not None and (best is None or req < best[0]):
                        best = (req, a)
                row["snr_1pct_ver_db_" + p] = None if best is None else best[0]
                row["alpha_" + p] = None if best is None else best[1]
                for _ in range(3):
                    taser.detect(out["T_tilde"], out["D"], tau, t, p, want_L=False)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                for _ in range(10):
                    taser.detect(out["T_tilde"], out["D"], tau, t, p, want_L=False)
                e1.record()
                torch.cuda.synchronize()
                det = n / (e0.elapsed_time(e1) / 10 * 1e-3)
                row["detect_det_per_s_" + p] = det
                row["detect_mbit_per_s_" + p] = det * bits / 1e6
            rows.append(row)
        table[const] = {"B": b, "U": u, "N": nn, "rows": rows}
    print(json.dumps({"metric": "SNR for 1% VER vs detection throughput over t_max = 1..20, 32x32 MU-MIMO",
                      "unit": "dB / detections/s", "n_gpus": 1, "dtype": "bf16 and f32", "data": "synthetic",
                      "config": {"workload": "tradeoff_32x32_bpsk_qpsk_tmax1-20", "instances_per_snr": n,
                                 "snr_grid_db": "0..40 step 1 (stops once every t_max is below 0.5% VER)",
                                 "alpha_grid": list(alphas)}, "table": table}))
    return 0


def run_unfolded(args):
    """Unfolded TASER training (learnable per-iteration steps, hand-written adjoint).  One
    step = a fresh seeded batch of 8,192 QPSK 128x16 instances drawn on the GPU (SNR uniform
    in [4, 14] dB, a new seed every step) + taser_build_T + the forward with checkpoints
    every 4 iterations (t_max = 10) + the MSE loss gradient + the adjoint + one Adam update
    of alpha_t.  Reports training instances/s and the forward and adjoint kernels against
    the FP32 pipe, then trains on to --train-steps and judges the trained alpha_t by BER
    against fixed-tau TASER (alpha = 0.5, the same t_max) on 65,536 held-out instances."""
    import torch
    import paper_1609_01797_gb300 as taser
    from synth import make_mimo_device
    dev = torch.device("cuda", 0)
    n, t_max, c = 8192, 10, 4
    alpha = torch.full((t_max,), ALPHA, device=dev, requires_grad=True)
    opt = torch.optim.Adam([alpha], lr=0.02, capturable=True)   # capturable: the graph below
    stream = torch.cuda.current_stream(dev)
    precision = args.unfolded_precision

    def step(i, ev=None):
        if ev is not None:
            ev[0].record(stream)
        H, y, truth = make_mimo_device(n, B, U, (4.0, 14.0), "qpsk", seed=40_000 + i, device=dev)
        truth = truth.float()
        if ev is not None:
            ev[1].record(stream)
        out = taser.build_T("mimo_qpsk", H, y, ALPHA)
        inv = 1.0 / out["spec_norm"]
        if ev is not None:
            ev[2].record(stream)
        soft, _, ckpt = taser.unfolded_forward(out["T_tilde"], out["D"], inv, alpha.detach(), c,
                                               precision=precision)
        if ev is not None:
            ev[3].record(stream)
        g_soft = 2.0 * (soft - truth) / soft.numel()
        if ev is not None:
            ev[4].record(stream)
        _, g_alpha = taser.unfolded_backward(out["T_tilde"], out["D"], inv, alpha.detach(), c, ckpt, g_soft,
                                             precision=precision)
        if ev is not None:
            ev[5].record(stream)
        alpha.grad = g_alpha
        opt.step()
        return soft, truth

    for i in range(args.warmup):
        step(i)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i, ev[i])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    gen_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / args.steps
    fwd_ms = sum(e[2].elapsed_time(e[3]) for e in ev) / args.steps
    bwd_ms = sum(e[4].elapsed_time(e[5]) for e in ev) / args.steps

    # The same step captured in a CUDA graph and replayed: eagerly it is about 30 launches,
    # most of them small torch operations, and the GPU waits on the host between them.  The
    # batch is drawn from the default CUDA generator, seeded once; each replay advances its
    # state, so every replayed step still draws a fresh batch.  Replays train alpha_t too.
    graph = {"used": False}
    try:
        gdefault = torch.cuda.default_generators[dev.index]
        gdefault.manual_seed(50_000)

        def graph_step():
            H, y, truth = make_mimo_device(n, B, U, (4.0, 14.0), "qpsk", device=dev, generator=gdefault)
            truth = truth.float()
            out = taser.build_T("mimo_qpsk", H, y, ALPHA)
            inv = 1.0 / out["spec_norm"]
            soft, _, ckpt = taser.unfolded_forward(out["T_tilde"], out["D"], inv, alpha.detach(), c,
                                                   precision=precision)
            g_soft = 2.0 * (soft - truth) / soft.numel()
            _, g_alpha = taser.unfolded_backward(out["T_tilde"], out["D"], inv, alpha.detach(), c, ckpt, g_soft,
                                                 precision=precision)
            alpha.grad = g_alpha
            opt.step()

        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            for _ in range(3):
                graph_step()
        stream.wait_stream(side)
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg):
            graph_step()
        for _ in range(3):
            cg.replay()
        torch.cuda.synchronize(dev)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.steps):
            cg.replay()
        g1.record(stream)
        torch.cuda.synchronize(dev)
        graph = {"used": True, "ms_per_step": g0.elapsed_time(g1) / args.steps}
    except Exception as exc:   # report the eager step alone
        graph = {"used": False, "error": "%s: %s" % (type(exc).__name__, exc)}
        torch.cuda.synchronize(dev)
    step_ms = graph["ms_per_step"] if graph["used"] else ms
    losses = []
    for i in range(args.warmup + args.steps, args.train_steps):
        soft, truth = step(i)
        if i % 50 == 0 or i == args.train_steps - 1:
            losses.append((i, float(torch.mean((soft - truth) ** 2))))
    trained = alpha.detach().clone()

    # BER of the trained steps against fixed-tau TASER on held-out instances: the training
    # distribution (SNR uniform in [4, 14] dB), and fixed low SNRs where errors are frequent
    # enough to separate the two.
    n_eval, chunk = 65536, 8192

    def heldout(snr, seed0):
        err = {"trained": 0, "fixed": 0, "discordant": 0}
        for k in range(n_eval // chunk):
            H, y, truth = make_mimo_device(chunk, B, U, snr, "qpsk", seed=seed0 + k, device=dev)
            out = taser.build_T("mimo_qpsk", H, y, ALPHA)
            _, s_tr, _ = taser.unfolded_forward(out["T_tilde"], out["D"], 1.0 / out["spec_norm"], trained, c,
                                                want_ckpt=False, precision=precision)
            s_fx, _, _ = taser.detect(out["T_tilde"], out["D"], out["tau"], t_max, precision, want_L=False)
            err["trained"] += int((s_tr != truth).sum())
            err["fixed"] += int((s_fx != truth).sum())
            err["discordant"] += int((s_tr != s_fx).sum())
        nbits = n_eval * (N - 1)
        r = {k: {"bit_errors": err[k], "ber": err[k] / nbits, "ber_ci95": list(clopper_pearson(err[k], nbits))}
             for k in ("trained", "fixed")}
        return {"instances": n_eval, "snr_db": snr if isinstance(snr, float) else "uniform %g..%g" % tuple(snr),
                "trained_alpha_t": r["trained"], "fixed_alpha_0.5": r["fixed"], "discordant_bits": err["discordant"],
                "trained_better": r["trained"]["ber_ci95"][1] < r["fixed"]["ber_ci95"][0],
                "fixed_better": r["fixed"]["ber_ci95"][1] < r["trained"]["ber_ci95"][0]}

    held = [heldout((4.0, 14.0), 90_000)] + [heldout(float(snr), 91_000 + 100 * i)
                                             for i, snr in enumerate((0.0, 2.0, 4.0))]
    props = torch.cuda.get_device_properties(dev)
    fp32_peak = props.multi_processor_count * 128 * 2 * 2070.0e6 / 1e12
    P = N * (N + 1) * (2 * N + 1) // 6
    it_fwd = 2 * P + 3 * N * (N + 1) // 2 + N
    fwd_fl = t_max * it_fwd
    bwd_fl = t_max * it_fwd + t_max * (2 * P + 9 * N * (N + 1) // 2)   # one recompute + the adjoint
    fwd_tf = n * fwd_fl / (fwd_ms * 1e-3) / 1e12
    bwd_tf = n * bwd_fl / (bwd_ms * 1e-3) / 1e12
    print(json.dumps({
        "metric": "unfolded TASER training instances/s, QPSK 128x16 (N = 33), t_max = 10, batch 8,192",
        "value": n / (step_ms * 1e-3), "unit": "instances/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "dtype": "f32" if precision == "fp32" else "bf16",
        "cuda_graph": graph, "eager_ms_per_step": ms, "eager_instances_per_s": n / (ms * 1e-3),
        "data": "synthetic, a fresh seeded batch drawn on the GPU every step",
        "config": {"workload": "unfolded_qpsk128x16_tmax10_c4_batch8192", "instances_per_step": n, "t_max": t_max,
                   "checkpoint_every": c, "precision": precision,
                   "step": "draw batch + build_T + forward + loss gradient + adjoint + Adam"},
        "draw_ms": gen_ms, "forward_ms": fwd_ms, "backward_ms": bwd_ms, "train_steps": args.train_steps,
        "loss_trace": losses, "alpha_t": [round(float(a), 4) for a in trained.cpu()],
        "heldout_ber": held,
        "roofline_forward": {"bound": "alu", "achieved": fwd_tf, "peak": fp32_peak, "unit": "TFLOP/s",
                             "frac": fwd_tf / fp32_peak, "algorithmic_flops_per_instance": fwd_fl},
        "roofline_backward": {"bound": "alu", "achieved": bwd_tf, "peak": fp32_peak, "unit": "TFLOP/s",
                              "frac": bwd_tf / fp32_peak, "algorithmic_flops_per_instance": bwd_fl}}))
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "uneven":
        return run_uneven(args)
    if args.workload == "tradeoff":
        return run_tradeoff(args)
    if args.workload == "unfolded":
        return run_unfolded(args)
    if args.workload == "ber":
        return run_ber(args)
    if args.workload == "jed":
        return run_jed(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_1609_01797_gb300 as taser
    from paper_1609_01797_gb300.replicas import max_over_ranks, sum_over_ranks

    n = args.instances
    w = make_workload(n, seed=1 + 1000 * rank)
    bits = truth_bits(w)
    H = torch.from_numpy(w["H"]).to(dev)
    y = torch.from_numpy(w["y"]).to(dev)
    bufs = {"T_tilde": torch.empty((n, N, N), device=dev), "D": torch.empty((n, N), device=dev),
            "tau": torch.empty((n,), device=dev), "flags": torch.zeros((n,), device=dev, dtype=torch.int32)}
    s_hat = torch.empty((n, N - 1), device=dev, dtype=torch.int8)
    nrm_buf = torch.empty((n,), device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def one_step(precision, ev=None):
        # taser_build_T (T~, D) -> taser_step_size (tau, QPSK structure) -> taser_detect
        if ev is not None:
            ev[0].record(stream)
        taser.build_T("mimo_qpsk", H, y, ALPHA, out=bufs, with_tau=False)
        if ev is not None:
            ev[1].record(stream)
        taser.step_size(bufs["T_tilde"], ALPHA, structure="mimo_qpsk", tau=bufs["tau"], spec_norm=nrm_buf)
        if ev is not None:
            ev[2].record(stream)
        taser.detect(bufs["T_tilde"], bufs["D"], bufs["tau"], T_MAX, precision, want_L=False,
                     flags=bufs["flags"], out_s=s_hat)
        if ev is not None:
            ev[3].record(stream)

    def run_path(precision, steps, warmup):
        for _ in range(warmup):
            one_step(precision)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize(dev)
        start.record(stream)
        for i in range(steps):
            one_step(precision, ev[i])
        end.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        ms = start.elapsed_time(end) / steps
        build_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / steps
        spectral_ms = sum(e[1].elapsed_time(e[2]) for e in ev) / steps
        detect_ms = sum(e[2].elapsed_time(e[3]) for e in ev) / steps
        per_step = sorted(e[0].elapsed_time(e[3]) for e in ev)   # build start to detect end
        errs = int((s_hat.cpu().numpy() != bits).sum())
        return {"ms_per_step": ms, "build_ms": build_ms, "spectral_ms": spectral_ms, "detect_ms": detect_ms,
                "step_ms_median": statistics.median(per_step), "step_ms_min": per_step[0], "bit_errors": errs}

    sampler = ClockSampler(local)
    sampler.start()
    paths = {}
    for precision in ("bf16_tc", "fp32", "fp16_tc", "fixed14"):
        paths[precision] = run_path(precision, args.steps, args.warmup)
    clocks = sampler.stop()

    # e2e through the C ABI with host buffers: H2D of H and y, the full path, D2H of s_hat.
    H_host = torch.from_numpy(w["H"]).pin_memory()
    y_host = torch.from_numpy(w["y"]).pin_memory()
    s_host = torch.empty((n, N - 1), dtype=torch.int8).pin_memory()
    ws = torch.empty(taser.host_workspace_bytes("mimo_qpsk", n, B, U), device=dev, dtype=torch.uint8)
    for _ in range(args.warmup):
        taser.run_host("mimo_qpsk", H_host, y_host, ALPHA, T_MAX, "bf16_tc", ws, s_host)
    torch.cuda.synchronize(dev)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        taser.run_host("mimo_qpsk", H_host, y_host, ALPHA, T_MAX, "bf16_tc", ws, s_host)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    e2e_errs = int((s_host.numpy() != bits).sum())
    # The host link's own rate: a plain pinned H2D copy of the same H (best of 3).
    h2d_bytes = int(H_host.numel() * 8 + y_host.numel() * 8)
    H_dev = torch.empty(H_host.shape, dtype=H_host.dtype, device=dev)
    link_ms = []
    for _ in range(3):
        e0.record(stream)
        H_dev.copy_(H_host, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        link_ms.append(e0.elapsed_time(e1))
    link_gbs = H_host.numel() * 8 / (min(link_ms) * 1e-3) / 1e9
    del H_dev

    # Whole-job numbers: max step time over ranks, instances summed over ranks.
    total = n * world
    for p in paths.values():
        p["ms_per_step"] = max_over_ranks(p["ms_per_step"], world)
        p["build_ms"] = max_over_ranks(p["build_ms"], world)
        p["spectral_ms"] = max_over_ranks(p["spectral_ms"], world)
        p["detect_ms"] = max_over_ranks(p["detect_ms"], world)
        p["step_ms_median"] = max_over_ranks(p["step_ms_median"], world)
        p["step_ms_min"] = max_over_ranks(p["step_ms_min"], world)
        p["bit_errors"] = sum_over_ranks(p["bit_errors"], world)
        p["det_per_s"] = total / (p["ms_per_step"] * 1e-3)
        p["detect_only_det_per_s"] = total / (p["detect_ms"] * 1e-3)
        nbits = total * (N - 1)
        p["ber"] = p["bit_errors"] / nbits
        p["ber_ci95"] = clopper_pearson(p["bit_errors"], nbits)
    lo, hi = paths["fp32"]["ber_ci95"]
    equal_ber = lo <= paths["bf16_tc"]["ber"] <= hi

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    peaks, peak_src = load_peaks()
    head = paths["bf16_tc"]
    smax = clocks.get("sm_max_mhz") or 2070.0
    props = torch.cuda.get_device_properties(dev)
    fp32_peak = props.multi_processor_count * 128 * 2 * smax * 1e6 / 1e12   # TFLOP/s, FMA = 2 flops
    bf16_peak = _peak(peaks, "bf16_tflops", "bf16_dense_tflops") or 1900.0
    hbm_peak = _peak(peaks, "hbm_gbs", "hbm_GBps", "copy_gbs") or 6800.0
    fl = flops_per_detection(N, T_MAX)
    traffic = measured_traffic()

    def tr(key):
        return traffic[key] * n if key in traffic else None

    det_tc = n / (head["detect_ms"] * 1e-3) / 1e12 * fl                      # TFLOP/s per GPU
    padded_tf = n / (head["detect_ms"] * 1e-3) / 1e12 * (14 * 4096 * T_MAX)
    prox_fl = T_MAX * (3 * N * (N + 1) // 2 + N)
    in_bytes = 4 * (N * (N - 1) // 2 + N + 1)
    bounds = {"tensor": bf16_peak * 1e12 / fl, "fp32_prox": fp32_peak * 1e12 / prox_fl,
              "hbm": hbm_peak * 1e9 / in_bytes}
    composite_by = min(bounds, key=bounds.get)
    composite = bounds[composite_by]
    pipe_util = measured_traffic("pipe_util.txt")
    build_gbs = n * build_bytes_per_instance(B, U, N) / (head["build_ms"] * 1e-3) / 1e9
    spec_tf = n * spectral_flops_per_instance(U) / (head["spectral_ms"] * 1e-3) / 1e12
    roofs = {
        "detect": (head["detect_ms"], {
            "kernel": "detect_tct_kernel<32,bf16> (transposed form, mma.sync m16n8k16)", "bound": "tensor", "achieved": det_tc,
            "peak": bf16_peak, "unit": "TFLOP/s", "frac": det_tc / bf16_peak, "traffic": tr("detect_tc"),
            "peak_source": peak_src, "algorithmic_flops_per_launch": fl * n, "ms_per_launch": head["detect_ms"],
            "fp32_pipe_frac": det_tc / fp32_peak,
            # the mma.sync work actually issued: 14 m16n8k16 per iteration at N = 33 (m-tile 0 of
            # the columns k: 1 + 1 + 2 + 2 + 2 over n-tiles 0..4, m-tile 1: 2 + 2 + 2 over n-tiles
            # 2..4; n-tile 4 holds row N), 4,096 flops each
            "padded_issue": {"flops_per_instance": 14 * 4096 * T_MAX, "achieved": padded_tf, "unit": "TFLOP/s",
                             "frac": padded_tf / bf16_peak},
            # min(tensor pipe at the algorithmic flops, FP32 pipe at the prox's flops, HBM at the
            # algorithmic input bytes of T~ lower off-diagonal, D and tau) in detections/s
            "composite_bound": {"det_per_s": composite, "limited_by": composite_by,
                                "achieved_det_per_s": n / (head["detect_ms"] * 1e-3),
                                "frac": n / (head["detect_ms"] * 1e-3) / composite},
            "tensor_pipe_active_ncu": pipe_util.get("detect_tc")}),
        "build": (head["build_ms"], {
            "kernel": "build_T_kernel<17> (TMA-staged, FP16 split mma.sync Gram)", "bound": "hbm", "achieved": build_gbs,
            "peak": hbm_peak, "unit": "GB/s", "frac": build_gbs / hbm_peak, "traffic": tr("build"),
            "peak_source": peak_src, "algorithmic_bytes_per_launch": n * build_bytes_per_instance(B, U, N),
            "ms_per_launch": head["build_ms"]}),
        "spectral": (head["spectral_ms"], {
            "kernel": "spectral_herm_fold_kernel<16> (Householder, two columns a lane, + Sturm)", "bound": "alu", "achieved": spec_tf,
            "peak": fp32_peak, "unit": "TFLOP/s", "frac": spec_tf / fp32_peak, "traffic": tr("spectral"),
            "peak_source": "derived FP32 pipe", "algorithmic_flops_per_launch": n * spectral_flops_per_instance(U),
            "ms_per_launch": head["spectral_ms"]}),
    }
    order = sorted(roofs, key=lambda k: -roofs[k][0])
    dominant = roofs[order[0]][1]
    others = {k: roofs[k][1] for k in order[1:]}
    fp32 = paths["fp32"]
    det_fp32 = n / (fp32["detect_ms"] * 1e-3) / 1e12 * fl
    out = {
        "metric": METRIC,
        "value": head["det_per_s"],
        "unit": "detections/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"],
        # per step, from the events around its first and last kernel (the gaps between steps
        # are outside): the median and the minimum over the timed steps
        "ms_per_step_median": head["step_ms_median"],
        "ms_per_step_min": head["step_ms_min"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "instances_per_gpu": n, "B": B, "U": U, "N": N, "t_max": T_MAX,
                   "alpha": ALPHA, "snr_db": "0..20 step 2, cycled over instances",
                   "l2": "inputs (%.2f GB per GPU) larger than L2; no flush" % (n * (8 * B * U + 8 * B) / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "paths": {k: {"det_per_s": v["det_per_s"], "detect_only_det_per_s": v["detect_only_det_per_s"],
                      "ms_per_step": v["ms_per_step"], "build_ms": v["build_ms"], "spectral_ms": v["spectral_ms"],
                      "detect_ms": v["detect_ms"], "step_ms_median": v["step_ms_median"],
                      "step_ms_min": v["step_ms_min"], "ber": v["ber"], "ber_ci95": v["ber_ci95"]}
                  for k, v in paths.items()},
        "equal_ber": equal_ber,
        "speedup_bf16_vs_fp32": fp32["ms_per_step"] / head["ms_per_step"],
        "roofline": dominant,
        "roofline_other": others,
        "roofline_fp32_path": {"kernel": "detect_fp32_kernel<32>", "bound": "alu", "achieved": det_fp32,
                               "peak": fp32_peak, "unit": "TFLOP/s", "frac": det_fp32 / fp32_peak,
                               "traffic": tr("detect_fp32"),
                               "peak_source": "derived: %d SMs x 128 FP32 lanes x 2 x %.0f MHz"
                                              % (props.multi_processor_count, smax)},
        "clocks": clocks,
        "e2e": {"value": total / (e2e_ms * 1e-3), "unit": "detections/s",
                "h2d_bytes_per_step": h2d_bytes,
                "d2h_bytes_per_step": int(s_host.numel()), "ms_per_step": e2e_ms,
                "path": "taser_run_host (bf16_tc)", "bit_errors": e2e_errs,
                "host_link": {"h2d_gbs": link_gbs, "bound": total / (h2d_bytes / (link_gbs * 1e9)),
                              "frac": (total / (e2e_ms * 1e-3)) / (total / (h2d_bytes / (link_gbs * 1e9))),
                              "note": "bound = instances / (H2D bytes / measured pinned H2D rate)"}},
        "gpu_launches": 3 * args.steps,
    }
    if world == 1 and not args.no_cpu_baseline:
        sample = min(args.cpu_sample, n)
        out["cpu_baseline"], r = cpu_baseline(w, sample)
        out["error_vs_fp64"] = error_vs_fp64(taser, bufs, r, sample)
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
