"""Autotuner of the uneven-batch launch (taser_detect_uneven).

Per size bucket (N <= 9, 17, 33, 65) it times the candidate launch shapes (persistent
blocks per SM; items a warp takes per queue pop, 0 = the library's default) on a sample
batch with CUDA events, one bucket at a time with the others at their current best, and
keeps the fastest.  The result is a taser_uneven_tuning (and a JSON-able dict).
"""
import json

import torch

from .api import detect_uneven, tuning as make_tuning


def _time(fn, repeats):
    fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(repeats):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    times.sort()
    return times[len(times) // 2]


def tune_uneven(items, T_pool, D_pool, tau, s_pool, workspace, precision="bf16_tc", blocks_candidates=(1, 2, 3, 4, 0),
                pop_candidates=(0, 1, 2, 4, 8), repeats=5):
    """Returns (taser_uneven_tuning, report dict with the timings in ms)."""
    bps = [0, 0, 0, 0]
    pop = [0, 0, 0, 0]
    report = {"precision": precision, "buckets": {}}

    def run():
        detect_uneven(items, T_pool, D_pool, tau, s_pool, workspace, precision=precision,
                      tune=make_tuning(bps, pop))

    base = _time(run, repeats)
    report["default_ms"] = base
    for b in (3, 2, 1, 0):
        best = (base, bps[b], pop[b])
        pops = pop_candidates if precision != "fixed14" and b < 3 else (0,)
        for cand_b in blocks_candidates:
            for cand_p in pops:
                bps[b], pop[b] = cand_b, cand_p
                t = _time(run, repeats)
                if t < best[0]:
                    best = (t, cand_b, cand_p)
        bps[b], pop[b] = best[1], best[2]
        base = best[0]
        report["buckets"][str(8 << b)] = {"blocks_per_sm": best[1], "pop": best[2], "ms": best[0]}
    report["tuned_ms"] = base
    return make_tuning(bps, pop), report


def save(report, path):
    with open(path, "w") as f:
        json.dump(report, f, indent=1)


def load(path):
    """The taser_uneven_tuning of a report written by save() (checkpoint of a tuning run)."""
    with open(path) as f:
        report = json.load(f)
    bps, pop = [0, 0, 0, 0], [0, 0, 0, 0]
    for b in range(4):
        entry = report["buckets"].get(str(8 << b))
        if entry is not None:
            bps[b], pop[b] = int(entry["blocks_per_sm"]), int(entry["pop"])
    return make_tuning(bps, pop)
