"""The autotuner's report survives a save / load round trip as a launch tuning (no GPU)."""
import os

from paper_1609_01797_gb300 import autotune


def test_tuning_report_round_trip(tmp_path):
    report = {"precision": "bf16_tc", "default_ms": 1.7, "tuned_ms": 1.6,
              "buckets": {"64": {"blocks_per_sm": 2, "pop": 0, "ms": 1.6},
                          "32": {"blocks_per_sm": 0, "pop": 2, "ms": 1.6},
                          "16": {"blocks_per_sm": 3, "pop": 4, "ms": 1.6},
                          "8": {"blocks_per_sm": 1, "pop": 8, "ms": 1.6}}}
    path = os.path.join(tmp_path, "tuning.json")
    autotune.save(report, path)
    t = autotune.load(path)
    assert list(t.blocks_per_sm) == [1, 3, 0, 2]
    assert list(t.pop) == [8, 4, 2, 0]
