"""The bounds-checked build (libtaser_debug.so, -DTASER_DEBUG) on the GPU.

compute-sanitizer is not available, so the debug build stands in for it: every kernel
checks the global and shared-memory indices it computes at run time and counts (and
skips) any that fail, without trapping.  Here the GPU suites of every entry point run in
child pytest sessions with TASER_LIBRARY=debug; conftest.py reads the counters when a
session ends and writes them to TASER_DEBUG_REPORT.

  * every suite except the non-finite-input cases: its own checks pass (against the
    oracle and the release library's contracts), no index check fails and no output is
    non-finite;
  * the non-finite-input cases: no index check fails and the non-finite outputs that the
    NaN inputs produce are counted;
  * test_gpu_debug_checks.py: an invalid uneven item is counted and skipped, and a
    withheld TMA staging copy ends in the bounded wait's timeout flag.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUITES = ["tests/test_gpu_parity.py", "tests/test_gpu_fixed.py", "tests/test_gpu_uneven.py",
          "tests/test_gpu_unfolded.py", "tests/test_gpu_monitor.py", "tests/test_zz_no_alloc.py"]


@pytest.fixture(scope="module")
def debug_lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01797_gb300 import build as B
    return B.build(debug=True)


def _session(args, report_path):
    env = dict(os.environ, TASER_LIBRARY="debug", TASER_DEBUG_REPORT=str(report_path))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-m", "gpu"] + args,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    rep = json.load(open(report_path)) if os.path.exists(report_path) else None
    return r, rep


def _tail(r):
    return r.stdout[-4000:] + r.stderr[-2000:]


def test_suites_pass_with_every_index_checked(debug_lib, tmp_path):
    r, rep = _session(SUITES + ["-k", "not nonfinite"], tmp_path / "finite.json")
    assert r.returncode == 0, _tail(r)
    assert rep is not None, _tail(r)
    assert rep["fails"] == 0 and rep["nonfinite"] == 0, rep


def test_nonfinite_inputs_are_counted(debug_lib, tmp_path):
    r, rep = _session(SUITES + ["-k", "nonfinite"], tmp_path / "nonfinite.json")
    assert r.returncode == 0, _tail(r)
    assert rep is not None, _tail(r)
    assert rep["fails"] == 0, rep
    assert rep["nonfinite"] > 0, rep


def test_failed_check_is_counted_and_skipped(debug_lib, tmp_path):
    r, rep = _session(["tests/test_gpu_debug_checks.py"], tmp_path / "control.json")
    assert r.returncode == 0, _tail(r)
    assert "3 passed" in r.stdout, _tail(r)
