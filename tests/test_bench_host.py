"""Host logic of bench.py (no GPU): the algorithmic work figures its roofline divides by, the
source hash that keeps committed ncu counters tied to the kernel code they were taken on,
and the Clopper-Pearson interval of the equal-BER check."""
import pytest

import bench


def test_flops_per_detection_is_the_triangular_count():
    """t_max (2 P(N) + 3 N (N+1) / 2 + N) with P(N) = N (N+1) (2N+1) / 6 multiply-adds per
    iteration (Table I's triangular array): 535,480 at N = 33, t_max = 20."""
    assert bench.flops_per_detection(33, 20) == 535_480
    for n, t in ((9, 10), (17, 20), (65, 20)):
        p = n * (n + 1) * (2 * n + 1) // 6
        assert bench.flops_per_detection(n, t) == t * (2 * p + 3 * n * (n + 1) // 2 + n)


def test_build_bytes_are_inputs_once_and_outputs_once():
    """H (B x U complex64) and y read once, T~ (N x N) and D (N) written once: 21,896 bytes
    per QPSK 128x16 instance."""
    assert bench.build_bytes_per_instance(128, 16, 33) == 21_896
    assert bench.build_bytes_per_instance(32, 4, 9) == 8 * 32 * 4 + 8 * 32 + 4 * 81 + 4 * 9


def test_spectral_flops_count_the_folded_search():
    n = 17
    assert bench.spectral_flops_per_instance(16) == 16 * n ** 3 // 3 + 7 * 8 * n * 4


def test_source_sha_ignores_comments_only(tmp_path):
    a = tmp_path / "a.cu"
    a.write_text("int f(int x) {\n  return x + 1;  // one\n}\n")
    b = tmp_path / "b.cu"
    b.write_text("// a new header line\nint f(int x) {\n\n  return x + 1;  // another comment\n}\n")
    c = tmp_path / "c.cu"
    c.write_text("int f(int x) {\n  return x + 2;\n}\n")
    assert bench.source_sha(str(a)) == bench.source_sha(str(b))
    assert bench.source_sha(str(a)) != bench.source_sha(str(c))


def test_measured_traffic_keeps_only_counters_of_unchanged_code(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1609_01797_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "build_T.cu").write_text("int build() { return 1; }\n")
    (csrc / "spectral.cu").write_text("int spectral() { return 2; }\n")
    good = bench.source_sha(str(csrc / "build_T.cu"))
    (tmp_path / "profiles" / "dram_traffic.txt").write_text(
        "# comment line\n"
        "build 20316.6 %s\n"
        "spectral 4356.6 %s\n"
        "detect_tc 4494.6 %s\n" % (good, "0" * 40, good))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    got = bench.measured_traffic()
    # build matches its source; spectral's counters were taken on other code; detect_tc's
    # source file does not exist here
    assert got == {"build": pytest.approx(20316.6)}


def test_clopper_pearson_closed_forms():
    """Zero errors: [0, 1 - (alpha/2)^(1/n)]; all errors: [(alpha/2)^(1/n), 1]."""
    n = 100
    lo, hi = bench.clopper_pearson(0, n)
    assert lo == 0.0 and hi == pytest.approx(1 - 0.025 ** (1 / n), rel=1e-9)
    lo, hi = bench.clopper_pearson(n, n)
    assert hi == 1.0 and lo == pytest.approx(0.025 ** (1 / n), rel=1e-9)
    lo, hi = bench.clopper_pearson(7, 1000)
    assert lo < 7 / 1000 < hi
    lo99, hi99 = bench.clopper_pearson(7, 1000, conf=0.99)
    assert lo99 < lo and hi < hi99            # a higher confidence widens the interval
