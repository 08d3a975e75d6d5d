"""Host statistics of the benchmark: the exact sign test against the binomial
distribution and the bootstrap interval of the median."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


@pytest.mark.parametrize("wins,losses", [(0, 0), (30, 0), (0, 30), (20, 10), (15, 15), (3, 9)])
def test_sign_test_matches_binomial(wins, losses):
    stats = pytest.importorskip("scipy.stats")
    a = [1.0] * wins + [3.0] * losses + [2.0] * 4      # 4 ties, dropped
    b = [2.0] * (wins + losses + 4)
    w, l, p = bench.sign_test(a, b)
    assert (w, l) == (wins, losses)
    ref = 1.0 if wins + losses == 0 else stats.binomtest(wins, wins + losses, 0.5).pvalue
    assert p == pytest.approx(ref, rel=1e-12)


def test_median_ci_brackets_the_median():
    x = np.random.default_rng(3).normal(10.0, 1.0, size=30)
    med, lo, hi = bench.median_ci(x, resamples=2000)
    assert med == np.median(x) and lo <= med <= hi and hi - lo < 2.0
    assert bench.median_ci([5.0] * 30, resamples=500) == (5.0, 5.0, 5.0)


def test_issue_roofline_arithmetic():
    # 152 SMs x 4 schedulers x 2.07 GHz = 1.25856 T warp instructions/s
    r = bench.issue_roofline(195.3e6, 0.25, 152, 2070.0)
    assert r["peak"] == pytest.approx(1.25856)
    assert r["achieved"] == pytest.approx(195.3e6 / 0.25e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert bench.issue_roofline(None, 0.25, 152, 2070.0) is None
    assert bench.issue_roofline(1e6, 0.0, 152, 2070.0) is None


def test_link_roofline_arithmetic():
    # 200 MB in at 200 GB/s (1 ms) and 100 MB out at 100 GB/s (1 ms) in a 4 ms step
    r = bench.link_roofline({"h2d_gbs": 200.0, "d2h_gbs": 100.0}, 200_000_000, 100_000_000, 4.0)
    assert r["transfer_ms"] == pytest.approx(2.0) and r["frac"] == pytest.approx(0.5)
    assert bench.link_roofline({"h2d_gbs": 1.0, "d2h_gbs": 1.0}, 0, 0, 0.0)["frac"] is None


def test_profile_summaries_parse():
    # a summary is used only while it matches the kernel's sources; when it
    # does, both counters are present and plausible
    for path, wl in (("grid", "event300k"), ("grid", "event500k"), ("tc", "event500k")):
        p = bench.profile_summary(path, wl)
        if p is None:
            continue
        assert p["traffic"] > 10e6 and 10e6 < p["warp_instructions"] < 10e9
        assert bench.profiled_traffic(path, wl) == p["traffic"]
    assert bench.profile_summary("grid", "no-such-workload") is None


def test_cpu_baseline_compares_sampled_rows_with_the_library_result():
    # the oracle's own full result stands in for the library's: equal; one
    # index changed in a sampled row: not equal
    from oracle import oracle
    from paper_2609_31980_gb300 import synth
    pts = synth.clustered(50, 20, 500, 8, 0.02, seed=9)
    c, i, d, _ = oracle.self_query(pts, 0.1, 16)
    out = bench.cpu_baseline(pts, 0.1, 16, len(pts), gpu=(c, i, d))
    assert out["gpu_rows_equal"]["equal"] and out["gpu_rows_equal"]["rows"] == len(pts)
    assert out["kind"] == "oracle" and out["cores"] >= 1
    i2 = i.copy()
    i2[5, 0] += 1
    assert not bench.cpu_baseline(pts, 0.1, 16, len(pts), gpu=(c, i2, d))["gpu_rows_equal"]["equal"]
