"""Host logic of the benchmark (no GPU): the roofline figures it takes from
the committed ncu summary of the count traversal are used only while that
summary was captured on the current traversal source, and then they agree
with the algorithmic bytes of one full-size launch."""
import pytest

import bench


def test_profile_figures_agree_with_the_algorithmic_bytes():
    v = bench.profile_values()
    if not v:
        pytest.skip("the committed traversal profile predates the current source (the bench reports null)")
    # one launch answers 1e7 segments in count mode: 24 B in + 4 B out each
    algorithmic = bench.BYTES_PER_RAY_COUNT * 10_000_000
    assert 0.9 * algorithmic <= bench.traffic_per_launch() <= 1.25 * algorithmic
    b = bench.issue_bound()
    for k in ("issue_active_frac", "l1tex_throughput_frac", "lts_throughput_frac"):
        assert 0.0 < b[k] < 1.0, k


def test_stale_profile_is_not_used(monkeypatch):
    monkeypatch.setattr(bench, "source_hash", lambda: "0000000000000000")
    assert bench.profile_values() == {}
    assert bench.traffic_per_launch() is None and bench.issue_bound() is None
