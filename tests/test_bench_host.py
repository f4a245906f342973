"""Host logic of the benchmark (no GPU): the roofline figures it takes from
the committed ncu summary of the count traversal are used only while that
summary was captured on the current traversal source, and then they agree
with the algorithmic bytes of one full-size launch."""
import pytest

import bench


def test_profile_figures_agree_with_the_algorithmic_bytes():
    v = bench.profile_values()
    # a capture of another traversal source is an error, not a skip: every
    # change to the traversal needs a new capture
    assert v, ("profiles/k_query_fp32_count_c2.md predates the current traversal source "
               f"(source_hash {bench.source_hash()}): capture it again")
    # one launch answers 1e7 segments in count mode: 24 B in + 4 B out each
    algorithmic = bench.BYTES_PER_RAY_COUNT * 10_000_000
    assert 0.9 * algorithmic <= bench.traffic_per_launch() <= 1.25 * algorithmic
    b = bench.issue_bound()
    for k in ("issue_active_frac", "l1tex_throughput_frac", "lts_throughput_frac"):
        assert 0.0 < b[k] < 1.0, k


def test_c3_profile_figures_agree_with_the_algorithmic_bytes():
    """The c3 leg's traffic comes from its own capture (6e6 of the leg's 1e8
    segments, scaled); it too must match the current traversal source."""
    v = bench.profile_values(bench.TRAFFIC_SUMMARY_C3)
    assert v, ("profiles/k_query_fp32_count_c3.md predates the current traversal source "
               f"(source_hash {bench.source_hash()}): capture it again")
    algorithmic = bench.BYTES_PER_RAY_COUNT * 100_000_000
    assert 0.9 * algorithmic <= v["dram_bytes_per_launch_full_size"] <= 1.25 * algorithmic


def test_stale_profile_is_not_used(monkeypatch):
    monkeypatch.setattr(bench, "source_hash", lambda: "0000000000000000")
    assert bench.profile_values() == {}
    assert bench.traffic_per_launch() is None and bench.issue_bound() is None
    assert "STALE" in bench.second_bound()["stale"]


def _json_lines(out):
    import json
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the oracle on the host cores and
    prints one JSON line with the keys the benchmark contract names."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--ref-rays", "300"], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    (line,) = _json_lines(r.stdout)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["warmup"] == 3 and line["steps"] == 1
    assert line["value"] > 0 and line["e2e"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert "workload" in line["config"] and line["config"]["rays_per_step"] == 300


def test_reference_arm_under_two_ranks_prints_once():
    """Launched as the benchmark contract launches N > 1 (torchrun, here on
    gloo CPU ranks): rank 0 alone runs and prints, the other rank exits 0."""
    import os
    import socket
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
                        "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-rays", "200"],
                       cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    (line,) = _json_lines(r.stdout)
    assert line["impl"] == "reference" and line["n_gpus"] == 2
