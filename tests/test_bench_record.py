"""bench.py's host-side bookkeeping, on the CPU: the committed ncu record of
the dominant kernel is taken on the kernel's current source (else the bench
line's `traffic` would be null), its traffic scales with the arcs swept, and
the BFS schedules the bench names are the ones its docstrings state."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _G:
    def __init__(self, m):
        self.m = m


def test_sweep_record_matches_the_kernel_source():
    raw = json.load(open(os.path.join(ROOT, "profiles", "pr_round_traffic.json")))
    for k in ("kernel", "source", "source_sha256_16", "command", "dram_bytes_per_launch",
              "arcs_per_launch", "ncu_limits"):
        assert k in raw, k
    d = bench.read_profile_record("pr_round")
    if d is None:
        pytest.skip("the record was taken on an earlier g2_pr_blk.cuh: the bench line's traffic "
                    "is null until the kernel is captured again")
    assert d["kernel"].startswith("k_pr_blk")
    lim = d["ncu_limits"]
    for k in ("issue_active_pct_of_active_cycles", "l1tex_throughput_pct", "dram_throughput_pct"):
        assert 0 < lim[k] <= 100, k


def test_sweep_traffic_scales_with_the_arcs():
    d = bench.read_profile_record("pr_round")
    if d is None:
        pytest.skip("no record taken on the current g2_pr_blk.cuh")
    per_arc = d["dram_bytes_per_launch"] / d["arcs_per_launch"]
    assert d["dram_bytes_per_launch"] == d["dram_bytes_read"] + d["dram_bytes_write"]
    for m in (10 ** 6, 128_305_908):
        assert bench.read_traffic("pr_round", _G(m)) == int(per_arc * m)


def test_record_of_a_changed_source_is_refused(tmp_path, monkeypatch):
    # a copy of the record whose hash no longer matches its source
    prof = tmp_path / "profiles"
    prof.mkdir()
    d = json.load(open(os.path.join(ROOT, "profiles", "pr_round_traffic.json")))
    d["source_sha256_16"] = "0" * 16
    (prof / "pr_round_traffic.json").write_text(json.dumps(d))
    csrc = tmp_path / "paper_2012_07990_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / d["source"]).write_text(
        open(os.path.join(ROOT, "paper_2012_07990_gb300", "csrc", d["source"])).read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.read_profile_record("pr_round") is None
    assert bench.read_traffic("pr_round", _G(10 ** 6)) is None


class _FakeG2:
    """The binding's schedule constructors, recording their arguments."""
    G2_PULL, G2_BITMAP, G2_UNFUSED_BITMAP = 1, 1, 1

    def schedule(self, lb, **kw):
        return ("schedule", lb, tuple(sorted(kw.items())))

    def hybrid(self, s1, s2, tau):
        return ("hybrid", s1, s2, tau)


def test_bench_bfs_schedules():
    g2 = _FakeG2()
    assert bench.bfs_schedule(g2) is None  # the library's tuned schedule
    kind, s1, s2, tau = bench.bfs_per_level_hybrid(g2)
    assert kind == "hybrid" and tau == 0.02
    assert s1[1] == "STRICT" and dict(s1[2]).get("kernel_fusion") is None
    kw = dict(s2[2])
    assert s2[1] == "VERTEX_BASED" and kw["direction"] == g2.G2_PULL
    assert kw["pull_frontier"] == g2.G2_BITMAP and "kernel_fusion" not in kw
