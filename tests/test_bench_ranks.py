"""bench.py under several ranks (replicas, no data-path collective): the job
time is the slowest rank's, the throughput counts every rank's edges, and the
reference arm runs on rank 0 only.  Two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow replica
    t = bench.max_over_ranks(local_ms, ws)
    out[rank] = (t, bench.job_gteps(ws, 10 ** 9, 4, t))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_all_edges():
    ws, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
    for r in range(ws):
        t, v = out[r]
        assert t == 150.0
        assert abs(v - 2 * 4 * 1e9 / 0.150 / 1e9) < 1e-9


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert abs(bench.job_gteps(1, 2 * 10 ** 9, 10, 1000.0) - 20.0) < 1e-12


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"scale": 10, "warmup": 0, "steps": 1})()
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
