"""Query server: dispatcher logic on CPU with a fake executor (batching up to
the caps, concurrency over slots, memory admission, open-loop latencies), and
on the GPU the alone-vs-in-the-mix equality of every result."""
import threading
import time
import types

import numpy as np
import pytest

from paper_2012_07990_gb300 import serve


class FakeExecutor:
    def __init__(self, nslots, per_item=0.002):
        self.nslots = nslots
        self.per_item = per_item
        self.lock = threading.Lock()
        self.active = 0
        self.max_active = 0
        self.batches = []

    def execute(self, slot, batch):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
            self.batches.append([(r.graph, r.kind) for r in batch])
        time.sleep(0.003 + self.per_item * len(batch))
        with self.lock:
            self.active -= 1
        return {r.rid: r.src for r in batch}


def fake_pool(names=("a", "b", "c"), n=1000):
    graphs = {}
    for nm in names:
        host = types.SimpleNamespace(n=n)
        graphs[nm] = types.SimpleNamespace(host=host, comp_arcs=np.full(n, 10, np.int64),
                                           nonisolated=np.arange(n, dtype=np.int32))
    return types.SimpleNamespace(graphs=graphs)


def test_trace_is_poisson_with_the_mix():
    pool = fake_pool()
    tr = serve.make_trace(pool, rate=2000, duration=2.0, seed=3)
    assert 3700 < len(tr) < 4300
    kinds = np.array([r.kind for r in tr])
    assert abs((kinds == "bfs").mean() - 0.6) < 0.03 and abs((kinds == "bc").mean() - 0.1) < 0.02
    gaps = np.diff([r.t_arrival for r in tr])
    assert abs(gaps.mean() - 1 / 2000) < 5e-5 and np.all(gaps >= 0)


def test_same_graph_batching_caps_and_concurrency():
    pool = fake_pool()
    tr = serve.make_trace(pool, rate=4000, duration=0.3, seed=1)
    ex = FakeExecutor(nslots=4)
    st = serve.Server(ex, pool, mem_budget=1 << 40).run(tr)
    assert st.latencies_ms.size == len(tr)
    assert np.all(st.latencies_ms >= 0)
    for b in ex.batches:
        assert len(set(b)) == 1  # one graph and one kind per batch
        kind = b[0][1]
        assert len(b) <= {"bfs": 64, "sssp": 32, "bc": 1}[kind]
    assert st.mean_batch > 1.5  # requests that arrive while slots are busy get batched
    assert ex.max_active > 1 and st.max_concurrent <= 4  # slots overlap
    assert set(st.results) == {r.rid for r in tr}


def test_memory_admission_limits_concurrency():
    pool = fake_pool(n=1 << 20)
    tr = [serve.Request(i, 0.0, "a", "bfs", i) for i in range(8)]
    one = serve.batch_bytes("bfs", 1, 1 << 20)
    ex = FakeExecutor(nslots=4)
    st = serve.Server(ex, pool, max_batch=dict(bfs=1), mem_budget=2 * one).run(tr)
    assert ex.max_active <= 2 and st.latencies_ms.size == 8


def test_batches_shrink_to_fit_the_budget():
    pool = fake_pool(n=1 << 20)
    tr = [serve.Request(i, 0.0, "a", "bfs", i) for i in range(64)]
    budget = serve.batch_bytes("bfs", 16, 1 << 20)
    ex = FakeExecutor(nslots=1)
    serve.Server(ex, pool, mem_budget=budget).run(tr)
    assert max(len(b) for b in ex.batches) <= 16


def test_queue_choice_fifo_and_response_ratio():
    R = serve.Request
    pending = {("g", "bfs"): [R(0, 0.00, "g", "bfs", 0)],
               ("h", "bc"): [R(1, 0.05, "h", "bc", 0)],
               ("k", "sssp"): [R(2, 0.09, "k", "sssp", 0)]}
    cost = serve.CostModel()
    # a queue never measured goes first
    assert serve._pick_queue("hrrn", cost, pending, 0.1) == ("g", "bfs")
    cost.update(("g", "bfs"), 1.0)     # slow
    cost.update(("h", "bc"), 0.001)    # fast
    cost.update(("k", "sssp"), 0.001)  # fast, but younger
    assert serve._pick_queue("fifo", cost, pending, 0.1) == ("g", "bfs")
    assert serve._pick_queue("hrrn", cost, pending, 0.1) == ("h", "bc")
    # the slow queue's ratio grows with its wait until it beats fresh short
    # requests: (wait + 1) / 1 against (wait' + 0.001) / 0.001 with wait' small
    pending[("h", "bc")] = [R(3, 9.9995, "h", "bc", 0)]
    pending[("k", "sssp")] = [R(4, 9.9995, "k", "sssp", 0)]
    assert serve._pick_queue("hrrn", cost, pending, 10.0) == ("g", "bfs")
    cost.update(("h", "bc"), 0.003)
    assert abs(cost.get(("h", "bc")) - (0.7 * 0.001 + 0.3 * 0.003)) < 1e-12
    with pytest.raises(ValueError):
        serve.Server(FakeExecutor(1), fake_pool(), mem_budget=1, policy="lifo")


class CostlyExecutor(FakeExecutor):
    """Graph 'a' batches take 40 ms, the others 2 ms."""

    def execute(self, slot, batch):
        time.sleep(0.040 if batch[0].graph == "a" else 0.002)
        return {r.rid: r.src for r in batch}


def test_response_ratio_cuts_median_latency_under_overload():
    pool = fake_pool(names=("a", "b", "c", "d"))
    tr = serve.make_trace(pool, rate=3000, duration=0.25, seed=7)
    p50 = {}
    for policy in ("fifo", "hrrn"):
        st = serve.Server(CostlyExecutor(nslots=2), pool, mem_budget=1 << 40, policy=policy).run(tr)
        assert st.latencies_ms.size == len(tr)
        p50[policy] = st.p50
    assert p50["hrrn"] < 0.8 * p50["fifo"], p50


@pytest.mark.gpu
def test_results_alone_equal_results_in_the_mix():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_07990_gb300 import build_native
    from paper_2012_07990_gb300 import graphgen as gg
    build_native.build()
    from paper_2012_07990_gb300 import g2
    specs = [serve.GraphSpec("rmat12", lambda: gg.rmat(12, seed=1), 255, 64),
             serve.GraphSpec("rmat13", lambda: gg.rmat(13, seed=2), 255, 64),
             serve.GraphSpec("grid96", lambda: gg.road_grid(96, seed=1), 1000, 4096, True)]
    pool = serve.GraphPool(g2, specs)
    tr = serve.make_trace(pool, rate=3000, duration=0.15, seed=5)
    ex = serve.GpuExecutor(g2, pool, slots=4, keep_results=True)
    mix = serve.Server(ex, pool).run(tr)
    assert mix.mean_batch > 1.0 and mix.max_concurrent > 1
    alone = serve.serve_alone(g2, pool, tr)
    for r in tr:
        a, b = alone[r.rid], mix.results[r.rid]
        if r.kind == "bc":
            tol = 1e-6 * np.abs(a) + 1e-12 * max(np.abs(a).max(), 1.0)
            assert np.all(np.abs(a - b) <= tol), r
        else:
            assert np.array_equal(a, b), r
