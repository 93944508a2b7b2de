"""The BFS entry point that allocates no device memory.

Some callers cannot call cudaMalloc (for instance code running inside another
runtime that has reserved the device memory for its own pool, or latency-bound
code that cannot afford the synchronisation an allocation may cause).
g2_bfs_csr_static serves them from a fixed scratch array inside the library.
This test calls it through the C ABI several times in a row -- a larger graph
first, then a smaller one, then the smaller one again from another source, so
that leftovers of an earlier call in the shared array (queue entries past the
smaller graph, counters, the round word) would show -- and checks depth and
parent of every call against the regular g2_bfs entry point and against the
CPU oracle, bit-exact as all BFS parity tests.  The file is named to be
collected last.
"""
import numpy as np
import pytest

import oracle
from paper_2012_07990_gb300 import graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_07990_gb300 import build_native
    build_native.build()
    from paper_2012_07990_gb300 import g2 as mod
    return mod


def regular_bfs(g2, g, src):
    dg = g2.load_graph(g)
    d = torch.empty(g.n, dtype=torch.int32, device="cuda")
    p = torch.empty(g.n, dtype=torch.int32, device="cuda")
    g2.g2_bfs(dg, src, d, p, g2.schedule("WM"))
    torch.cuda.synchronize()
    return d.cpu().numpy(), p.cpu().numpy()


def static_bfs(g2, n, rowptr, col, src):
    rp = torch.from_numpy(np.ascontiguousarray(rowptr, np.int32)).cuda()
    cl = torch.from_numpy(np.ascontiguousarray(col, np.int32)).cuda()
    d = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    p = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    g2.g2_bfs_csr_static(n, rp, cl, src, d, p)
    torch.cuda.synchronize()
    return d.cpu().numpy(), p.cpu().numpy()


def test_static_bfs_calls_in_a_row_match_g2_bfs_and_the_oracle(g2):
    grid = gg.road_grid(300, seed=2)            # 90,000 vertices
    rmat = gg.rmat(14, seed=1)                  # 16,384 vertices
    cases = [(grid, 0), (rmat, rmat.max_degree_vertex()), (rmat, 1234)]
    for g, src in cases:
        want_d, want_p = oracle.bfs_graph(g, src)
        reg_d, reg_p = regular_bfs(g2, g, src)
        got_d, got_p = static_bfs(g2, g.n, g.rowptr, g.col, src)
        assert np.array_equal(got_d, want_d) and np.array_equal(got_p, want_p), (g.name, src)
        assert np.array_equal(got_d, reg_d) and np.array_equal(got_p, reg_p), (g.name, src)


def test_static_bfs_rejects_graphs_beyond_its_scratch(g2):
    n = (1 << 20) + 1
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    cl = torch.zeros(1, dtype=torch.int32, device="cuda")[:0]
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(g2.G2Error) as e:
        g2.g2_bfs_csr_static(n, rp, cl, 0, d)
    assert e.value.status == g2.G2_EINVAL


def test_static_bfs_rejects_an_invalid_csr_without_traversing_it(g2):
    """The caller's CSR is checked on the device before the traversal reads
    it: a column id past n, a decreasing row offset and an offset past m each
    return G2_EINVAL; the next call with a valid graph is exact again."""
    g = gg.path(64)
    bad_col = g.col.copy()
    bad_col[10] = 5000
    bad_rows = g.rowptr.copy()
    bad_rows[20], bad_rows[21] = bad_rows[21], bad_rows[20]
    past_m = g.rowptr.copy()
    past_m[30] = g.m + 100
    for rp, cl in ((g.rowptr, bad_col), (bad_rows, g.col), (past_m, g.col)):
        with pytest.raises(g2.G2Error) as e:
            static_bfs(g2, g.n, rp, cl, 0)
        assert e.value.status == g2.G2_EINVAL
    want_d, want_p = oracle.bfs_graph(g, 0)
    got_d, got_p = static_bfs(g2, g.n, g.rowptr, g.col, 0)
    assert np.array_equal(got_d, want_d) and np.array_equal(got_p, want_p)
