"""The BFS entry point that allocates no device memory.

Some callers cannot call cudaMalloc (for instance code running inside another
runtime that has reserved the device memory for its own pool, or latency-bound
code that cannot afford the synchronisation an allocation may cause).
g2_bfs_csr_static serves them from a fixed scratch array inside the library.
This test calls it through the C ABI twice in a row (two different graphs and
sources, so the second call must not see the first call's leftovers) and
checks depth and parent against the regular g2_bfs entry point, bit-exact as
all BFS parity tests.  The file is named to be collected last.
"""
import numpy as np
import pytest

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


def static_bfs(g2, g, src):
    rp = torch.from_numpy(g.rowptr).cuda()
    cl = torch.from_numpy(g.col).cuda()
    d = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
    p = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
    g2.g2_bfs_csr_static(g.n, rp, cl, src, d, p)
    torch.cuda.synchronize()
    return d.cpu().numpy(), p.cpu().numpy()


def test_static_bfs_two_calls_match_g2_bfs(g2):
    cases = [(gg.rmat(14, seed=1), None), (gg.road_grid(300, seed=2), 0)]
    for g, src in cases:
        src = g.max_degree_vertex() if src is None else src
        want_d, want_p = regular_bfs(g2, g, src)
        got_d, got_p = static_bfs(g2, g, src)
        assert np.array_equal(got_d, want_d), g.name
        assert np.array_equal(got_p, want_p), g.name


def test_static_bfs_rejects_graphs_beyond_its_scratch(g2):
    n = (1 << 20) + 1
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    cl = torch.zeros(1, dtype=torch.int32, device="cuda")[:0]
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(g2.G2Error) as e:
        g2.g2_bfs_csr_static(n, rp, cl, 0, d)
    assert e.value.status == g2.G2_EINVAL
