"""SSSP on the heap (Section 5.7.1) against textbook Dijkstra, through the C ABI.

Shortest-path distances are unique, so every distance must equal the
oracle's bit for bit, whatever batch size and heap shape the GPU run uses.
Beyond the distances: every inserted key is deleted exactly once
(keys_deleted = keys_inserted + 1 for the source key), and with one key per
deleteMin the heap pops in exact Dijkstra order, so each reachable vertex is
expanded exactly once.
"""
import numpy as np
import pytest

import oracle
from paper_1906_06504_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

U32_MAX = 0xFFFFFFFF


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_06504_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def SSSP(*a, **kw):
    from paper_1906_06504_gb300.apps import SSSP as S
    return S(*a, **kw)


def to_dev(rowptr, col, w):
    r = torch.from_numpy(np.ascontiguousarray(rowptr, dtype=np.uint64).view(np.int64)).cuda()
    c = torch.from_numpy(np.ascontiguousarray(col, dtype=np.uint32).view(np.int32)).cuda()
    ww = torch.from_numpy(np.ascontiguousarray(w, dtype=np.uint32).view(np.int32)).cuda()
    return r, c, ww


def run_gpu(graph, source=0, k=1024, batch=16384, heap_capacity=0, ctx=None):
    rowptr, col, w = graph
    n, e = rowptr.size - 1, col.size
    d = to_dev(rowptr, col, w)
    own = ctx is None
    ctx = ctx or SSSP(n, e, k=k, batch=batch, heap_capacity=heap_capacity)
    try:
        dist, stats = ctx.run(*d, source=source)
        torch.cuda.synchronize()
        return dist.cpu().numpy().view(np.uint32), stats
    finally:
        if own:
            ctx.close()


def check(graph, source=0, **kw):
    got, stats = run_gpu(graph, source=source, **kw)
    want = oracle.dijkstra(*graph, src=source)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, (bad[:10], got[bad[:10]], want[bad[:10]])
    assert stats["keys_deleted"] == stats["keys_inserted"] + 1
    assert stats["visited"] >= int((want != U32_MAX).sum())
    return got, want, stats


def csr(n, edges):
    """CSR of a directed edge list [(u, v, w), ...]."""
    if not edges:
        return np.zeros(n + 1, np.uint64), np.zeros(0, np.uint32), np.zeros(0, np.uint32)
    u, v, w = (np.array(x, dtype=np.int64) for x in zip(*edges))
    return inputs._to_csr(n, u, v, w)


@pytest.mark.parametrize("k,batch", [(64, 64), (64, 1000), (256, 4096), (1024, 16384)])
def test_grid_small(k, batch):
    check(inputs.grid_graph(48, inputs.config_seed(3)), k=k, batch=batch)


def test_exact_order_with_one_key_per_batch():
    """batch = 1, k = 1: the heap is a plain priority queue and the run is
    Dijkstra itself; each reachable vertex is expanded once."""
    g = inputs.rmat_graph(10, 8, inputs.config_seed(3) + 7)
    got, want, st = check(g, k=1, batch=1)
    assert st["visited"] == int((want != U32_MAX).sum())
    assert st["iterations"] == st["keys_deleted"]


@pytest.mark.parametrize("k", [8, 64])
def test_exact_order_k_keys_per_node(k):
    """A batch of one key still comes from the root of a k-key heap: exact
    Dijkstra order whatever k."""
    g = inputs.grid_graph(40, inputs.config_seed(3) + 1)
    got, want, st = check(g, k=k, batch=1)
    assert st["visited"] == int((want != U32_MAX).sum())


def test_rmat_small_multi_edges_and_self_loops():
    g = inputs.rmat_graph(14, 8, inputs.config_seed(3) + 2)
    rowptr, col, _ = g
    src = np.repeat(np.arange(rowptr.size - 1), np.diff(rowptr.astype(np.int64)))
    assert (src == col).any()                  # self-loops present
    check(g, k=256, batch=2048)


def test_heavy_vertices_are_spread_over_the_grid():
    """A hub with 300,000 out-edges (above the per-block expansion limit) and
    a second hub reached through it."""
    n = 400_000
    rng = np.random.default_rng(5)
    e = [(0, int(v), int(rng.integers(1, 1000))) for v in range(1, 300_001)]
    e += [(7, int(v), int(rng.integers(1, 50))) for v in range(200_000, 400_000)]
    e += [(int(v), int(v) + 1, 3) for v in range(1000, 1200)]
    g = csr(n, e)
    check(g, k=1024, batch=4096)


def test_edge_cases():
    # one vertex, no edges
    check(csr(1, []), k=64, batch=64)
    # no edges at all, source not 0
    got, _, st = check(csr(5, []), source=3, k=64, batch=64)
    assert list(got) == [U32_MAX] * 3 + [0] + [U32_MAX]
    # two components; source the last vertex; zero-weight edges
    e = [(0, 1, 4), (1, 2, 0), (2, 0, 0), (3, 4, 0), (4, 5, 7), (5, 3, 1), (5, 4, 0)]
    got, _, _ = check(csr(6, e), source=5, k=8, batch=3)
    assert list(got[:3]) == [U32_MAX] * 3
    # distances at the top of the representable range: 2^32 - 2 is reachable,
    # 2^32 - 1 is not
    big = 0xFFFFFFFF
    e = [(0, 1, big - 1), (1, 2, 1), (0, 3, big), (0, 4, 1), (4, 5, big - 3)]
    got, _, _ = check(csr(6, e), k=64, batch=64)
    assert got[1] == big - 1 and got[2] == U32_MAX and got[3] == U32_MAX and got[5] == big - 2


def test_context_reuse_and_smaller_graph():
    g = inputs.grid_graph(64, inputs.config_seed(3) + 3)
    small = inputs.grid_graph(20, inputs.config_seed(3) + 4)
    n, e = g[0].size - 1, g[1].size
    with SSSP(n, e, k=256, batch=2048) as ctx:
        for graph, src in ((g, 0), (g, n - 1), (small, 17), (g, 1234)):
            got, _ = run_gpu(graph, source=src, ctx=ctx)
            assert np.array_equal(got, oracle.dijkstra(*graph, src=src))


def test_heap_full_is_reported():
    from paper_1906_06504_gb300.heap import ERR_FULL, GHeapError
    g = inputs.rmat_graph(12, 8, inputs.config_seed(3) + 5)   # vertex 0: ~1000 out-edges
    with pytest.raises(GHeapError) as ei:
        run_gpu(g, k=64, batch=64, heap_capacity=128)
    assert ei.value.code == ERR_FULL


def test_argument_errors():
    from paper_1906_06504_gb300.heap import GHeapError
    with pytest.raises(GHeapError):
        SSSP(0, 10)
    with pytest.raises(GHeapError):
        SSSP(10, 10, batch=0)
    g = inputs.grid_graph(8, 1)
    with SSSP(64, g[1].size, k=64, batch=64) as ctx:
        with pytest.raises(GHeapError):
            run_gpu(g, source=64, ctx=ctx)
        big = inputs.grid_graph(9, 1)
        with pytest.raises(GHeapError):
            run_gpu(big, ctx=ctx)


def test_grid_1024_full_size():
    """The 1024 x 1024 grid, weights U[1, 100], source 0."""
    check(inputs.grid_graph(1024, inputs.config_seed(3)), k=1024, batch=16384)


def test_rmat_2p20_full_size():
    """R-MAT with 2^20 vertices, 2^23 edges, weights U[1, 1000], source 0."""
    check(inputs.rmat_graph(20, 8, inputs.config_seed(3)), k=1024, batch=16384)
