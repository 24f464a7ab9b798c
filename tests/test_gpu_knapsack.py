"""0/1 knapsack branch and bound on the heap (Section 5.7.2) against the
textbook dynamic program, through the C ABI.

The optimum value is unique, so the GPU search must return exactly the
dynamic program's value on every instance, whatever the batch size, heap
shape and garbage-collection setting.
"""
import numpy as np
import pytest

import oracle
from paper_1906_06504_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_06504_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def Knapsack(*a, **kw):
    from paper_1906_06504_gb300.apps import Knapsack as K
    return K(*a, **kw)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def solve(w, v, cap, ctx=None, **kw):
    own = ctx is None
    ctx = ctx or Knapsack(max(len(w), 1), **kw)
    try:
        return ctx.run(dev(w), dev(v), cap)
    finally:
        if own:
            ctx.close()


def instance(kind, n, seed):
    w = inputs.uniform_range(seed, n, 1, 1000)
    if kind == "strong":
        v = w + 100
    elif kind == "uncorrelated":
        v = inputs.uniform_range(seed + 1, n, 1, 1000)
    elif kind == "subset":
        v = w.copy()
    else:
        raise ValueError(kind)
    cap = int(w.astype(np.int64).sum()) // 2
    return w.astype(np.uint32), v.astype(np.uint32), cap


@pytest.mark.parametrize("kind", ["strong", "uncorrelated", "subset"])
@pytest.mark.parametrize("n", [1, 2, 7, 20, 40])
def test_optimum_matches_dynamic_program(kind, n):
    for s in range(3):
        w, v, cap = instance(kind, n, inputs.config_seed(4) + 100 * n + s)
        st = solve(w, v, cap, k=64, batch=256)
        assert st["best"] == oracle.knapsack_dp(w, v, cap), (kind, n, s)


@pytest.mark.parametrize("k,batch", [(1, 1), (8, 3), (256, 1000), (1024, 16384)])
def test_heap_shapes(k, batch):
    w, v, cap = instance("strong", 40, inputs.config_seed(4) + 7)
    st = solve(w, v, cap, k=k, batch=batch)
    assert st["best"] == oracle.knapsack_dp(w, v, cap)
    assert st["explored"] > 0
    # every inserted key was either deleted or left behind dead
    assert st["keys_deleted"] <= st["keys_inserted"] + 1


def test_edge_cases():
    cases = [
        ([5], [7], 4),                      # the only item does not fit
        ([5], [7], 5),                      # it fits exactly
        ([3, 4, 5], [1, 2, 3], 0),          # capacity 0
        ([0, 0, 3], [5, 0, 4], 0),          # weightless items, one of them worthless
        ([1, 2, 3], [10, 20, 30], 100),     # everything fits: the greedy root is optimal
        ([10, 20, 30, 40], [10, 20, 30, 40], 50),   # all ratios equal
        ([7, 7, 7, 7, 7], [9, 9, 9, 9, 9], 20),      # identical items
    ]
    for w, v, cap in cases:
        w = np.array(w, np.uint32)
        v = np.array(v, np.uint32)
        st = solve(w, v, cap, k=8, batch=4)
        assert st["best"] == oracle.knapsack_dp(w, v, cap), (w, v, cap)
    # weights whose sums pass 2^32 (the dynamic program would need a table of
    # 2^32 entries): any two items fit, all three do not
    st = solve(np.array([2 ** 31, 2 ** 31 - 1, 5], np.uint32), np.array([3, 4, 5], np.uint32),
               2 ** 32 - 1, k=8, batch=4)
    assert st["best"] == 9


def test_garbage_collection_keeps_the_optimum():
    # about 57,000 nodes explored one at a time; the open list peaks near 2,800
    w, v, cap = instance("strong", 30, inputs.config_seed(4) + 50)
    plain = solve(w, v, cap, k=256, batch=512)
    gc = solve(w, v, cap, k=256, batch=512, gc_threshold=256)
    want = oracle.knapsack_dp(w, v, cap)
    assert plain["best"] == gc["best"] == want
    assert gc["gc_runs"] >= 1
    # keys leave the heap by a deleteMin or a filter pass, never twice
    assert gc["keys_deleted"] + gc["gc_dropped"] <= gc["keys_inserted"] + 1


def test_context_reuse():
    with Knapsack(64, k=256, batch=1024) as ctx:
        for s in range(4):
            w, v, cap = instance(["strong", "uncorrelated", "subset", "strong"][s], 30 + 10 * s,
                                 inputs.config_seed(4) + 50 + s)
            assert ctx.run(dev(w), dev(v), cap)["best"] == oracle.knapsack_dp(w, v, cap)


def test_node_pool_exhaustion_is_reported():
    from paper_1906_06504_gb300.heap import ERR_FULL, GHeapError
    w, v, cap = instance("strong", 40, inputs.config_seed(4) + 7)
    with pytest.raises(GHeapError) as ei:
        solve(w, v, cap, k=8, batch=8, max_nodes=32)
    assert ei.value.code == ERR_FULL


def test_argument_errors():
    from paper_1906_06504_gb300.heap import GHeapError
    with pytest.raises(GHeapError):
        Knapsack(0)
    with pytest.raises(GHeapError):
        Knapsack(5000)
    with Knapsack(4, k=8, batch=8) as ctx:
        with pytest.raises(GHeapError):           # more items than the context holds
            ctx.run(dev(np.ones(5)), dev(np.ones(5)), 3)
        big = np.array([0xFFFFFFF0, 0xFFFFFFF0], np.uint32)
        with pytest.raises(GHeapError):           # values sum past 32 bits
            ctx.run(dev([1, 1]), dev(big), 1)


@pytest.mark.parametrize("n", [100, 200])
def test_full_size_strongly_correlated(n):
    """Strongly correlated instances: w ~ U[1, 1000], v = w + 100,
    capacity = half the total weight."""
    w, v, cap = inputs.knapsack_instance(n, inputs.config_seed(4))
    st = solve(w, v, cap, k=1024, batch=16384)
    assert st["best"] == oracle.knapsack_dp(w, v, cap)
