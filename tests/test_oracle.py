"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each test checks an oracle function against brute force, an independent
textbook routine, a closed form, a published vector or a hand-worked example
(tests/golden), chosen so that a dropped term, a wrong index or a swapped
operand in the oracle fails at least one of them.  CPU only.
"""
import heapq
import itertools
import os

import numpy as np
import pytest

import oracle
from oracle.genheap import GeneralizedHeapModel, node_of, bitrev
from paper_1906_06504_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# input generator: published splitmix64 vectors
# --------------------------------------------------------------------------

def test_splitmix64_published_vectors():
    lines = [l.split() for l in open(os.path.join(GOLDEN,
             "splitmix64_seed1234567.txt")) if l.strip() and l[0] != "#"]
    seed = int(lines[0][1])
    want = np.array([int(l[0]) for l in lines[1:]], dtype=np.uint64)
    assert np.array_equal(inputs.splitmix64(seed, want.size), want)
    # counter-based: a window of the stream equals the same outputs
    assert np.array_equal(inputs.splitmix64(seed, 3, start=2), want[2:5])


def test_key_distributions_share_multiset():
    u = inputs.keys_u32(7, 5000, "uniform")
    a = inputs.keys_u32(7, 5000, "ascending")
    d = inputs.keys_u32(7, 5000, "descending")
    assert np.array_equal(np.sort(u), a)
    assert np.array_equal(a[::-1], d)
    assert np.all(np.diff(a.astype(np.int64)) >= 0)


# --------------------------------------------------------------------------
# binary-heap priority queue (Section 2.1) against brute force and heapq
# --------------------------------------------------------------------------

def _random_ops(rng, n_ops, maxn, keymax):
    ops = []
    for _ in range(n_ops):
        if rng.random() < 0.55:
            ops.append(("ins", rng.integers(0, keymax, rng.integers(0, maxn + 1),
                                            dtype=np.uint64).astype(np.uint32)))
        else:
            ops.append(("del", int(rng.integers(0, maxn + 1))))
    return ops


@pytest.mark.parametrize("seed", range(6))
def test_pq_replay_equals_bruteforce_sort(seed):
    rng = np.random.default_rng(seed)
    keymax = [4, 1000, 2**32][seed % 3]     # heavy duplicates .. full range
    ops = _random_ops(rng, 200, 40, keymax)
    got = oracle.replay(ops)
    multiset = []
    want = []
    for kind, arg in ops:
        if kind == "ins":
            multiset.extend(int(x) for x in arg)
        else:
            multiset.sort()
            want.append(multiset[:arg])
            multiset = multiset[arg:]
    assert len(got) == len(want)
    for g, w in zip(got, want):
        assert [int(x) for x in g] == w


def test_pq_matches_heapq_u64_extremes():
    rng = np.random.default_rng(11)
    keys = rng.integers(0, 2**64 - 1, 3000, dtype=np.uint64, endpoint=True)
    keys[:5] = [0, 2**64 - 1, 2**64 - 1, 0, 2**63]
    q = oracle.BinaryHeapPQ(4)            # forces growth
    h = []
    for i in range(0, 3000, 300):
        q.push(keys[i:i + 300])
        for x in keys[i:i + 300]:
            heapq.heappush(h, int(x))
        out = q.pop(137)
        ref = [heapq.heappop(h) for _ in range(137)]
        assert [int(x) for x in out] == ref
    assert len(q) == len(h)
    assert q.pop(10**6).size == len(h)
    assert len(q) == 0
    assert q.pop(5).size == 0             # delete from empty: count 0


def test_pq_phased_output_is_sorted_input():
    keys = inputs.keys_u32(inputs.config_seed(1), 1 << 16)
    out = oracle.replay([("ins", keys), ("del", 1 << 16)])[0]
    assert np.array_equal(out, np.sort(keys))


# --------------------------------------------------------------------------
# MergeAndSort by definition (Section 3.2.1)
# --------------------------------------------------------------------------

def test_merge_and_sort_worked_example():
    # a = [1,4,9,12], b = [2,3,10,11]: the union sorted is
    # [1,2,3,4,9,10,11,12]; the 4 smallest stay ("hi" in the paper).
    s, l = oracle.merge_and_sort([1, 4, 9, 12], [2, 3, 10, 11])
    assert list(s) == [1, 2, 3, 4] and list(l) == [9, 10, 11, 12]


@pytest.mark.parametrize("k", [1, 2, 7, 64, 1024])
def test_merge_and_sort_postconditions(k):
    rng = np.random.default_rng(k)
    for keymax in (3, 2**32):
        a = np.sort(rng.integers(0, keymax, k, dtype=np.uint64))
        b = np.sort(rng.integers(0, keymax, k, dtype=np.uint64))
        s, l = oracle.merge_and_sort(a, b)
        assert s.size == k and l.size == k
        assert np.all(np.diff(s.astype(np.float64)) >= 0)
        assert np.all(np.diff(l.astype(np.float64)) >= 0)
        assert s[-1] <= l[0]
        assert sorted(np.concatenate([s, l]).tolist()) == \
            sorted(np.concatenate([a, b]).tolist())


def test_merge_and_sort_uneven_split():
    s, l = oracle.merge_and_sort([5, 6], [1, 2, 3], k_small=4)
    assert list(s) == [1, 2, 3, 5] and list(l) == [6]


# --------------------------------------------------------------------------
# Properties 1-3 checker (Section 3.1): accepts valid heaps, catches plants
# --------------------------------------------------------------------------

def _valid_snapshot(k=4):
    m = GeneralizedHeapModel(k)
    rng = np.random.default_rng(5)
    for _ in range(12):
        m.insert(rng.integers(0, 1000, k, dtype=np.uint64).astype(np.uint32))
    m.insert(np.array([999, 998], dtype=np.uint32))
    return m.snapshot()


def test_properties_accept_valid():
    nodes, present, buf = _valid_snapshot()
    assert oracle.check_properties(nodes, present, 4, buf) == (0, 0)


def test_properties_catch_planted_violations():
    nodes, present, buf = _valid_snapshot()
    n2 = nodes.copy(); n2[3] = n2[3][::-1]    # a node out of order
    assert n2[3, 0] != n2[3, -1]
    assert oracle.check_properties(n2, present, 4, buf) == (2, 3)
    n1 = nodes.copy(); n1[2, :] = 0          # child below its parent's max
    assert oracle.check_properties(n1, present, 4, buf) == (1, 2)
    b3 = buf.copy(); b3[0] = 0               # buffer below the root max
    assert oracle.check_properties(nodes, present, 4, b3)[0] == 3
    b3 = buf.copy()[::-1].copy()             # buffer out of order
    if b3.size > 1 and b3[0] != b3[-1]:
        assert oracle.check_properties(nodes, present, 4, b3)[0] == 3
    p4 = present.copy(); p4[2] = False       # orphaned children of node 2
    assert oracle.check_properties(nodes, p4, 4, buf)[0] == 4
    big = np.arange(4, dtype=np.uint64) + 10**6
    assert oracle.check_properties(nodes, present, 4, big)[0] == 4


# --------------------------------------------------------------------------
# sequential generalized heap model: hand-worked example, brute force, k=1
# --------------------------------------------------------------------------

def _parse_state(line):
    st = {}
    for tok in line.split()[1:]:
        name, _, val = tok.partition("=")
        st[name] = [int(x) for x in val.split(",")] if val else []
    return st


def test_genheap_hand_worked_k2():
    m = GeneralizedHeapModel(2)
    for line in open(os.path.join(GOLDEN, "genheap_k2_worked.txt")):
        line = line.strip()
        if not line or line[0] == "#":
            continue
        if line.startswith("ins"):
            m.insert(np.array([int(x) for x in line.split()[1:]], np.uint32))
        elif line.startswith("del"):
            lhs, _, rhs = line.partition("->")
            out = m.delete(int(lhs.split()[1]))
            assert [int(x) for x in out] == [int(x) for x in rhs.split()]
        elif line.startswith("state"):
            st = _parse_state(line)
            have = {("root" if i == 1 else "n%d" % i): [int(x) for x in v]
                    for i, v in m.nodes.items()}
            have["buf"] = [int(x) for x in m.buf]
            assert have == st, line


@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_genheap_equals_bruteforce_and_keeps_properties(k):
    rng = np.random.default_rng(100 + k)
    m = GeneralizedHeapModel(k)
    multiset = []
    for step in range(400):
        if rng.random() < 0.55:
            n = int(rng.integers(1, k + 1))
            keys = rng.integers(0, 50, n, dtype=np.uint64).astype(np.uint32)
            m.insert(keys)
            multiset.extend(int(x) for x in keys)
        else:
            n = int(rng.integers(1, k + 1))
            out = m.delete(n)
            multiset.sort()
            assert [int(x) for x in out] == multiset[:n]
            multiset = multiset[n:]
        assert m.size() == len(multiset)
        nodes, present, buf = m.snapshot()
        assert oracle.check_properties(nodes, present, k, buf) == (0, 0)


def test_genheap_k1_reduces_to_conventional_heap():
    # k = 1: no partial buffer is ever used and every DEL returns the single
    # minimum, exactly as the textbook heap (Section 3.1, remark after P3).
    rng = np.random.default_rng(3)
    m = GeneralizedHeapModel(1)
    h = []
    for _ in range(2000):
        if rng.random() < 0.6:
            x = int(rng.integers(0, 2**32))
            m.insert(np.array([x], np.uint32))
            heapq.heappush(h, x)
        elif h:
            assert [int(v) for v in m.delete(1)] == [heapq.heappop(h)]
        assert m.buf.size == 0


def test_bitreversal_targets():
    # j-th node at level d: 2^d + rev_d(j - 2^d); level 2 fills 4, 6, 5, 7
    assert [node_of(j) for j in range(1, 8)] == [1, 2, 3, 4, 6, 5, 7]
    assert bitrev(0b0011, 4) == 0b1100
    # consecutive targets on one level share no node below the root
    for j in range(8, 63):
        a, b = node_of(j), node_of(j + 1)
        if a.bit_length() == b.bit_length():
            assert (a >> (a.bit_length() - 2)) != (b >> (b.bit_length() - 2))
    # the map is a permutation of each level
    for d in range(1, 10):
        lvl = {node_of(j) for j in range(1 << d, 1 << (d + 1))}
        assert lvl == set(range(1 << d, 1 << (d + 1)))


# --------------------------------------------------------------------------
# Dijkstra: closed form on uniform grids, brute force on small graphs
# --------------------------------------------------------------------------

def test_dijkstra_grid_closed_form():
    side = 33
    rowptr, col, w = inputs.grid_graph(side, 1, wlo=7, whi=7)
    d = oracle.dijkstra(rowptr, col, w, src=0)
    r, c = np.divmod(np.arange(side * side), side)
    assert np.array_equal(d.astype(np.int64), 7 * (r + c))


def _bellman_ford(n, rowptr, col, w, src):
    INF = 2**32 - 1
    d = [INF] * n
    d[src] = 0
    for _ in range(n):
        changed = False
        for u in range(n):
            if d[u] == INF:
                continue
            for e in range(int(rowptr[u]), int(rowptr[u + 1])):
                nd = d[u] + int(w[e])
                if nd < d[int(col[e])]:
                    d[int(col[e])] = nd
                    changed = True
        if not changed:
            break
    return d


@pytest.mark.parametrize("seed", range(4))
def test_dijkstra_bruteforce_rmat(seed):
    rowptr, col, w = inputs.rmat_graph(7, 3, seed)
    d = oracle.dijkstra(rowptr, col, w, src=0)
    ref = _bellman_ford(rowptr.size - 1, rowptr, col, w, 0)
    assert [int(x) for x in d] == ref
    assert int(d[0]) == 0


# --------------------------------------------------------------------------
# knapsack DP: brute-force enumeration, closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_knapsack_dp_bruteforce(seed):
    w, v, cap = inputs.knapsack_instance(12, seed)
    best = 0
    for mask in range(1 << 12):
        sel = [(mask >> i) & 1 for i in range(12)]
        tw = sum(int(w[i]) for i in range(12) if sel[i])
        if tw <= cap:
            best = max(best, sum(int(v[i]) for i in range(12) if sel[i]))
    assert oracle.knapsack_dp(w, v, cap) == best


def test_knapsack_dp_closed_forms():
    w = np.array([3, 5, 9], np.uint32)
    v = np.array([4, 6, 1], np.uint32)
    assert oracle.knapsack_dp(w, v, 100) == 11      # everything fits
    assert oracle.knapsack_dp(w, v, 0) == 0         # nothing fits
    assert oracle.knapsack_dp(w, v, 2) == 0
    assert oracle.knapsack_dp(w, v, 8) == 10


def test_stl_baseline_sorts_and_reports_its_time():
    """The std::priority_queue baseline of the paper's Table 1 (timed beside
    the GPU heap, not used by any check): its push-all/pop-all output is the
    sorted input, on duplicates and the u32 extremes too."""
    rng = np.random.default_rng(17)
    for n in (1, 2, 1000, 65537):
        keys = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
        keys[:: max(1, n // 7)] = 0xFFFFFFFF
        keys[1:: max(1, n // 5)] = 0
        out, dt = oracle.stl_insert_delete(keys)
        assert np.array_equal(out, np.sort(keys)) and dt >= 0.0
