"""Parity of the CUDA heap (through the C ABI) with the CPU oracle.

* single thread block: the GPU runs the same sequence of steps as the
  sequential model, so every node, the partial buffer and every output must
  match it bit for bit after every call;
* many thread blocks: every DEL output must equal the oracle's replay of the
  recorded root-lock order (linearizability, Section 3.3.3 Theorem 1), the
  multiset must be conserved and Properties 1-3 must hold when quiescent;
* the full-size workload in the benchmark's launch shape.
"""
import numpy as np
import pytest

import oracle
from oracle.genheap import GeneralizedHeapModel
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


from heaputil import (Recorder, check_properties, mixed_ops, model_matches,  # noqa: E402
                      np_dtype, to_dev, to_host)


def GHeap(*a, **kw):
    from paper_1906_06504_gb300.heap import GHeap as G
    return G(*a, **kw)


def special_keys(rng, n, key_bytes, dup=False):
    dt = np_dtype(key_bytes)
    hi = np.iinfo(dt).max
    if dup:
        x = rng.integers(0, 6, n).astype(dt)
        x[x == 5] = hi
        return x
    x = rng.integers(0, hi, n, dtype=dt, endpoint=True)
    x[rng.integers(0, n, max(1, n // 50))] = hi
    x[rng.integers(0, n, max(1, n // 50))] = 0
    return x


# ---------------------------------------------------------------------------
# one thread block: node-level parity with the sequential model
# ---------------------------------------------------------------------------

def test_config1_single_cta_k64():
    """2^16 uniform keys, k=64, one block: insert all in batches of 64, then
    deleteMin all in batches of 64; output = sorted input; the heap after the
    inserts equals the sequential model node for node."""
    n, k = 1 << 16, 64
    keys = inputs.keys_u32(inputs.config_seed(1), n)
    with GHeap(capacity=n, k=k, log_capacity=4 * n // k) as h:
        h.set_launch(ctas=1)
        r = Recorder(h)
        r.insert(keys)
        h.sync()
        model = GeneralizedHeapModel(k)
        for i in range(0, n, k):
            model.insert(keys[i:i + k])
        model_matches(h, model)
        check_properties(h)
        rec = r.delete_min(n)
        h.sync()
        out = to_host(rec["out"], 4)
        assert int(rec["cnt"].item()) == n
        assert np.array_equal(out, oracle.replay([("ins", keys), ("del", n)])[0])
        assert r.replay_and_compare() == n // k
        assert h.size() == 0


@pytest.mark.parametrize("k,key_bytes", [(1, 4), (4, 4), (8, 8), (64, 4), (256, 8), (1024, 4),
                                         (2048, 4)])
def test_single_cta_random_calls_match_model(k, key_bytes):
    """Random insert/deleteMin calls with partial sizes, one block: outputs,
    nodes and the partial buffer equal the sequential model after every call."""
    rng = np.random.default_rng(1000 + k + key_bytes)
    cap = 40 * k + 7
    with GHeap(capacity=cap, k=k, key_bytes=key_bytes, log_capacity=4096) as h:
        h.set_launch(ctas=1, items_per_thread=16 if k >= 2048 else 4)
        model = GeneralizedHeapModel(k, dtype=np_dtype(key_bytes))
        r = Recorder(h)
        size = 0
        for step in range(40 if k < 1024 else 16):
            if rng.random() < 0.55 and size < cap - 3 * k:
                n = int(rng.integers(1, 3 * k + 2))
                keys = special_keys(rng, n, key_bytes, dup=(step % 3 == 0))
                r.insert(keys)
                for i in range(0, n, k):
                    model.insert(keys[i:i + k])
                size += n
            else:
                n = int(rng.integers(1, 3 * k + 2))
                rec = r.delete_min(n)
                h.sync()
                got = to_host(rec["out"], key_bytes)[:int(rec["cnt"].item())]
                want = []
                left = n
                while left > 0 and model.size() > 0:
                    part = model.delete(min(k, left))
                    want.append(part)
                    left -= part.size
                want = np.concatenate(want) if want else np.empty(0, np_dtype(key_bytes))
                assert np.array_equal(got, want)
                size -= want.size
            h.sync()
            model_matches(h, model)
        r.replay_and_compare()


# ---------------------------------------------------------------------------
# many thread blocks: linearizability replay
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dist", ["uniform", "ascending", "descending"])
def test_concurrent_phased(dist):
    """Insert-all then deleteMin-all with every block of the device busy; the
    output is the sorted input (the three distributions hold one multiset)."""
    n, k = (1 << 20) + 333, 1024
    keys = inputs.keys_u32(inputs.config_seed(2), n, dist)
    with GHeap(capacity=n, k=k, log_capacity=2 * (n // k + 2), stats=True) as h:
        r = Recorder(h)
        r.insert(keys)
        h.sync()
        check_properties(h)
        assert h.size() == n
        rec = r.delete_min(n)
        h.sync()
        out = to_host(rec["out"], 4)
        assert int(rec["cnt"].item()) == n
        assert np.array_equal(out, np.sort(keys))
        r.replay_and_compare()


def test_ascending_input_never_merges():
    """Ascending keys, one block: every insert finds smaller keys on its whole
    path and only places its batch at the target, with no MergeAndSort
    (Section 5.2); deleteMin-all still returns the input."""
    n, k = 1 << 14, 64
    keys = inputs.keys_u32(inputs.config_seed(1), n, "ascending")
    with GHeap(capacity=n, k=k, stats=True) as h:
        h.set_launch(ctas=1)
        h.insert(to_dev(keys))
        st = h.stats()
        assert st["merges"] == 0 and st["ins_ops"] == n // k, st
        out, cnt = h.delete_min(n)
        h.sync()
        assert np.array_equal(to_host(out, 4), keys)


@pytest.mark.parametrize("yields", [64, 0])
@pytest.mark.parametrize("k,key_bytes,partial", [(1024, 4, False), (1024, 4, True),
                                                  (2048, 4, True), (64, 8, True), (8, 4, True)])
def test_concurrent_mixed_replay(k, key_bytes, partial, yields):
    """A prefilled heap under alternating INS/DEL ops from all blocks (the
    ins-del pairs of Section 5.5); every DEL equals the oracle's replay.
    yields = 0 is the paper's INS/DEL cooperation (Section 3.3.2): a DEL
    whose last node is an in-flight INS target marks it and waits for the
    keys, which the counters must show happened."""
    rng = np.random.default_rng(7 + k)
    prefill = special_keys(rng, 64 * k + 5, key_bytes)
    n_pairs = 512 if k >= 1024 else 2048
    ops, keys, out_size = mixed_ops(rng, n_pairs, k, key_bytes, partial=partial)
    cap = prefill.size + keys.size + k
    with GHeap(capacity=cap, k=k, key_bytes=key_bytes, log_capacity=4 * n_pairs + 4096,
               stats=True) as h:
        h.set_yields(yields)
        r = Recorder(h)
        r.insert(prefill)
        r.ops(ops, keys, out_size)
        assert r.replay_and_compare() >= n_pairs
        check_properties(h)
        st = h.stats()
        if yields == 0:
            assert st["deliveries"] > 0 and st["del_yields"] == 0, st


def test_concurrent_drain_from_empty_mixed():
    """DELs that start before any INS (empty heap, partial buffer only)."""
    rng = np.random.default_rng(99)
    k = 16
    ops, keys, out_size = mixed_ops(rng, 3000, k, 4, partial=True, del_first=True)
    with GHeap(capacity=keys.size + k, k=k, log_capacity=8000) as h:
        r = Recorder(h)
        r.ops(ops, keys, out_size)
        r.replay_and_compare()
        check_properties(h)


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def test_edge_cases():
    k = 64
    with GHeap(capacity=1000, k=k, log_capacity=256) as h:
        r = Recorder(h)
        rec = r.delete_min(10)                 # empty heap: count 0
        h.sync()
        assert int(rec["cnt"].item()) == 0
        r.insert(np.array([], np.uint32))      # n = 0 is a no-op
        r.insert(np.array([0xFFFFFFFF, 0, 0xFFFFFFFF, 5], np.uint32))
        rec = r.delete_min(100)                # more than present
        h.sync()
        assert int(rec["cnt"].item()) == 4
        assert list(to_host(rec["out"], 4)[:4]) == [0, 5, 0xFFFFFFFF, 0xFFFFFFFF]
        r.insert(np.full(999, 7, np.uint32))   # duplicates up to capacity - 1
        from paper_1906_06504_gb300.heap import GHeapError
        with pytest.raises(GHeapError) as e:
            h.insert(to_dev(np.arange(2, dtype=np.uint32)))
        assert e.value.code == -3              # FULL, nothing enqueued
        assert h.size() == 999
        r.insert(np.array([3], np.uint32))     # exactly at capacity
        rec = r.delete_min(1000)
        h.sync()
        out = to_host(rec["out"], 4)
        assert out[0] == 3 and np.all(out[1:] == 7)
        r.replay_and_compare()


def test_bounded_wait_reports_timeout():
    """A root lock that nothing releases: the op's wait runs out after the
    configured bound and the call reports GHEAP_ERR_TIMEOUT; the device stays
    usable (the next heap works)."""
    with GHeap(capacity=4096, k=64) as h:
        h.set_timeout(50_000_000)               # 50 ms
        h.debug_hold_root()
        h.insert(to_dev(np.arange(256, dtype=np.uint32)))
        assert h.sync_code() == -4
        from paper_1906_06504_gb300.heap import GHeapError
        with pytest.raises(GHeapError):
            h.insert(to_dev(np.arange(4, dtype=np.uint32)))
        h.reset()
        h.insert(to_dev(np.arange(256, dtype=np.uint32)))
        out, cnt = h.delete_min(256)
        h.sync()
        assert np.array_equal(to_host(out, 4), np.arange(256, dtype=np.uint32))


# ---------------------------------------------------------------------------
# full size, in the benchmark's launch shape
# ---------------------------------------------------------------------------

def test_full_size_phased_2p26_k1024():
    """2^26 uniform u32 keys, k = 1024, all blocks: deleteMin-all returns the
    sorted input (the property fixes every output of a phased run)."""
    n, k = 1 << 26, 1024
    keys = inputs.keys_u32(inputs.config_seed(2), n)
    with GHeap(capacity=n, k=k) as h:
        h.insert(to_dev(keys))
        out, cnt = h.delete_min(n)
        h.sync()
        assert int(cnt.item()) == n
        got = to_host(out, 4)
        assert np.array_equal(got, np.sort(keys))
        assert h.size() == 0
