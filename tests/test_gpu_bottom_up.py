"""Bottom-up inserts (BU-INS, Sections 3.2.2 and 3.3.4) against the oracle,
through the C ABI (GHEAP_FLAG_BOTTOM_UP).

Inserts of a bottom-up heap place their batch at the target node and rise.
Internal node contents differ from top-down insertion, so parity is checked
on what the method fixes: every DEL output equals the oracle's replay of the
recorded linearization order (an insert is numbered under its last lock), the
multiset is conserved, Properties 1-3 hold at quiescence, phased runs return
the sorted input, and an insert whose batch is above its parent stops at once
(early stop: ascending input never merges).
"""
import numpy as np
import pytest

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


from heaputil import Recorder, check_properties, mixed_ops, np_dtype, to_dev, to_host  # noqa: E402


def GHeap(*a, **kw):
    from paper_1906_06504_gb300.heap import GHeap as G
    return G(*a, bottom_up=True, **kw)


@pytest.mark.parametrize("k,key_bytes", [(1, 4), (8, 4), (64, 8), (256, 4), (1024, 4), (2048, 8)])
def test_single_block_calls_replay(k, key_bytes):
    """One block, random insert/delete calls of any size: every deleteMin
    equals the oracle, the properties hold after every call."""
    rng = np.random.default_rng(500 + k + key_bytes)
    dt = np_dtype(key_bytes)
    cap = 40 * k + 64
    with GHeap(capacity=cap, k=k, key_bytes=key_bytes, log_capacity=1 << 14) as h:
        h.set_launch(ctas=1, items_per_thread=16 if k >= 2048 else 4)
        r = Recorder(h)
        size = 0
        for step in range(60):
            if rng.random() < 0.6 and size + 4 * k < cap:
                n = int(rng.integers(1, 4 * k + 1))
                keys = rng.integers(0, np.iinfo(dt).max, n, dtype=dt, endpoint=True)
                if step % 7 == 0:
                    keys[: n // 2] = 0
                r.insert(keys)
                size += n
            else:
                n = int(rng.integers(1, 3 * k + 1))
                r.delete_min(n)
                size = max(0, size - n)
            if step % 10 == 9:
                check_properties(h)
        assert r.replay_and_compare() > 0
        check_properties(h)


@pytest.mark.parametrize("dist", ["uniform", "ascending", "descending"])
def test_concurrent_phased(dist):
    """Insert-all bottom-up from every block, then deleteMin-all: the output
    is the sorted input; the record replays exactly."""
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
        assert int(rec["cnt"].item()) == n
        assert np.array_equal(to_host(rec["out"], 4), np.sort(keys))
        r.replay_and_compare()


def test_ascending_input_stops_at_once():
    """Each ascending batch is above everything already in the heap: a
    bottom-up insert compares with its parent once and stops (no merge)."""
    n, k = 1 << 16, 256
    keys = inputs.keys_u32(inputs.config_seed(1), n, "ascending")
    with GHeap(capacity=n, k=k, stats=True) as h:
        h.set_launch(ctas=1)              # batches arrive in input order
        h.insert(to_dev(keys))
        st = h.stats()
        assert st["merges"] == 0, st
        # one parent comparison per batch below the root
        assert st["ins_levels"] == n // k - 1, st
        out, cnt = h.delete_min(n)
        h.sync()
        assert np.array_equal(to_host(out, 4), keys)


def test_descending_input_rises_to_the_root():
    """Each descending batch is below everything: it rises to the root."""
    n, k = 1 << 14, 64
    keys = inputs.keys_u32(inputs.config_seed(1), n, "descending")
    with GHeap(capacity=n, k=k, stats=True) as h:
        h.set_launch(ctas=1)
        h.insert(to_dev(keys))
        st = h.stats()
        # batch j (j >= 2) sits at level floor(log2 j) and merges with every
        # ancestor up to the root
        want = sum(int(np.floor(np.log2(j))) for j in range(2, n // k + 1))
        assert st["merges"] == want, (st["merges"], want)
        out, cnt = h.delete_min(n)
        h.sync()
        assert np.array_equal(to_host(out, 4), np.sort(keys))


@pytest.mark.parametrize("k,key_bytes", [(1024, 4), (64, 8)])
def test_inserts_between_delete_launches_replay(k, key_bytes):
    """Alternating insert and deleteMin launches (bottom-up inserts, top-down
    deletes), all blocks busy: every DEL replays exactly."""
    rng = np.random.default_rng(77 + k)
    dt = np_dtype(key_bytes)
    with GHeap(capacity=600 * k, k=k, key_bytes=key_bytes, log_capacity=1 << 16) as h:
        r = Recorder(h)
        for step in range(12):
            n = int(rng.integers(20 * k, 40 * k))
            r.insert(rng.integers(0, np.iinfo(dt).max, n, dtype=dt, endpoint=True))
            r.delete_min(int(rng.integers(5 * k, 25 * k)) + int(rng.integers(0, k)))
        assert r.replay_and_compare() > 0
        check_properties(h)


def test_mixed_op_lists_insert_top_down():
    """A mixed INS/DEL list on a bottom-up heap inserts top-down and replays
    exactly (bottom-up inserts are for insert launches)."""
    rng = np.random.default_rng(3)
    k = 256
    ops, keys, out_size = mixed_ops(rng, 1024, k, 4, partial=True)
    with GHeap(capacity=keys.size + 64 * k, k=k, log_capacity=8192) as h:
        r = Recorder(h)
        r.insert(rng.integers(0, 2 ** 32, 32 * k, dtype=np.uint32))
        r.ops(ops, keys, out_size)
        assert r.replay_and_compare() > 0
        check_properties(h)


def test_full_size_phased_2p26_k1024():
    n, k = 1 << 26, 1024
    keys = inputs.keys_u32(inputs.config_seed(2), n)
    d = to_dev(keys)
    with GHeap(capacity=n, k=k) as h:
        h.insert(d)
        out, cnt = h.delete_min(n)
        h.sync()
        assert int(cnt.item()) == n
        got = to_host(out, 4)
    assert np.array_equal(got, np.sort(keys))
