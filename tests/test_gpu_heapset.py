"""Parity of heap sets (many heaps, one persistent launch) with the CPU oracle.

Every heap of a set keeps its own linearization record; replaying each one
through the oracle must reproduce every DEL output of that heap bit for bit,
whatever the other heaps did in the same launch.
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


from heaputil import check_properties, np_dtype, to_dev, to_host  # noqa: E402

OP_INS, OP_DEL = 1, 2


def GHeapSet(*a, **kw):
    from paper_1906_06504_gb300.heap import GHeapSet as G
    return G(*a, **kw)


BU = [pytest.param(False, id="top-down"), pytest.param(True, id="bottom-up")]


class SetRun:
    """Launches op lists on a set and replays each heap's record."""

    def __init__(self, hs):
        self.hs = hs
        self.launches = {}
        self.next_id = 1
        self.kb = hs.key_bytes

    def launch(self, ops, in_keys, out_size):
        dt = np_dtype(self.kb)
        ops = np.ascontiguousarray(ops)
        in_keys = np.ascontiguousarray(in_keys, dtype=dt)
        ops_dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
        out = torch.zeros(max(out_size, 1), dtype=torch.int32 if self.kb == 4 else torch.int64,
                          device="cuda")
        counts = torch.zeros(len(ops), dtype=torch.int32, device="cuda")
        self.hs.ops(ops_dev, to_dev(in_keys) if in_keys.size else None, out, counts)
        self.launches[self.next_id] = (ops, in_keys, out, counts)
        self.next_id += 1
        return out, counts

    def replay(self):
        self.hs.sync()
        dt = np_dtype(self.kb)
        host = {cid: (to_host(o, self.kb), c.cpu().numpy())
                for cid, (_, _, o, c) in self.launches.items()}
        checked = 0
        for hid, h in enumerate(self.hs.heaps):
            log, total = h.log()
            assert log.size == total
            q = oracle.BinaryHeapPQ()
            try:
                for e in log:
                    ops, ins, _, _ = self.launches[int(e["call_id"])]
                    ref = int(e["ref"])
                    kind = int(e["kind_n"]) >> 24
                    n = int(e["kind_n"]) & 0xFFFFFF
                    op = ops[ref]
                    assert int(op["heap"]) == hid
                    assert (int(op["kind_n"]) >> 24) == kind
                    off = int(op["offset"])
                    want_n = int(op["kind_n"]) & 0xFFFFFF
                    if kind == OP_INS:
                        assert n == want_n
                        q.push(ins[off:off + n])
                    else:
                        out, cnt = host[int(e["call_id"])]
                        assert n == min(want_n, len(q)) == int(cnt[ref])
                        want = q.pop(n, dtype=dt)
                        assert np.array_equal(out[off:off + n], want), (hid, ref)
                        checked += 1
                assert len(q) == h.size()
            finally:
                q.close()
        return checked


def random_set_ops(rng, n_heaps, k, n_ops, key_bytes, prefill=0):
    dt = np_dtype(key_bytes)
    heap = rng.integers(0, n_heaps, n_ops)
    kind = np.where(rng.random(n_ops) < 0.55, OP_INS, OP_DEL)
    n = rng.integers(1, k + 1, n_ops)
    n[:prefill] = k
    kind[:prefill] = OP_INS
    ops = np.zeros(n_ops, dtype=[("heap", "<u4"), ("kind_n", "<u4"), ("offset", "<u8")])
    ops["heap"] = heap
    ops["kind_n"] = (kind.astype(np.int64) << 24) | n
    ins = kind == OP_INS
    in_off = np.zeros(n_ops, dtype=np.int64)
    in_off[ins] = np.concatenate([[0], np.cumsum(n[ins])[:-1]])
    out_off = np.zeros(n_ops, dtype=np.int64)
    out_off[~ins] = np.concatenate([[0], np.cumsum(n[~ins])[:-1]]) if (~ins).any() else []
    ops["offset"] = np.where(ins, in_off, out_off)
    keys = rng.integers(0, np.iinfo(dt).max, int(n[ins].sum()), dtype=dt, endpoint=True)
    return ops, keys, int(n[~ins].sum())


@pytest.mark.parametrize("bottom_up", BU)
@pytest.mark.parametrize("k,key_bytes", [(64, 4), (1024, 4), (2048, 4), (256, 8)])
def test_heapset_random_ops_replay(k, key_bytes, bottom_up):
    """Mixed lists: a bottom-up set must detect the DELs and insert top-down."""
    rng = np.random.default_rng(31 + k + key_bytes)
    n_heaps = 12
    caps = [int(c) for c in rng.integers(200 * k, 300 * k, n_heaps)]
    n_ops = 3000 if k <= 256 else 1200
    with GHeapSet(caps, k=k, key_bytes=key_bytes, log_capacity=n_ops + 64,
                  bottom_up=bottom_up) as hs:
        run = SetRun(hs)
        ops, keys, out_size = random_set_ops(rng, n_heaps, k, n_ops, key_bytes, prefill=n_heaps * 4)
        run.launch(ops, keys, out_size)
        # a second launch on the same heaps continues from their state
        ops2, keys2, out2 = random_set_ops(rng, n_heaps, k, n_ops // 2, key_bytes)
        run.launch(ops2, keys2, out2)
        assert run.replay() > 0
        for h in hs.heaps:
            check_properties(h)


@pytest.mark.parametrize("bottom_up", BU)
def test_heapset_phased_loguniform_sizes(bottom_up):
    """Insert-all then delete-all on 48 heaps with log-uniform sizes; in each
    heap's root order the DEL outputs concatenate to its sorted input.  A
    bottom-up set inserts bottom-up here (the insert list has no DEL)."""
    k = 256
    sizes = inputs.loguniform_sizes(inputs.config_seed(5), 48, 8, 15)
    total = int(sizes.sum())
    keys = inputs.keys_u32(inputs.config_seed(5), total)
    with GHeapSet([int(s) for s in sizes], k=k, log_capacity=int(-(-sizes.max() // k)) * 2 + 8,
                  bottom_up=bottom_up) as hs:
        run = SetRun(hs)
        run.launch(inputs.set_phase_ops(sizes, k, OP_INS), keys, 0)
        hs.sync()
        for h in hs.heaps:
            check_properties(h)
        dops = inputs.set_phase_ops(sizes, k, OP_DEL)
        out, counts = run.launch(dops, np.empty(0, np.uint32), total)
        run.replay()
        hs.sync()
        got = to_host(out, 4)
        base = np.concatenate([[0], np.cumsum(sizes)[:-1]])
        for hid in range(sizes.size):
            seg = got[base[hid]:base[hid] + sizes[hid]]
            # the ops of one heap may take the root in any order, so check the
            # multiset and that each batch is ascending
            mine = keys[base[hid]:base[hid] + sizes[hid]]
            assert np.array_equal(np.sort(seg), np.sort(mine))
            assert hs.heaps[hid].size() == 0


@pytest.mark.parametrize("bottom_up", BU)
def test_heapset_graph_replay_matches_direct(bottom_up):
    """A captured launch replayed twice (with a reset between) gives the same
    per-heap contents as the direct launch."""
    k = 128
    sizes = np.array([1000, 5000, 128, 70, 20000, 3333])
    keys = inputs.keys_u32(77, int(sizes.sum()))
    ins = inputs.set_phase_ops(sizes, k, OP_INS)
    with GHeapSet([int(s) for s in sizes], k=k, bottom_up=bottom_up) as hs:
        ops_dev = torch.from_numpy(ins.view(np.uint8).copy()).cuda()
        kd = to_dev(keys)
        g = hs.graph(ops_dev, kd, None)
        snaps = []
        for _ in range(2):
            hs.reset()
            g.launch()
            hs.sync()
            snaps.append([h.snapshot() for h in hs.heaps])
        g.close()
        hs.reset()
        hs.ops(ops_dev, kd, None)
        hs.sync()
        direct = [h.snapshot() for h in hs.heaps]
        for s0, s1, d in zip(snaps[0], snaps[1], direct):
            # same multiset per heap and same node count, whatever the order
            for s in (s0, s1):
                assert s[3][:2] == d[3][:2]
                m = d[3][0]
                a = np.sort(np.concatenate([s[0][1:m + 1].ravel(), s[2][:s[3][1]]]))
                b = np.sort(np.concatenate([d[0][1:m + 1].ravel(), d[2][:d[3][1]]]))
                assert np.array_equal(a, b)


@pytest.mark.parametrize("k,key_bytes", [(1024, 4), (2048, 4), (256, 8)])
def test_heapset_delete_only_launch(k, key_bytes):
    """A list with no input keys runs the delete-only walk (the root step's
    fetches included, on heaps of 16 nodes and more): after a prefill, random
    DELs of 1..k keys over heaps of uneven sizes, more than some heaps hold;
    every DEL equals the replay of its heap's record, the per-op counts
    included, and the heaps keep Properties 1-3.  An INS in a list with no
    input keys is its heap's sticky error; the other heaps go on."""
    rng = np.random.default_rng(900 + k + key_bytes)
    dt = np_dtype(key_bytes)
    sizes = np.array([60 * k + 17, 5 * k, 300 * k + 3, 33, 40 * k, 128 * k])
    keys = rng.integers(0, np.iinfo(dt).max, int(sizes.sum()), dtype=dt, endpoint=True)
    with GHeapSet([int(c) for c in sizes], k=k, key_bytes=key_bytes, log_capacity=2048) as hs:
        run = SetRun(hs)
        run.launch(inputs.set_phase_ops(sizes, k, OP_INS), keys, 0)
        n_ops = 900
        heap = rng.integers(0, sizes.size, n_ops)
        n = rng.integers(1, k + 1, n_ops)
        ops = np.zeros(n_ops, dtype=[("heap", "<u4"), ("kind_n", "<u4"), ("offset", "<u8")])
        ops["heap"] = heap
        ops["kind_n"] = (OP_DEL << 24) | n
        ops["offset"] = np.concatenate([[0], np.cumsum(n)[:-1]])
        out, counts = run.launch(ops, np.empty(0, dt), int(n.sum()))
        assert run.replay() == n_ops
        c = counts.cpu().numpy()
        assert (c <= n).all() and c.sum() == sizes.sum() - sum(h.size() for h in hs.heaps)
        for h in hs.heaps:
            check_properties(h)
        # an INS among the DELs of a list with no input keys
        bad = np.zeros(3, dtype=ops.dtype)
        bad["heap"] = [0, 2, 4]
        bad["kind_n"] = [(OP_DEL << 24) | 5, (OP_INS << 24) | 5, (OP_DEL << 24) | 5]
        bad["offset"] = [0, 0, 5]
        before = [h.size() for h in hs.heaps]
        o = torch.zeros(16, dtype=torch.int32 if key_bytes == 4 else torch.int64, device="cuda")
        hs.ops(torch.from_numpy(bad.view(np.uint8).copy()).cuda(), None, o)
        assert hs.heaps[2].sync_code() == -6
        assert hs.heaps[0].sync_code() == 0 and hs.heaps[4].sync_code() == 0
        assert hs.heaps[0].size() == max(before[0] - 5, 0)
        assert hs.heaps[4].size() == max(before[4] - 5, 0)


def test_heapset_delete_only_request_cursors():
    """Delete-only list through heapset_ops_req: the DELs of one request fill
    its output range contiguously in the order they hold their heap's root,
    and the request's cursor ends at the keys it got."""
    k = 1024
    sizes = np.array([40 * k, 9 * k + 100, 70 * k])
    keys = inputs.keys_u32(inputs.config_seed(5) + 21, int(sizes.sum()))
    reqs = [(0, 5 * k + 3), (2, 3 * k), (1, 12 * k), (0, 700), (2, 2 * k + 1)]
    ops, bases, pos = [], [], 0
    for r, (h, want) in enumerate(reqs):
        bases.append(pos)
        pos += want
        for j in range(0, want, k):
            ops.append((h, (OP_DEL << 24) | (1 << 23) | min(k, want - j), r))
    ops = np.array(ops, dtype=[("heap", "<u4"), ("kind_n", "<u4"), ("offset", "<u8")])
    with GHeapSet([int(c) for c in sizes], k=k) as hs:
        SetRun(hs).launch(inputs.set_phase_ops(sizes, k, OP_INS), keys, 0)
        hs.sync()
        # one block: the operations take their heaps' roots in list order
        hs.set_launch(ctas=1)
        out = torch.zeros(pos, dtype=torch.int32, device="cuda")
        req_base = torch.tensor(bases, dtype=torch.int64, device="cuda")
        cursor = torch.zeros(len(reqs), dtype=torch.int64, device="cuda")
        hs.ops_req(torch.from_numpy(ops.view(np.uint8).copy()).cuda(), None, out, None,
                   req_base, cursor)
        hs.sync()
        got = to_host(out, 4)
        cur = cursor.cpu().numpy()
        base = np.concatenate([[0], np.cumsum(sizes)[:-1]])
        left = {h: np.sort(keys[base[h]:base[h] + sizes[h]]) for h in range(sizes.size)}
        for r, (h, want) in enumerate(reqs):
            # each request gets the next smallest keys of its heap
            take = min(want, left[h].size)
            assert cur[r] == take
            assert np.array_equal(got[bases[r]:bases[r] + take], left[h][:take])
            left[h] = left[h][take:]


def test_heapset_error_is_per_heap():
    """A heap whose root lock never frees times out; the other heaps of the
    same launch finish correctly."""
    k = 64
    sizes = np.array([4096, 4096, 4096])
    keys = inputs.keys_u32(9, int(sizes.sum()))
    with GHeapSet([int(s) for s in sizes], k=k, log_capacity=256) as hs:
        hs.set_timeout(50_000_000)
        hs.heaps[1].debug_hold_root()
        run = SetRun(hs)
        run.launch(inputs.set_phase_ops(sizes, k, OP_INS), keys, 0)
        assert hs.sync_code() == -4
        assert hs.heaps[0].size() == 4096 and hs.heaps[2].size() == 4096
        check_properties(hs.heaps[0])
        check_properties(hs.heaps[2])


def test_heapset_insert_only_launch_runs_bottom_up():
    """Ascending batches, one block (list order): a bottom-up insert compares
    with one parent and stops, a top-down insert walks its whole path, so the
    set's level counter tells which ran.  A list that holds a DEL inserts
    top-down even in a bottom-up set."""
    k, nb = 64, 128
    keys = inputs.keys_u32(inputs.config_seed(5) + 9, k * nb, "ascending")
    sizes = np.array([keys.size])
    ins = inputs.set_phase_ops(sizes, k, OP_INS)
    # the same inserts plus one DEL of a single key at the end
    mixed = np.concatenate([ins, inputs.set_phase_ops(np.array([1]), k, OP_DEL)])
    # walk depth of top-down insert j (1-based slot j >= 2): floor(log2 j) levels
    td_levels = sum(int(np.floor(np.log2(j))) for j in range(2, nb + 1))

    def levels(bottom_up, ops):
        with GHeapSet([keys.size], k=k, bottom_up=bottom_up, stats=True) as hs:
            hs.set_launch(ctas=1)
            out = torch.zeros(1, dtype=torch.int32, device="cuda")
            hs.ops(torch.from_numpy(ops.view(np.uint8).copy()).cuda(), to_dev(keys), out)
            hs.sync()
            st = hs.stats()
            if ops.size == ins.size:
                assert st["merges"] == 0, st      # ascending: nothing to merge
            assert hs.heaps[0].size() == keys.size - (ops.size - ins.size)
            return st["ins_levels"]

    assert levels(True, ins) == nb - 1
    assert levels(False, ins) == td_levels
    assert levels(True, mixed) == td_levels
