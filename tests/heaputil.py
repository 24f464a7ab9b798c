"""Test helpers: drive a GHeap, record its calls, and replay the recorded
linearization order through the CPU oracle."""
import numpy as np

import oracle
from paper_1906_06504_gb300.heap import (GHeap, OP_DEL, OP_DTYPE, OP_INS,
                                         slot_to_node)

MAXK = {4: np.uint32(0xFFFFFFFF), 8: np.uint64(0xFFFFFFFFFFFFFFFF)}


def np_dtype(key_bytes):
    return np.uint32 if key_bytes == 4 else np.uint64


def to_dev(arr):
    import torch
    arr = np.ascontiguousarray(arr)
    view = arr.view(np.int32 if arr.dtype.itemsize == 4 else np.int64)
    return torch.from_numpy(view.copy()).cuda()


def to_host(t, key_bytes):
    return t.cpu().numpy().view(np_dtype(key_bytes))


class Recorder:
    """Wraps a GHeap; remembers each launching call so that the heap's
    linearization record can be replayed through the oracle."""

    def __init__(self, heap):
        self.h = heap
        self.calls = {}        # call_id -> (kind, data)
        self.next_id = 1

    def insert(self, keys):
        keys = np.ascontiguousarray(keys, dtype=np_dtype(self.h.key_bytes))
        if keys.size == 0:
            return
        self.h.insert(to_dev(keys))
        self.calls[self.next_id] = ("insert", keys)
        self.next_id += 1

    def delete_min(self, n):
        if n == 0:
            return None
        out, cnt = self.h.delete_min(n)
        rec = {"out": out, "cnt": cnt, "n": n}
        self.calls[self.next_id] = ("delete", rec)
        self.next_id += 1
        return rec

    def ops(self, ops, in_keys, out_size):
        import torch
        ops = np.ascontiguousarray(ops, dtype=OP_DTYPE)
        dt = np_dtype(self.h.key_bytes)
        in_keys = np.ascontiguousarray(in_keys, dtype=dt)
        ops_dev = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
        out = torch.zeros(max(out_size, 1), dtype=torch.int32 if dt == np.uint32 else torch.int64,
                          device="cuda")
        counts = torch.zeros(len(ops), dtype=torch.int32, device="cuda")
        ins_total = int(ops["n"][ops["kind"] == OP_INS].sum())
        self.h.ops(ops_dev, to_dev(in_keys) if in_keys.size else None, out, counts,
                   max_insert_keys=ins_total)
        rec = {"ops": ops, "in": in_keys, "out": out, "counts": counts}
        self.calls[self.next_id] = ("ops", rec)
        self.next_id += 1
        return rec

    def replay_and_compare(self):
        """Replays the recorded root order through the oracle and checks every
        DEL output bit for bit; returns the number of DEL ops checked."""
        self.h.sync()
        log, total = self.h.log()
        assert log.size == total, "linearization record truncated"
        kb = self.h.key_bytes
        host = {}
        for cid, (kind, rec) in self.calls.items():
            if kind == "delete":
                host[cid] = (to_host(rec["out"], kb), int(rec["cnt"].item()))
            elif kind == "ops":
                host[cid] = (to_host(rec["out"], kb), rec["counts"].cpu().numpy())
        q = oracle.BinaryHeapPQ()
        dt = np_dtype(kb)
        checked = 0
        seen = {cid: 0 for cid in self.calls}
        delivered = {}
        try:
            for e in log:
                cid = int(e["call_id"])
                kind_op = int(e["kind_n"]) >> 24
                n = int(e["kind_n"]) & 0xFFFFFF
                ref = int(e["ref"])
                kind, rec = self.calls[cid]
                seen[cid] += 1
                if kind == "insert":
                    assert kind_op == OP_INS
                    q.push(rec[ref:ref + n])
                elif kind == "delete":
                    assert kind_op == OP_DEL
                    # the op asks for min(k, keys still wanted by the call) and
                    # receives min(that, keys present) at its root hold
                    done = delivered.get(cid, 0)
                    assert ref == done
                    ask = min(self.h.k, rec["n"] - done)
                    assert n == min(ask, len(q)), (n, ask, len(q))
                    want = q.pop(n, dtype=dt)
                    got = host[cid][0][ref:ref + n]
                    assert np.array_equal(got, want), "DEL at offset %d differs" % ref
                    delivered[cid] = done + n
                    checked += 1
                else:
                    op = rec["ops"][ref]
                    assert int(op["kind"]) == kind_op
                    if kind_op == OP_INS:
                        assert n == int(op["n"])
                        off = int(op["offset"])
                        q.push(rec["in"][off:off + n])
                    else:
                        assert n == min(int(op["n"]), len(q)) == int(host[cid][1][ref])
                        want = q.pop(n, dtype=dt)
                        off = int(op["offset"])
                        got = host[cid][0][off:off + n]
                        assert np.array_equal(got, want), "op %d differs" % ref
                        checked += 1
            # every op of every call was linearized exactly once
            for cid, (kind, rec) in self.calls.items():
                if kind == "insert":
                    assert seen[cid] == -(-rec.size // self.h.k)
                elif kind == "ops":
                    assert seen[cid] == len(rec["ops"])
                else:
                    # a delete launch linearizes at most ceil(n/k) ops and
                    # returns the recorded count
                    assert seen[cid] <= -(-rec["n"] // self.h.k)
                    assert host[cid][1] == delivered.get(cid, 0)
            assert len(q) == self.h.size(), "multiset not conserved"
        finally:
            q.close()
        return checked


def snapshot_nodes(h):
    """Tree view of a quiescent heap: (nodes[n_slots, k], present, buffer, m)."""
    keys, st, buf, (m, s, _) = h.snapshot()
    occ = np.nonzero(st == 1)[0]
    assert set(occ.tolist()) == set(range(1, m + 1)) or (m == 0 and occ.size == 0), \
        "occupied slots %s != 1..%d" % (occ[:20], m)
    top = max([slot_to_node(j) for j in occ] + [1])
    nodes = np.zeros((top + 1, h.k), dtype=keys.dtype)
    present = np.zeros(top + 1, dtype=bool)
    for j in occ:
        p = slot_to_node(j)
        nodes[p] = keys[j]
        present[p] = True
    return nodes, present, buf[:s].copy(), m


def check_properties(h):
    nodes, present, buf, m = snapshot_nodes(h)
    code, where = oracle.check_properties(nodes, present, h.k, buf)
    assert code == 0, "%s violated at node %d" % (oracle.PROPERTY_NAMES[code], where)
    return m


def model_matches(h, model):
    """Bit-exact node-level equality with the sequential model."""
    nodes, present, buf, m = snapshot_nodes(h)
    assert m == model.m
    assert np.array_equal(buf, model.buf)
    have = {int(p) for p in np.nonzero(present)[0]}
    assert have == set(model.nodes)
    for p, v in model.nodes.items():
        assert np.array_equal(nodes[p], v), "node %d differs" % p


def mixed_ops(rng, n_pairs, k, key_bytes, partial=False, del_first=False):
    """Alternating INS/DEL ops (Section 5.5 ins-del pairs) with their input
    keys and output offsets."""
    dt = np_dtype(key_bytes)
    ops = np.zeros(2 * n_pairs, dtype=OP_DTYPE)
    ins_sizes = (rng.integers(1, k + 1, n_pairs) if partial else np.full(n_pairs, k))
    del_sizes = (rng.integers(1, k + 1, n_pairs) if partial else np.full(n_pairs, k))
    in_off = np.concatenate([[0], np.cumsum(ins_sizes)[:-1]])
    out_off = np.concatenate([[0], np.cumsum(del_sizes)[:-1]])
    a, b = (1, 0) if del_first else (0, 1)
    ops["kind"][a::2] = OP_INS
    ops["n"][a::2] = ins_sizes
    ops["offset"][a::2] = in_off
    ops["kind"][b::2] = OP_DEL
    ops["n"][b::2] = del_sizes
    ops["offset"][b::2] = out_off
    total_in = int(ins_sizes.sum())
    keys = rng.integers(0, np.iinfo(dt).max, total_in, dtype=dt, endpoint=True)
    return ops, keys, int(del_sizes.sum())
