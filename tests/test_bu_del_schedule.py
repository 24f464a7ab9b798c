"""Bottom-up inserts concurrent with top-down deletes (Sections 3.3.4-3.3.5):
a CPU model of the protocol on explicit schedules.

The model follows the paper's BU-INS/TD-DEL heap step by step: a bottom-up
INS stores its batch at the target node and rises one level at a time,
releasing its node as INSHOLD while it locks the parent, then taking the node
back; a DEL returns the root batch, refills the root from the last node and
sifts down with MergeAndSort(l, r) and MergeAndSort(cur, small half)
(Section 3.2.1), and it may take an INSHOLD node -- as the last node, or as a
child on its way down -- releasing a child it took from INSHOLD as DELMOD.
An INS that finds its node no longer INSHOLD stops.  Each schedule below runs
whole operations and single INS levels in a fixed order, so the outcome is
exact; operations that do not overlap an INS are sequential, as in the paper.

Section 3.3.5 orders a history by the release of each operation's last lock
(the root for a DEL, the last node an INS held for a BU-INS) and claims that
replaying the operations in that order gives every DEL's result.  On these
schedules it does not: a DEL returns keys of an INS that is still rising.
Nor does any fixed point of the INS's own steps, or the DEL that first takes
its node: the keys of the INS become the root's content only when later
DELs have carried them up, so the one order that replays depends on where
the keys travel afterwards.  This is why the GPU heap runs bottom-up inserts
only in launches without deletes (its record must be replayable).
"""
import itertools

INSHOLD, DELMOD, AVAIL = "INSHOLD", "DELMOD", "AVAIL"


def mas(a, b):
    """MergeAndSort (Section 3.2.1): the len(a) smallest and the rest."""
    u = sorted(list(a) + list(b))
    return u[:len(a)], u[len(a):]


class Model:
    """Nodes at tree positions 1..m (children of p: 2p, 2p+1), k keys each."""

    def __init__(self, nodes):
        self.nodes = {p: sorted(v) for p, v in nodes.items()}
        self.state = {p: AVAIL for p in self.nodes}
        self.m = len(self.nodes)

    def all_keys(self):
        return sorted(x for v in self.nodes.values() for x in v)

    # -- TD-DEL, run whole
    def delete(self):
        out = self.nodes[1]
        last = self.m
        refill = self.nodes.pop(last)
        self.state.pop(last)
        self.m -= 1
        if last == 1:
            return out
        cur, pos = refill, 1
        while True:
            kids = [c for c in (2 * pos, 2 * pos + 1) if c <= self.m]
            if not kids or max(cur) <= min(min(self.nodes[c]) for c in kids):
                break
            for c in kids:                       # taken from INSHOLD: DELMOD
                if isinstance(self.state[c], tuple) and self.state[c][0] == INSHOLD:
                    self.state[c] = (DELMOD, self.state[c][1])
            if len(kids) == 1:
                (c,) = kids
                self.nodes[pos], cur = mas(cur, self.nodes[c])
                pos = c
                continue
            l, r = kids
            lo, hi = mas(self.nodes[l], self.nodes[r])
            big = l if max(self.nodes[l]) > max(self.nodes[r]) else r
            small = r if big == l else l
            self.nodes[big] = hi
            self.nodes[pos], cur = mas(cur, lo)
            pos = small
        self.nodes[pos] = cur
        return out

    # -- BU-INS, one step at a time
    def ins_place(self, owner, batch):
        """Stores the batch at the target (the next free position); returns it."""
        self.m += 1
        self.nodes[self.m] = sorted(batch)
        self.state[self.m] = (INSHOLD, owner)
        return self.m

    def ins_rise(self, owner, pos):
        """One level: lock the parent, take the own node back, MergeAndSort.
        Returns the new position, or None when the INS is done (its node was
        taken by a DEL, the root was reached, or the parent was no larger)."""
        if self.state.get(pos) != (INSHOLD, owner):
            return None                          # DELMOD or gone: stop
        par = pos // 2
        if max(self.nodes[par]) <= min(self.nodes[pos]):
            self.state[pos] = AVAIL
            return None
        self.nodes[par], self.nodes[pos] = mas(self.nodes[par], self.nodes[pos])
        self.state[pos] = AVAIL
        if par == 1:
            return None
        self.state[par] = (INSHOLD, owner)
        return par


def replay(initial, order, ins_keys, k):
    """Sequential replay (a plain priority queue): DEL returns the k smallest."""
    pool = list(initial)
    outs = []
    for op in order:
        if op == "INS":
            pool = sorted(pool + list(ins_keys))
        else:
            pool.sort()
            outs.append(pool[:k])
            pool = pool[k:]
    return outs


def full_nodes(n, k=2):
    # node p holds [10p, 10p + 1, ...]: a valid heap
    return {p: [10 * p + j for j in range(k)] for p in range(1, n + 1)}


def orders_with_ins(n_dels):
    """Every place of the one INS among n_dels DELs."""
    for i in range(n_dels + 1):
        yield i, ["DEL"] * i + ["INS"] + ["DEL"] * (n_dels - i)


def test_del_takes_a_rising_insert_as_its_last_node():
    """The last node is the INS's target, still INSHOLD: DEL 1 refills the
    root with the INS's keys and DEL 2 returns them, before the INS (which
    then finds its node gone) releases its last lock."""
    k = 2
    h = Model(full_nodes(7, k))
    initial = h.all_keys()
    pos = h.ins_place("X", [1, 2])               # target: node 8
    got = [h.delete(), h.delete()]
    assert got == [[10, 11], [1, 2]]
    assert h.ins_rise("X", pos) is None          # gone: the INS ends here
    # Section 3.3.5's order: both DELs released the root before the INS's
    # last lock -- the replay disagrees with what DEL 2 returned
    paper = ["DEL", "DEL", "INS"]
    assert replay(initial, paper, [1, 2], k) != got
    # the only replayable place: between the two DELs (under DEL 1's root hold)
    ok = [i for i, o in orders_with_ins(2) if replay(initial, o, [1, 2], k) == got]
    assert ok == [1]


def test_del_sift_carries_a_rising_insert_up_before_its_last_lock():
    """The INS has risen one level and waits, INSHOLD, for its parent; DEL 1
    sifts through that parent and takes the INS's node (DELMOD), carrying the
    INS's keys one level up -- above a root that does not have them yet.  DEL
    2 still returns the old root; DEL 3 returns the INS's keys; only then does
    the INS take its node back, find DELMOD and stop."""
    k = 2
    h = Model(full_nodes(9, k))
    initial = h.all_keys()
    pos = h.ins_place("X", [5, 25])             # target: node 10
    pos = h.ins_rise("X", pos)                   # now INSHOLD at node 5
    assert pos == 5 and h.nodes[5] == [5, 25]
    got = [h.delete()]                           # sifts 1 -> 2 -> 5, takes node 5
    assert h.state[5] == (DELMOD, "X") and h.nodes[2] == [5, 25]
    got += [h.delete(), h.delete()]
    assert got == [[10, 11], [20, 21], [5, 25]]
    assert h.ins_rise("X", pos) is None          # DELMOD: the INS stops now
    n = len(got)
    # Section 3.3.5's order (the INS last): DEL 3 should not see the keys
    assert replay(initial, ["DEL"] * n + ["INS"], [5, 25], k) != got
    # the DEL that took the INS's node (DEL 1) is no place for it either:
    # then DEL 2 would have had to return 5
    assert replay(initial, ["DEL", "INS", "DEL", "DEL"], [5, 25], k) != got
    # the one order that replays puts the INS between DEL 2 and DEL 3: a
    # point that no lock of the INS, nor of DEL 1, marks
    ok = [i for i, o in orders_with_ins(n) if replay(initial, o, [5, 25], k) == got]
    assert ok == [2]


def test_model_is_the_sequential_heap_without_overlap():
    """Pin of the model itself: with no INS in flight it is the sequential
    generalized heap -- deletes return the k smallest, in order -- and a
    bottom-up INS that rises to the end leaves a heap the DELs drain in
    sorted order."""
    k = 2
    h = Model(full_nodes(15, k))
    keys = h.all_keys()
    pos = h.ins_place("Y", [3, 144])
    while pos is not None:
        pos = h.ins_rise("Y", pos)
    keys = sorted(keys + [3, 144])
    out = []
    while h.m:
        out += h.delete()
    assert out == keys
    # every order of one INS among DELs, run sequentially, replays
    for i, o in orders_with_ins(3):
        g = Model(full_nodes(7, k))
        init = g.all_keys()
        res = []
        for op in o:
            if op == "INS":
                p = g.ins_place("Z", [7, 8])
                while p is not None:
                    p = g.ins_rise("Z", p)
            else:
                res.append(g.delete())
        assert res == replay(init, o, [7, 8], k), (i, res)
