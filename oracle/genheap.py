"""Sequential model of the generalized heap (arXiv 1906.06504, Sections 3-4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

This is a slow, plain statement of the INS and DEL steps of the generalized
heap executed one operation at a time, for node-by-node comparison with a GPU
run that uses a single thread block (where the concurrent heap executes the
very same sequence of steps).  It is for small cases only.

Every MergeAndSort below is taken by its definition (sort the union, split at
k; Section 3.2.1).  The paper's shortcuts -- swapping or keeping two nodes
whose key ranges do not overlap instead of merging (Section 4.3) -- produce
the same keys as that definition, so the model does not need them.

Readings taken where the paper is silent (the same ones the GPU code takes):

* Node numbering is 1-based (root = 1, children 2i and 2i+1).  The j-th
  allocated node sits at level d = floor(log2 j) at position
  2^d + bitreverse_d(j - 2^d): the bit-reversal permutation of Section 4.3, so
  consecutive inserts use disjoint paths below the root.  DEL removes the most
  recently allocated node (the same map applied to the current node count).
* Occupancy is tracked by counts, never by a MAX sentinel (Section 3.2.1
  fills with MAX; a legal key may equal MAX).
* DEL's placement: the larger half of MergeAndSort(l, r) goes to the child
  whose maximum was larger, the right child on a tie (Section 3.2.1).
* A DEL asked for r < k keys returns the r smallest of the root; the root is
  then refilled first from the partial buffer and, if that is not enough,
  from the last node, and sifted down like a full DEL.  With no full node
  left, DEL returns keys from the partial buffer (Section 3.3.2).
* A partial INS (n < k) merges into the partial buffer; if the buffer would
  reach k keys, its k smallest go down as a full batch (Section 3.3.2).
"""
import numpy as np


def bitrev(x, d):
    r = 0
    for _ in range(d):
        r = (r << 1) | (x & 1)
        x >>= 1
    return r


def node_of(j):
    """Physical node of the j-th allocated node (j >= 1), Section 4.3."""
    d = j.bit_length() - 1
    return (1 << d) + bitrev(j - (1 << d), d)


def path_to(t):
    """Nodes from the root down to node t, inclusive."""
    p = []
    while t >= 1:
        p.append(t)
        t //= 2
    return p[::-1]


def _ms(a, b, k):
    """MergeAndSort by definition: (k smallest, the rest), both ascending."""
    u = np.sort(np.concatenate([a, b]), kind="stable")
    return u[:k].copy(), u[k:].copy()


class GeneralizedHeapModel:
    def __init__(self, k, dtype=np.uint32):
        self.k = int(k)
        self.dtype = dtype
        self.nodes = {}          # physical node -> ascending array of k keys
        self.m = 0               # number of allocated (full) nodes
        self.buf = np.empty(0, dtype=dtype)

    # -- INS (Section 3.2.2 top-down insertion, Section 3.3.2 partial buffer)
    def insert(self, keys):
        k = self.k
        a = np.sort(np.asarray(keys, dtype=self.dtype))
        n = a.size
        if n == 0:
            return
        if n > k:
            raise ValueError("one INS takes at most k keys")
        if n < k:
            t = np.sort(np.concatenate([a, self.buf]))
            if t.size < k:
                if self.m >= 1:
                    self.nodes[1], self.buf = _ms(self.nodes[1], t, k)
                else:
                    self.buf = t
                return
            a, self.buf = t[:k].copy(), t[k:].copy()
        # a full batch of k keys
        if self.m == 0:
            self.m = 1
            self.nodes[1], self.buf = _ms(a, self.buf, k)
            return
        self.m += 1
        target = node_of(self.m)
        for x in path_to(target)[:-1]:
            self.nodes[x], a = _ms(self.nodes[x], a, k)
        self.nodes[target] = a

    # -- DEL (Section 3.2.1, partial buffer of Section 3.3.2)
    def delete(self, want):
        k = self.k
        want = int(want)
        if self.m == 0:
            take = min(want, self.buf.size)
            out, self.buf = self.buf[:take].copy(), self.buf[take:].copy()
            return out
        take = min(want, k)
        root = self.nodes[1]
        out = root[:take].copy()
        t = np.sort(np.concatenate([root[take:], self.buf]))
        if t.size >= k:
            self.nodes[1], self.buf = t[:k].copy(), t[k:].copy()
        else:
            if self.m == 1:
                del self.nodes[1]
                self.m = 0
                self.buf = t
                return out
            last = node_of(self.m)
            self.m -= 1
            lk = self.nodes.pop(last)
            self.nodes[1], self.buf = _ms(t, lk, k)
        self._sift_down(1)
        return out

    def _sift_down(self, cur):
        k = self.k
        nodes = self.nodes
        while True:
            l, r = 2 * cur, 2 * cur + 1
            kids = [c for c in (l, r) if c in nodes]
            if not kids:
                return
            c_keys = nodes[cur]
            if len(kids) == 1:
                c = kids[0]
                if c_keys[-1] <= nodes[c][0]:
                    return
                nodes[cur], nodes[c] = _ms(c_keys, nodes[c], k)
                cur = c
                continue
            if c_keys[-1] <= min(nodes[l][0], nodes[r][0]):
                return
            big = l if nodes[l][-1] > nodes[r][-1] else r
            sm = r if big == l else l
            nodes[sm], nodes[big] = _ms(nodes[l], nodes[r], k)
            if c_keys[-1] <= nodes[sm][0]:
                return
            nodes[cur], nodes[sm] = _ms(c_keys, nodes[sm], k)
            cur = sm

    # -- inspection
    def size(self):
        return self.m * self.k + self.buf.size

    def snapshot(self, n_slots=None):
        """(nodes[n_slots, k], present[n_slots], buffer)."""
        top = max(self.nodes) if self.nodes else 0
        if n_slots is None:
            n_slots = top + 1
        arr = np.zeros((n_slots, self.k), dtype=self.dtype)
        present = np.zeros(n_slots, dtype=bool)
        for i, v in self.nodes.items():
            arr[i] = v
            present[i] = True
        return arr, present, self.buf.copy()
