"""Config 2's mixed run at full size, replayed through the CPU oracle.

A heap of k = 1024 prefilled with 2^24 uniform uint32 keys takes 2^16
ins-del pairs of 1024 keys each (Section 5.5) from every thread block of the
device at once -- the heap is 14 levels deep.  The GPU records the order in
which operations held the root; replaying that order through the textbook
binary heap fixes every DEL output (Section 3.3.3, Theorem 1), and every one
of the 2^16 DELs must match it bit for bit.  Properties 1-3 (Section 3.1)
must hold on the heap left at the end.  A DEL treats a child that an INS
still on its way down has reserved as absent (that INS merges with the
child's parent before it fills the child); the counters show such children
were met, and the replay shows the results stayed exact.  With yields = 0 (the paper's INS/DEL
cooperation of Section 3.3.2, the default: a DEL whose last node is an INS
target still in flight marks it and waits, holding the root, for the keys)
the device counters must show that such deliveries happened at this depth,
and that INSs handed their keys over at the level they were on when they saw
the mark, before reaching their target.
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


from heaputil import Recorder, check_properties  # noqa: E402


@pytest.mark.parametrize("yields", [64, 0])
def test_config2_mixed_full_size_replay(yields):
    from paper_1906_06504_gb300.heap import GHeap
    n_prefill, n_pairs, k = 1 << 24, 1 << 16, 1024
    pre, stream, ops = inputs.mixed_pairs(n_prefill, n_pairs, k)
    log_cap = n_prefill // k + 2 * n_pairs + 1024
    with GHeap(capacity=n_prefill + n_pairs * k, k=k, log_capacity=log_cap, stats=True) as h:
        h.set_yields(yields)
        r = Recorder(h)
        r.insert(pre)
        h.sync()
        before = h.stats()
        rec = r.ops(ops, stream, n_pairs * k)
        h.sync()
        st = h.stats()
        counts = rec["counts"].cpu().numpy()
        assert np.all(counts[0::2] == k)
        # every DEL of the list, each checked against the oracle's replay
        assert r.replay_and_compare() == n_pairs
        check_properties(h)
        deliveries = st["deliveries"] - before["deliveries"]
        absent = st["target_children"] - before["target_children"]
        early = st["intercepts"] - before["intercepts"]
        if yields == 0:
            # the hand-off ran (mostly before the INS reached its target),
            # and DELs sifted past children that in-flight INSs had reserved
            # (treated as absent: each such INS merges with the child's
            # parent before it fills the child)
            assert deliveries > 0 and early > 0 and absent > 0, st
            assert early <= deliveries, st
        print("yields=%d: %d deliveries (%d before the target), %d root hand-backs, "
              "%d reserved children passed, %d DEL levels"
              % (yields, deliveries, early, st["del_yields"] - before["del_yields"],
                 absent, st["del_levels"] - before["del_levels"]))
