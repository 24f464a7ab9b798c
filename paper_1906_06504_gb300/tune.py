"""Autotuner for heap sets: picks the node capacity k and the merge width
(items per thread, which sets the block shape) for a given set of heap sizes
by timing an insert-all + deleteMin-all pass of a scaled-down copy of the
workload for each candidate on the device.  Each candidate is one heap-set
launch pair through the C ABI; the fastest aggregate keys/s wins."""
import numpy as np

from . import inputs
from .heap import GHeapSet, OP_DEL, OP_INS

K_CANDIDATES = (256, 512, 1024, 2048)


def ipt_candidates(k):
    # merge threads 2k/ipt must fit the block bound (512 for ipt 4, 256 above)
    out = []
    for ipt in (4, 8, 16):
        nmt = max(32, 2 * k // ipt)
        if nmt <= (512 if ipt == 4 else 256):
            out.append(ipt)
    return out


def _time_pass(torch, sizes, keys_dev, k, ipt, reps=2, bottom_up=False):
    ins = inputs.set_phase_ops(sizes, k, OP_INS)
    dele = inputs.set_phase_ops(sizes, k, OP_DEL)
    total = int(np.sum(sizes))
    out = torch.empty(total, dtype=torch.int32, device="cuda")
    d_ins = torch.from_numpy(ins.view(np.uint8).copy()).cuda()
    d_del = torch.from_numpy(dele.view(np.uint8).copy()).cuda()
    best = None
    with GHeapSet([int(s) for s in sizes], k=k, bottom_up=bottom_up) as hs:
        hs.set_launch(items_per_thread=ipt)
        for r in range(reps + 1):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            hs.ops(d_ins, keys_dev, None)
            hs.ops(d_del, None, out)
            e1.record()
            torch.cuda.synchronize()
            hs.sync()
            ms = e0.elapsed_time(e1)
            if r > 0:
                best = ms if best is None else min(best, ms)
    return 2.0 * total / (best / 1e3)


def autotune_set(sizes, keys, scale=0.25, k_candidates=K_CANDIDATES, verbose=False,
                 bottom_up=False):
    """Returns (best, table): best = dict(k, items_per_thread, keys_per_s) for
    a copy of the workload with every heap scaled by `scale`."""
    import torch
    s = np.maximum(1, (np.asarray(sizes, dtype=np.float64) * scale).astype(np.int64))
    total = int(s.sum())
    keys_dev = torch.from_numpy(np.ascontiguousarray(keys[:total]).view(np.int32)).cuda()
    table = []
    for k in k_candidates:
        for ipt in ipt_candidates(k):
            v = _time_pass(torch, s, keys_dev, k, ipt, bottom_up=bottom_up)
            table.append({"k": k, "items_per_thread": ipt, "keys_per_s": v})
            if verbose:
                print("tune k=%d ipt=%d %.3e keys/s" % (k, ipt, v))
    best = max(table, key=lambda r: r["keys_per_s"])
    return best, table
