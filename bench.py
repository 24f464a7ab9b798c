"""Benchmark: insert + deleteMin throughput of the generalized concurrent heap.

Workload (one step): the raw heap throughput configuration of arXiv 1906.06504
Section 5.2 at GB300 scale -- 2^26 uniform uint32 keys, node capacity k = 1024,
inserted into an empty heap and then all deleted (insert-all, deleteMin-all),
every thread block of the device running operations concurrently, on the
paper's BU-INS/TD-DEL heap (Section 3.3.4: bottom-up inserts, top-down
deleteMin).  --top-down runs it on the TD-INS/TD-DEL heap instead; the
JSON line reports the other variant beside the headline.

value  : (keys inserted + keys deleted) / device time, inputs resident in HBM.
e2e    : the same through the C ABI from pinned host buffers, the H2D copy of
         the keys and the D2H copy of the sorted output inside the timed region.
roofline: algorithmic node bytes of the dominant launch (deleteMin-all) over
         its CUDA-event duration, against the measured HBM copy bandwidth.
cpu_baseline: the CPU oracle (sequential binary heap) on a bounded sample.

--impl reference times that CPU oracle as the reference arm.
Multi-GPU (torchrun): every rank drives its own heap (independent replicas;
a single heap has one root and does not shard), weak scaling.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_KEYS = 1 << 26
K = 1024
METRIC = "insert+deleteMin keys/s (k=1024, 2^26 u32)"
UNIT = "keys/s"


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one full-size
# launch (2^26 u32 keys, k=1024, one block per SM), from one ncu capture of
# the kernel built from sources whose code (comments and white space
# removed) has these SHA-256 digests; reported as null once the code differs.
MEASURED_TRAFFIC = {
    "sources": {
        "gheap_kernel.cuh": "bd6d668cdea2fe64e6068bbd8123bace844d47106568a53ca6c985f4f013bf98",
        "gheap.cu": "56668c8fe054a818490fc522934010fe5a2811ddded996e425da626848c352bb",
    },
    "bottom_up": True,
    "insert": 707904256 + 749434624,
    "delete": 1165813504 + 1428330752,
}


def code_digest(text):
    """SHA-256 of C/C++ source with comments and white space removed."""
    import hashlib
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return hashlib.sha256(" ".join(text.split()).encode()).hexdigest()


def measured_traffic(kind, n, k, ctas, bottom_up):
    """DRAM bytes of one `kind` launch if the capture applies to this run."""
    if n != N_KEYS or k != K or ctas not in (0, None) or bottom_up != MEASURED_TRAFFIC["bottom_up"]:
        return None
    csrc = os.path.join(ROOT, "paper_1906_06504_gb300", "csrc")
    for name, digest in MEASURED_TRAFFIC["sources"].items():
        with open(os.path.join(csrc, name)) as f:
            if code_digest(f.read()) != digest:
                return None
    return MEASURED_TRAFFIC[kind]


def roofline_of(bytes_moved, ms, kernel, what):
    """Roofline object for `bytes_moved` algorithmic bytes in `ms`."""
    peak, kind = peaks()
    achieved = bytes_moved / (ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": kind, "algorithmic_bytes": int(bytes_moved),
            "kernel": kernel, "bytes": what}


def node_bytes(st, k, key_bytes):
    """Node batches loaded and stored, as counted by the kernel."""
    return (st["node_loads"] + st["node_stores"]) * k * key_bytes


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, dist=None):
    """The largest of every rank's x (the job ends when its slowest rank does);
    x itself without a process group."""
    if dist is None:
        return float(x)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(keys_per_rank_step, steps, world_size, ms):
    """Keys per second of the whole job: every rank's keys over the max time."""
    return float(keys_per_rank_step) * steps * world_size / (ms / 1e3)


def _cpu_full_worker(args):
    """Worker: insert-all then delete-all of n keys of `seed`, `reps` times,
    through the oracle's binary heap or std::priority_queue; returns the
    seconds of each run (inputs generated before the clock starts)."""
    kind, n, reps, seed = args
    import oracle
    from paper_1906_06504_gb300 import inputs
    keys = inputs.keys_u32(seed, n)
    times = []
    for _ in range(reps):
        if kind == "oracle":
            q = oracle.BinaryHeapPQ(n)
            t0 = time.perf_counter()
            q.push(keys)
            out = q.pop(n, dtype=np.uint32)
            dt = time.perf_counter() - t0
            q.close()
        else:
            out, dt = oracle.stl_insert_delete(keys)
        assert out.size == n and bool(np.all(out[1:] >= out[:-1]))
        times.append(dt)
        del out
    return times


class CpuBaselines:
    """The sequential CPU heaps -- the oracle's binary heap and the paper's
    std::priority_queue baseline (Table 1) -- timed on the full workload, the
    oracle best of `reps` runs and the standard-library heap (about twice as
    slow on this host) of `stl_reps`, one run after another in a
    spawn-started worker process per heap (one host core each), while the GPU
    benchmark runs: they add CPU work, not wall time."""

    def __init__(self, n, seed, reps=3, stl_reps=1):
        import multiprocessing as mp
        self.n, self.reps, self.stl_reps = n, reps, stl_reps
        self.pool = mp.get_context("spawn").Pool(2)
        self.res = {kind: [self.pool.apply_async(_cpu_full_worker, ((kind, n, r, seed),))]
                    for kind, r in (("oracle", reps), ("stl", stl_reps))}

    def result(self, timeout=1800):
        runs = {kind: [t for r in rs for t in r.get(timeout)] for kind, rs in self.res.items()}
        self.pool.close()
        self.pool.join()
        n = self.n
        what = ("the full workload: insert-all + deleteMin-all of the same %d uniform u32 keys "
                "(one sequential heap, one thread), best of %d runs one after another in a "
                "worker process on its own host core, beside the other CPU heap's worker, "
                "while the GPU benchmark runs" % (n, self.reps))
        return {"value": 2.0 * n / min(runs["oracle"]), "unit": UNIT, "cores": 1,
                "kind": "oracle", "host": host_cpu(), "sample": what, "same_config": True,
                "runs_s": runs["oracle"], "build": "gcc -O3",
                "stl_priority_queue": {"value": 2.0 * n / min(runs["stl"]), "unit": UNIT,
                                       "cores": 1, "runs_s": runs["stl"], "build": "g++ -O3",
                                       "what": "std::priority_queue<uint32_t> min-queue, the "
                                               "sequential CPU heap of the paper's Table 1, "
                                               "best of %d run(s) on the same workload"
                                               % self.stl_reps}}


def cpu_oracle_sample(n_sample):
    """Insert-all then delete-all of n_sample keys through the oracle's
    binary heap; returns (keys/s, seconds)."""
    import oracle
    from paper_1906_06504_gb300 import inputs
    keys = inputs.keys_u32(inputs.config_seed(2), n_sample)
    q = oracle.BinaryHeapPQ(n_sample)
    t0 = time.perf_counter()
    q.push(keys)
    out = q.pop(n_sample, dtype=np.uint32)
    dt = time.perf_counter() - t0
    q.close()
    assert out.size == n_sample
    return 2 * n_sample / dt, dt


def host_cpu():
    """The host CPU model and logical core count, for the CPU timings."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    if key == "model name":
                        break
    except OSError:
        pass
    # Arm cores report a part number (MIDR): name the ones of this class of host
    arm_parts = {"0xd4f": "Arm Neoverse-V2", "0xd40": "Arm Neoverse-V1", "0xd0c": "Arm Neoverse-N1",
                 "0xd49": "Arm Neoverse-N2"}
    if model in arm_parts:
        model = "%s (part %s)" % (arm_parts[model], model)
    import platform
    return {"model": model or platform.processor() or platform.machine(),
            "arch": platform.machine(), "logical_cores": os.cpu_count()}


def _oracle_heaps(args):
    """Worker: insert-all then delete-all through one oracle binary heap per
    (offset, size) of `spans`; returns the seconds spent."""
    keys, spans = args
    import oracle
    t0 = time.perf_counter()
    for off, size in spans:
        q = oracle.BinaryHeapPQ(int(size))
        q.push(keys[off:off + size])
        out = q.pop(int(size), dtype=np.uint32)
        q.close()
        assert out.size == size
    return time.perf_counter() - t0


def cpu_oracle_heapset(sizes, keys, scale=1.0 / 16):
    """The oracle on the heap-set workload, heaps scaled by `scale`, spread
    over every host core (independent heaps, a spawn-started pool); returns
    (keys/s, cores, seconds)."""
    import multiprocessing as mp
    s = np.maximum(1, (np.asarray(sizes, dtype=np.float64) * scale).astype(np.int64))
    offs = np.concatenate([[0], np.cumsum(s)[:-1]])
    cores = os.cpu_count() or 1
    order = np.argsort(-s)                    # largest heaps first, dealt round-robin
    parts = [[] for _ in range(cores)]
    for j, h in enumerate(order):
        parts[j % cores].append((int(offs[h]), int(s[h])))
    ks = np.ascontiguousarray(keys[:int(s.sum())])
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_heaps, [(ks[:1], [(0, 1)])] * cores)      # start-up, untimed
        t0 = time.perf_counter()
        pool.map(_oracle_heaps, [(ks, p) for p in parts if p])
        dt = time.perf_counter() - t0
    return 2.0 * float(s.sum()) / dt, cores, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            dist.destroy_process_group()
            return
    n_sample = 1 << 23
    vals, secs = [], []
    for i in range(args.warmup + args.steps):
        v, dt = cpu_oracle_sample(n_sample)
        if i >= args.warmup:
            vals.append(v)
            secs.append(dt)
    value = float(np.median(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        # a step is the bounded sample (config.sample_keys keys in and out)
        "ms_per_step": float(np.median(secs)) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": "insert-all + deleteMin-all, 2^26 uniform u32 keys, k=1024",
                   "keys": N_KEYS, "k": K, "sample_keys": n_sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "host": host_cpu(),
                         "sample": "insert-all + delete-all of the first 2^23 of the same "
                                   "uniform keys per step (the full 2^26-key workload takes "
                                   "about half a minute per step on one core), sequential "
                                   "binary heap (gcc -O3), 1 thread", "same_config": False},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def replay_ops_record(log, pre, stream, ops, out, counts, k):
    """Replays a mixed run's linearization record through the CPU oracle's
    binary heap (Section 3.3.3, Theorem 1): call 1 inserted the prefill, call
    2 ran the op list.  Returns (DELs checked, all equal, oracle seconds)."""
    import oracle
    q = oracle.BinaryHeapPQ(int(pre.size) + int(stream.size))
    checked, ok = 0, True
    t0 = time.perf_counter()
    try:
        for e in log:
            cid = int(e["call_id"])
            n = int(e["kind_n"]) & 0xFFFFFF
            ref = int(e["ref"])
            if cid == 1:
                q.push(pre[ref:ref + n])
                continue
            off = int(ops["offset"][ref])
            if int(ops["kind"][ref]) == 1:
                q.push(stream[off:off + n])
            else:
                want = q.pop(n, dtype=np.uint32)
                ok = ok and n == int(counts[ref]) and bool(np.array_equal(out[off:off + n], want))
                checked += 1
    finally:
        dt = time.perf_counter() - t0
        q.close()
    return checked, ok, dt


def run_mixed(torch, n_prefill=1 << 24, n_pairs=1 << 16, k=K, ipt=8, ctas=0, seed_off=0,
              replay=True, count=True):
    """Mixed concurrent workload: prefill 2^24 keys, then 2^16 ins-del pairs
    of k keys issued to all blocks at once (Section 5.5 ins-del pairs).  The
    timed launch keeps its linearization record, which the CPU oracle then
    replays: every DEL of the list is compared with the oracle's output."""
    from paper_1906_06504_gb300 import inputs
    from paper_1906_06504_gb300.heap import GHeap
    pre, stream_keys, ops = inputs.mixed_pairs(n_prefill, n_pairs, k, seed_off)
    d_ops = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
    d_pre = torch.from_numpy(pre.view(np.int32)).cuda()
    d_in = torch.from_numpy(stream_keys.view(np.int32)).cuda()
    d_out = torch.empty(n_pairs * k, dtype=torch.int32, device="cuda")
    counts = torch.zeros(2 * n_pairs, dtype=torch.int32, device="cuda")
    log_cap = n_prefill // k + 2 * n_pairs + 1024
    with GHeap(capacity=n_prefill + n_pairs * k, k=k, log_capacity=log_cap) as h:
        h.set_launch(ctas=ctas, items_per_thread=ipt)
        h.insert(d_pre)
        h.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        h.ops(d_ops, d_in, d_out, counts)
        e1.record()
        torch.cuda.synchronize()
        h.sync()
        ms = e0.elapsed_time(e1)
        c = counts.cpu().numpy().astype(np.int64)
        assert h.size() == n_prefill + int(c[0::2].sum()) - int(c[1::2].sum())
        log, total = h.log()
    moved = int(counts.sum().item())
    r = {"workload": "prefill %d keys, then %d ins-del pairs of k=%d keys, all blocks"
                     % (n_prefill, n_pairs, k),
         "value": moved / (ms / 1e3), "unit": UNIT, "ms": ms, "keys": moved,
         "record": "linearization record kept in the timed launch (%d entries)" % total}
    if replay:
        assert log.size == total
        checked, ok, dt = replay_ops_record(log, pre, stream_keys, ops,
                                            d_out.cpu().numpy().view(np.uint32), c, k)
        r["exact"] = bool(ok and checked == n_pairs)
        r["dels_checked"] = checked
        r["cpu_oracle_replay_s"] = dt
    if count:
        with GHeap(capacity=n_prefill + n_pairs * k, k=k) as h:
            h.set_launch(ctas=ctas, items_per_thread=ipt)
            h.insert(d_pre)
            h.sync()
            h.set_stats(True)
            h.ops(d_ops, d_in, d_out, counts)
            h.sync()
            st = h.stats()
        r["roofline"] = roofline_of(node_bytes(st, k, 4) + moved * 4, ms,
                                    "heap_kernel (operation-list launch)",
                                    "node batches loaded + stored (kernel counters, separate "
                                    "run) + the keys inserted and returned")
    return r


def run_batched(torch, steps=3, tune=True, n_heaps=256, verify_heaps=8, bottom_up=False,
                best=None, scale=1.0, cpu=True):
    """Batched heaps: 256 heaps with log-uniform sizes 2^10 to 2^22 keys; one
    launch inserts all of them, one launch deletes all, both replayed from
    captured CUDA graphs; k and the merge width autotuned (or `best`).
    `scale` shrinks every heap (a small case for profiling)."""
    from paper_1906_06504_gb300 import inputs, tune as tuner
    from paper_1906_06504_gb300.heap import GHeapSet, OP_INS, OP_DEL
    sizes = inputs.loguniform_sizes(inputs.config_seed(5), n_heaps, 10, 22)
    if scale != 1.0:
        sizes = np.maximum(1, (sizes * scale).astype(np.int64))
    total = int(sizes.sum())
    keys = inputs.keys_u32(inputs.config_seed(5), total)
    if best is not None:
        table = []
    elif tune:
        best, table = tuner.autotune_set(sizes, keys, scale=0.125, bottom_up=bottom_up)
    else:
        best, table = {"k": 1024, "items_per_thread": 8}, []
    k, ipt = best["k"], best["items_per_thread"]
    ins = inputs.set_phase_ops(sizes, k, OP_INS)
    dele = inputs.set_phase_ops(sizes, k, OP_DEL)
    d_ins = torch.from_numpy(ins.view(np.uint8).copy()).cuda()
    d_del = torch.from_numpy(dele.view(np.uint8).copy()).cuda()
    d_keys = torch.from_numpy(keys.view(np.int32)).cuda()
    d_out = torch.empty(total, dtype=torch.int32, device="cuda")
    with GHeapSet([int(x) for x in sizes], k=k, bottom_up=bottom_up) as hs:
        hs.set_launch(items_per_thread=ipt)
        g_ins = hs.graph(d_ins, d_keys, None)
        g_del = hs.graph(d_del, None, d_out)
        g_ins.launch()
        g_del.launch()
        torch.cuda.synchronize()
        hs.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            g_ins.launch()
            g_del.launch()
        e1.record()
        torch.cuda.synchronize()
        hs.sync()
        ms = e0.elapsed_time(e1) / steps
        # every heap ends empty; sampled heaps returned exactly their input
        assert all(h.size() == 0 for h in hs.heaps)
        out = d_out.cpu().numpy().view(np.uint32)
        base = np.concatenate([[0], np.cumsum(sizes)[:-1]])
        for hid in np.linspace(0, n_heaps - 1, verify_heaps).astype(int):
            seg = slice(base[hid], base[hid] + sizes[hid])
            assert np.array_equal(np.sort(out[seg]), np.sort(keys[seg]))
        g_ins.close()
        g_del.close()
    # node traffic of one step, counted by the kernel in a separate run
    with GHeapSet([int(x) for x in sizes], k=k, bottom_up=bottom_up, stats=True) as hs:
        hs.set_launch(items_per_thread=ipt)
        hs.ops(d_ins, d_keys, None)
        hs.ops(d_del, None, d_out)
        torch.cuda.synchronize()
        st = hs.stats()
    step_bytes = node_bytes(st, k, 4) + 2 * total * 4
    cpu_v, cores, cpu_s = cpu_oracle_heapset(sizes, keys) if cpu else (None, None, None)
    return {"workload": "256 heaps, log-uniform 2^10..2^22 keys (%d total), insert-all + "
                        "deleteMin-all, one launch each, CUDA-graph replay" % total,
            "insert": "bottom-up" if bottom_up else "top-down",
            "value": 2.0 * total / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "k": k, "items_per_thread": ipt, "autotune": table,
            "roofline": roofline_of(step_bytes, ms, "heap_kernel (heap-set insert + deleteMin "
                                    "launches)", "node batches loaded + stored (kernel "
                                    "counters, separate run) + input and output keys"),
            "cpu_oracle": {"value": cpu_v, "unit": UNIT, "cores": cores, "seconds": cpu_s,
                           "host": host_cpu(),
                           "sample": "the same 256 heaps scaled to 1/16 of their sizes, one "
                                     "oracle binary heap each, spread over every host core"}}


def run_serve(torch, n_requests=20000, rate=50000.0, n_heaps=256, count=True):
    """Served heaps: Poisson arrivals of insert / deleteMin requests of
    1..4096 keys over 256 heaps, continuously batched through one persistent
    serving launch.  A second, untimed run of the same requests with the
    kernel's counters on gives the node traffic: each heap takes its requests
    in arrival order in both runs, so each heap sees the same operations."""
    from paper_1906_06504_gb300 import inputs
    from paper_1906_06504_gb300.serve import HeapServer, latency_summary, poisson_requests
    sizes = inputs.loguniform_sizes(inputs.config_seed(5), n_heaps, 10, 22)
    caps = [int(max(s, 1 << 18)) for s in sizes]

    def serve(stats, realtime, n=n_requests, seed_off=7):
        reqs = poisson_requests(inputs.config_seed(5) + seed_off, n, n_heaps, rate,
                                max_keys=4096)
        srv = HeapServer(caps, k=1024, arena_keys=1 << 24, stats=stats)
        try:
            srv.preadmit(range(n_heaps))
            srv.run(reqs, realtime=realtime)
            info = dict(srv.stats)
            if stats:
                info["counters"] = srv.set.stats()
        finally:
            srv.close()
        return reqs, info

    # an untimed warm-up of the serving path first (first launches, the host
    # thread, pinned memory first touched)
    serve(False, True, n=max(n_requests // 10, 1), seed_off=3)
    reqs, info = serve(False, True)
    summ = latency_summary(reqs)
    summ.update({"arrival_rate_per_s": rate, "heaps": n_heaps,
                 "max_in_flight": info["max_inflight"],
                 "submitted_while_busy": info["submitted_while_busy"],
                 "refused": info["refused"],
                 "workload": "Poisson arrivals, 1..4096 keys, 50/50 insert/deleteMin, "
                             "256 heaps, k=1024, one persistent serving launch, native host "
                             "loop"})
    if count:
        _, cinfo = serve(True, False)
        span_s = summ["keys"] / summ["keys_per_s"]
        summ["roofline"] = roofline_of(
            node_bytes(cinfo["counters"], 1024, 4), span_s * 1e3,
            "heap_kernel (serving launch)", "node batches loaded + stored (kernel counters, "
            "untimed run of the same requests) over the served span; request keys move "
            "between pinned host memory and the GPU over the host link, not counted")
    return summ


def _timed(torch, fn, reps=3):
    """Median wall time (ms) of fn() with the device synchronized around it;
    fn synchronizes itself (the application runs end when the heap is empty)."""
    fn()
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        ts.append((time.perf_counter() - t0) * 1e3)
    return float(np.median(ts)), r


def run_variant(torch, bottom_up, n=N_KEYS, k=K, ipt=8, steps=3):
    """The headline workload on the other heap variant of the paper: insert-all
    (top-down or bottom-up, Sections 3.3.1 / 3.3.4), then deleteMin-all."""
    from paper_1906_06504_gb300 import inputs
    keys = torch.from_numpy(inputs.keys_u32(inputs.config_seed(2), n).view(np.int32)).cuda()
    ins, dele = [], []
    for _ in range(steps):
        a, b = _phased(torch, keys, k, ipt, bottom_up=bottom_up)
        ins.append(a)
        dele.append(b)
    ins_ms, del_ms = float(np.median(ins)), float(np.median(dele))
    name = "bottom-up" if bottom_up else "top-down"
    return {"workload": "insert-all (%s) + deleteMin-all, 2^26 uniform u32, k=1024" % name,
            "heap": "BU-INS/TD-DEL" if bottom_up else "TD-INS/TD-DEL",
            "value": 2.0 * n / ((ins_ms + del_ms) / 1e3), "unit": UNIT,
            "insert_ms": ins_ms, "delete_ms": del_ms}


def run_apps(torch):
    """The heap as the priority queue of its applications (Section 5.7): SSSP
    on a 1024x1024 grid and an R-MAT graph (2^20 vertices, 2^23 edges), and
    best-first knapsack branch and bound (n = 100, 200, strongly correlated).
    Each result is checked against the oracle (Dijkstra, dynamic program),
    which is timed on one host core beside it."""
    import oracle
    from paper_1906_06504_gb300 import inputs
    from paper_1906_06504_gb300.apps import SSSP, Knapsack
    res = {}
    graphs = [("sssp_grid_1024x1024", inputs.grid_graph(1024, inputs.config_seed(3)), 1024, 1024),
              ("sssp_rmat_2p20", inputs.rmat_graph(20, 8, inputs.config_seed(3)), 1024, 16384)]
    for name, g, k, batch in graphs:
        rowptr, col, w = g
        t0 = time.perf_counter()
        want = oracle.dijkstra(*g)
        cpu_ms = (time.perf_counter() - t0) * 1e3
        d = (torch.from_numpy(rowptr.view(np.int64)).cuda(), torch.from_numpy(col.view(np.int32)).cuda(),
             torch.from_numpy(w.view(np.int32)).cuda())
        with SSSP(rowptr.size - 1, col.size, k=k, batch=batch) as sp:
            ms, (dist, st) = _timed(torch, lambda: sp.run(*d))
            # node traffic of one run, counted by the kernel (separate run)
            hp = sp.heap()
            c0 = hp.stats()
            hp.set_stats(True)
            sp.run(*d)
            hp.set_stats(False)
            c1 = hp.stats()
        exact = bool(np.array_equal(dist.cpu().numpy().view(np.uint32), want))
        assert exact
        keys = st["keys_deleted"] + st["keys_inserted"]
        cnt = {a: c1[a] - c0[a] for a in c1}
        # graph and queue traffic of the relaxation kernels: per visited
        # vertex its row pointers, per scanned edge (col, w) and the distance,
        # per lowering the atomic, the insert-buffer write and read, per
        # deleted key the delete-buffer write and read
        app_b = (st["visited"] * 16 + st["edges"] * 12 + st["keys_inserted"] * 20
                 + st["keys_deleted"] * 16)
        res[name] = {"ms": ms, "heap_keys_per_s": keys / (ms / 1e3), "k": k, "batch": batch,
                     "vertices": int(rowptr.size - 1), "edges": int(col.size), "exact": exact,
                     "cpu_oracle_ms": cpu_ms, "cpu_oracle": "textbook Dijkstra, binary heap, 1 core",
                     "roofline": roofline_of(node_bytes(cnt, k, 8) + app_b, ms,
                                             "heap_kernel + sssp_relax kernels",
                                             "heap node batches (kernel counters, separate run) "
                                             "+ graph and queue traffic of the relaxations"),
                     **st}
    for n, k, batch in ((100, 1024, 65536), (200, 2048, 16384)):
        w, v, cap = inputs.knapsack_instance(n, inputs.config_seed(4))
        t0 = time.perf_counter()
        want = oracle.knapsack_dp(w, v, cap)
        cpu_ms = (time.perf_counter() - t0) * 1e3
        dw = torch.from_numpy(w.view(np.int32)).cuda()
        dv = torch.from_numpy(v.view(np.int32)).cuda()
        with Knapsack(n, k=k, batch=batch) as ks:
            ks.set_launch(items_per_thread=16 if k >= 2048 else 8)
            ms, st = _timed(torch, lambda: ks.run(dw, dv, cap))
            hp = ks.heap()
            c0 = hp.stats()
            hp.set_stats(True)
            ks.run(dw, dv, cap)
            hp.set_stats(False)
            c1 = hp.stats()
        assert st["best"] == want
        keys = st["keys_deleted"] + st["keys_inserted"]
        cnt = {a: c1[a] - c0[a] for a in c1}
        # per expanded node its pool record read and two children written,
        # per heap key the delete/insert buffer write and read
        app_b = st["explored"] * 48 + keys * 16
        res["knapsack_n%d" % n] = {"ms": ms, "heap_keys_per_s": keys / (ms / 1e3), "k": k,
                                   "batch": batch, "capacity": cap, "exact": True,
                                   "cpu_oracle_ms": cpu_ms,
                                   "cpu_oracle": "textbook O(n*C) dynamic program, 1 core",
                                   "roofline": roofline_of(node_bytes(cnt, k, 8) + app_b, ms,
                                                           "heap_kernel + ks_expand kernels",
                                                           "heap node batches (kernel counters, "
                                                           "separate run) + node pool and "
                                                           "buffer traffic"),
                                   **st}
    return res


# ---------------------------------------------------------------------------
# parameter sweeps of Section 5 (bench.py --sweep NAME); one JSON line per point
# ---------------------------------------------------------------------------

def _ev_ms(torch, fn):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def _phased(torch, keys, k, ipt, ctas=0, bottom_up=False):
    """Insert-only then delete-only of `keys` on a fresh heap; (ins ms, del ms)."""
    from paper_1906_06504_gb300.heap import GHeap
    n = keys.numel()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    with GHeap(capacity=n, k=k, bottom_up=bottom_up) as h:
        h.set_launch(ctas=ctas, items_per_thread=ipt)
        h.insert(keys)                    # warm-up pass
        h.delete_min(n, out=out, count=cnt)
        h.sync()
        ins = _ev_ms(torch, lambda: h.insert(keys))
        dele = _ev_ms(torch, lambda: h.delete_min(n, out=out, count=cnt))
        h.sync()
        assert int(cnt.item()) == n
    return ins, dele


def sweep_k_threads(torch, n=1 << 24):
    """Node capacity k x block size (Section 5.4): insert-only and delete-only
    of n uniform keys; the block has 2k/ipt merge threads plus the control and
    release warps."""
    from paper_1906_06504_gb300 import inputs
    keys = torch.from_numpy(inputs.keys_u32(inputs.config_seed(2), n).view(np.int32)).cuda()
    for k in (64, 128, 256, 512, 1024, 2048):
        for ipt in (4, 8, 16):
            threads = max(32, 2 * k // ipt)
            if threads > (512 if ipt == 4 else 256):
                continue
            ins, dele = _phased(torch, keys, k, ipt)
            yield {"sweep": "k_threads", "k": k, "items_per_thread": ipt,
                   "threads": threads + 64, "keys": n, "insert_ms": ins, "delete_ms": dele,
                   "insert_keys_per_s": n / ins * 1e3, "delete_keys_per_s": n / dele * 1e3}


def sweep_ctas(torch, n=1 << 26, k=1024, ipt=8):
    """Thread-block count (Section 5.3): insert-only and delete-only, 2^26 keys."""
    from paper_1906_06504_gb300 import inputs
    keys = torch.from_numpy(inputs.keys_u32(inputs.config_seed(2), n).view(np.int32)).cuda()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for ctas in (16, 32, 64, 128, sms, 2 * sms, 256, 512):
        ins, dele = _phased(torch, keys, k, ipt, ctas=ctas)
        yield {"sweep": "ctas", "ctas": ctas, "k": k, "keys": n, "insert_ms": ins,
               "delete_ms": dele, "insert_keys_per_s": n / ins * 1e3,
               "delete_keys_per_s": n / dele * 1e3, "del_over_ins": dele / ins}


def sweep_distribution(torch, n=1 << 26, k=1024, ipt=8):
    """Key order x insert variant (Section 5.2, Table 1): uniform, ascending,
    descending keys, top-down and bottom-up inserts; all six runs hold one
    multiset, so the deleteMin output must be identical."""
    from paper_1906_06504_gb300 import inputs
    from paper_1906_06504_gb300.heap import GHeap
    first = None
    for variant in ("top-down", "bottom-up"):
        for dist in ("uniform", "ascending", "descending"):
            keys = torch.from_numpy(inputs.keys_u32(inputs.config_seed(2), n, dist)
                                    .view(np.int32)).cuda()
            out = torch.empty(n, dtype=torch.int32, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            with GHeap(capacity=n, k=k, bottom_up=variant == "bottom-up") as h:
                h.set_launch(items_per_thread=ipt)
                ins = _ev_ms(torch, lambda: h.insert(keys))
                dele = _ev_ms(torch, lambda: h.delete_min(n, out=out, count=cnt))
                h.sync()
            same = first is None or bool(torch.equal(out, first))
            if first is None:
                first = out
            yield {"sweep": "distribution", "insert": variant, "dist": dist, "keys": n, "k": k,
                   "insert_ms": ins, "delete_ms": dele, "total_ms": ins + dele,
                   "same_output_as_first": same}
            del keys


def sweep_partial(torch, n=1 << 24, k=1024, ipt=8):
    """Partial insert batches (Section 5.6): a fraction f of the INS ops carry
    a full k-key batch, the others 1..k-1 keys (uniform); same key total."""
    from paper_1906_06504_gb300 import inputs
    from paper_1906_06504_gb300.heap import GHeap, OP_DTYPE, OP_INS
    keys_np = inputs.keys_u32(inputs.config_seed(2) + 300, n)
    d_keys = torch.from_numpy(keys_np.view(np.int32)).cuda()
    for f in (0.0, 0.25, 0.5, 0.75, 1.0):
        rnd = inputs.splitmix64(inputs.config_seed(2) + 301, n // 64 + 16)
        full = ((rnd >> np.uint64(11)).astype(np.float64) / float(1 << 53)) < f
        part = (rnd % np.uint64(k - 1) + np.uint64(1)).astype(np.int64)
        sizes = np.where(full, k, part)
        cs = np.cumsum(sizes)
        m = int(np.searchsorted(cs, n)) + 1
        sizes = sizes[:m].copy()
        sizes[-1] -= int(cs[m - 1]) - n
        sizes = sizes[sizes > 0]
        ops = np.zeros(sizes.size, dtype=OP_DTYPE)
        ops["kind"] = OP_INS
        ops["n"] = sizes
        ops["offset"] = np.concatenate([[0], np.cumsum(sizes)[:-1]])
        d_ops = torch.from_numpy(ops.view(np.uint8).copy()).cuda()
        with GHeap(capacity=n, k=k) as h:
            h.set_launch(items_per_thread=ipt)
            ms = _ev_ms(torch, lambda: h.ops(d_ops, d_keys, None, max_insert_keys=n))
            h.sync()
            assert h.size() == n
        yield {"sweep": "partial", "full_fraction": f, "ops": int(sizes.size), "keys": n,
               "insert_ms": ms, "insert_keys_per_s": n / ms * 1e3}


def sweep_levels(torch, k=1024, ipt=8, pairs=1 << 14):
    """Initial heap utilization (Section 5.5): prefill to L full levels, then
    `pairs` ins-del pairs of k keys from all blocks."""
    for L in (6, 8, 10, 12, 14, 16, 18):
        pre = ((1 << L) - 1) * k
        # the oracle replays the runs up to a 2^24-key prefill (a bigger one
        # takes minutes to replay on one host core)
        r = run_mixed(torch, n_prefill=pre, n_pairs=pairs, k=k, ipt=ipt, seed_off=L,
                      count=False, replay=pre <= (1 << 24))
        yield {"sweep": "levels", "levels": L, "prefill_keys": pre, "pairs": pairs,
               "ms": r["ms"], "keys_per_s": r["value"], "exact": r.get("exact")}


def sweep_serve(torch, n_requests=20000):
    """Serving: arrival rate swept up to saturation; p50/p99 latency."""
    for rate in (10000.0, 50000.0, 100000.0, 200000.0, 400000.0, 800000.0, 1200000.0,
                 1600000.0):
        r = run_serve(torch, n_requests=n_requests if rate < 1e6 else 2 * n_requests, rate=rate,
                      count=False)
        r["sweep"] = "serve_rate"
        yield r


def sweep_apps(torch):
    """The application workloads alone (one line each), e.g. for a profile."""
    for name, r in run_apps(torch).items():
        yield {"sweep": "apps", "app": name, **r}


def sweep_heapset(torch):
    """The heap-set workload of the default run (256 heaps, log-uniform sizes,
    insert-all + deleteMin-all graph replays) at the configuration the
    autotuner picks on GB300 (k = 2048, 16 merge outputs per thread), without
    the tuning launches (for launch lists)."""
    r = run_batched(torch, steps=3, best={"k": 2048, "items_per_thread": 16})
    r.pop("autotune", None)
    yield dict(sweep="heapset", **r)


def sweep_heapset_small(torch):
    """The heap-set workload with every heap at 1/8 of its size (about 15 M
    keys; inputs, outputs and heaps each still larger than L2): a small case
    of the same launches for multi-pass profiler captures."""
    r = run_batched(torch, steps=3, best={"k": 2048, "items_per_thread": 16}, scale=0.125,
                    cpu=False)
    r.pop("autotune", None)
    yield dict(sweep="heapset_small", **r)


SWEEPS = {"apps": sweep_apps, "heapset": sweep_heapset, "heapset_small": sweep_heapset_small, "k_threads": sweep_k_threads, "ctas": sweep_ctas, "distribution": sweep_distribution,
          "partial": sweep_partial, "levels": sweep_levels, "serve_rate": sweep_serve}


def run_sweeps(names):
    import torch
    from paper_1906_06504_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    for name in names:
        for row in SWEEPS[name](torch):
            print(json.dumps(row), flush=True)


def run_gpu(args):
    ws, rank, local = dist_env()
    # the CPU heaps run on other host cores meanwhile; their workers are
    # spawned before this process makes its first CUDA call
    cpu_jobs = None
    if rank == 0 and not args.no_cpu_baseline:
        from paper_1906_06504_gb300 import inputs as _inputs
        cpu_jobs = CpuBaselines(args.keys, _inputs.config_seed(2))
    import torch
    from paper_1906_06504_gb300 import build, inputs
    build.build()
    from paper_1906_06504_gb300.heap import GHeap

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    n, k = args.keys, args.k
    keys_np = inputs.keys_u32(inputs.config_seed(2) + rank, n)
    keys = torch.from_numpy(keys_np.view(np.int32)).cuda()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    bottom_up = not args.top_down
    heap = GHeap(capacity=n, k=k, bottom_up=bottom_up)
    heap.set_launch(ctas=args.ctas, items_per_thread=args.ipt)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        heap.insert(keys)
        if ev is not None:
            ev[1].record(stream)
        heap.delete_min(n, out=out, count=cnt)
        if ev is not None:
            ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    heap.sync()
    # correctness of the timed configuration (cheap property check)
    assert int(cnt.item()) == n

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            step(evs[i])
        t_end.record(stream)
        torch.cuda.synchronize()
    barrier()
    heap.sync()
    ms = t_start.elapsed_time(t_end)
    ins_ms = [e[0].elapsed_time(e[1]) for e in evs]
    del_ms = [e[1].elapsed_time(e[2]) for e in evs]
    ms = max_over_ranks(ms, dist)
    value = whole_job_rate(2 * n, args.steps, ws, ms)

    # node traffic of one step, counted by the kernel (separate untimed run)
    cheap = GHeap(capacity=n, k=k, stats=True, bottom_up=bottom_up)
    cheap.set_launch(ctas=args.ctas, items_per_thread=args.ipt)
    cheap.insert(keys)
    cheap.sync()
    st_ins = cheap.stats()
    cheap.delete_min(n, out=out, count=cnt)
    cheap.sync()
    st_all = cheap.stats()
    cheap.close()
    st_del = {a: st_all[a] - st_ins[a] for a in st_all}
    node_b = k * 4
    del_bytes = (st_del["node_loads"] + st_del["node_stores"]) * node_b + n * 4
    ins_bytes = (st_ins["node_loads"] + st_ins["node_stores"]) * node_b + n * 4
    del_avg_ms = float(np.mean(del_ms))
    ins_avg_ms = float(np.mean(ins_ms))
    dom = "delete" if del_avg_ms >= ins_avg_ms else "insert"
    dom_bytes, dom_ms = (del_bytes, del_avg_ms) if dom == "delete" else (ins_bytes, ins_avg_ms)
    peak, peak_kind = peaks()
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9

    # end to end through the C ABI from pinned host memory
    host_in = torch.from_numpy(keys_np.view(np.int32)).pin_memory()
    host_out = torch.empty(n, dtype=torch.int32).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    heap.sync()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        keys.copy_(host_in, non_blocking=True)
        heap.insert(keys)
        heap.delete_min(n, out=out, count=cnt)
        host_out.copy_(out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    # the whole output of the last end-to-end step is the sorted input
    assert np.array_equal(host_out.numpy().view(np.uint32), np.sort(keys_np))
    e2e_ms = max_over_ranks(e2e_ms, dist)
    e2e_value = whole_job_rate(2 * n, e2e_steps, ws, e2e_ms)

    heap.close()
    extras = {}
    if not args.skip_extras:
        extras["mixed"] = run_mixed(torch, ipt=args.ipt)
        extras["batched"] = run_batched(torch, tune=not args.no_tune)
        extras["serve"] = {"low_load": run_serve(torch, rate=50000.0),
                           "near_saturation": run_serve(torch, rate=800000.0)}
        extras["other_variant"] = run_variant(torch, not bottom_up, ipt=args.ipt)
        extras["apps"] = run_apps(torch)
    cpu = cpu_jobs.result() if cpu_jobs is not None else None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "insert-all + deleteMin-all, 2^26 uniform u32 keys, k=1024",
                       "heap": "BU-INS/TD-DEL (Section 3.3.4)" if bottom_up
                               else "TD-INS/TD-DEL (Section 3.3.1)",
                       "keys": n, "k": k, "merge_threads_per_block": 2 * k // args.ipt,
                       "threads_per_block": 2 * k // args.ipt + 64,
                       "ctas": args.ctas or "one per SM",
                       "l2": "inputs and heap (256 MB each) exceed the 126 MB L2",
                       "insert_ms": ins_avg_ms, "delete_ms": del_avg_ms},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": measured_traffic(dom, n, k, args.ctas, bottom_up)
                         if args.ipt == 8 else None,
                         "peak_kind": peak_kind,
                         "kernel": "heap_kernel (%s-all launch)" % dom,
                         "algorithmic_bytes": dom_bytes},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * 4,
                    "d2h_bytes_per_step": n * 4},
            "gpu_launches": 2 * args.steps,
            "clocks": clk.summary(),
            "stats_delete": st_del, "stats_insert": st_ins,
            "root_hold_ns_per_op": {
                "insert": st_ins["root_hold_ns"] / max(1, st_ins["ins_ops"]),
                "delete": st_del["root_hold_ns"] / max(1, st_del["del_ops"])},
        }
        line.update(extras)
        if "batched" in extras:
            line["batched"]["vs_plain"] = extras["batched"]["value"] / value
        if "serve" in extras:
            sat = line["serve"]["near_saturation"]
            sat["vs_plain"] = sat["keys_per_s"] / value
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--keys", type=int, default=N_KEYS)
    ap.add_argument("--k", type=int, default=K)
    ap.add_argument("--ctas", type=int, default=0)
    ap.add_argument("--ipt", type=int, default=8)
    ap.add_argument("--top-down", action="store_true",
                    help="headline on the TD-INS/TD-DEL heap (default: BU-INS/TD-DEL)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-extras", action="store_true",
                    help="only the headline single-heap workload")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--sweep", action="append", choices=sorted(SWEEPS),
                    help="run a Section 5 parameter sweep instead of the benchmark "
                         "(one JSON line per point; may repeat)")
    args = ap.parse_args()
    if args.sweep:
        run_sweeps(args.sweep)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
