#!/usr/bin/env python3
"""Benchmark of the PI batch path on GB300: Mqueries/s and the HBM roofline fraction.

Default workload: the skewed configuration -- 2^27 distinct uniform uint64 keys with
value = splitmix64(key), promotion p = 1/4, batches of 2^22 queries with Zipf(0.99)
keys over the key set, 90% search / 5% insert / 5% delete, index layer rebuilt after
every batch that changes it. One "step" = one pi_execute_batch: pack + sort, descent,
ownership + apply, merge, layout, rebuild.

Inputs are synthetic and seeded (paper_1601_00159_gb300/workloads.py), generated on
the host outside the timed region and resident in HBM before it starts. The storage
layer (2 GB) and the cycled batch inputs (32 x 71 MB) are larger than L2, so no L2
flush is inserted between steps.

Output: one JSON line (rank 0). `--impl reference` times the CPU oracle instead (the
paper ships no code; the oracle is the only reference implementation here).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1601_00159_gb300 import workloads as wl  # noqa: E402

METRIC = "Mqueries/s and % of HBM roofline on 1 GB300; p50/p99 latency in serving loop"
UNIT = "Mqueries/s"
# Per-kernel DRAM bytes and L2 hit rates of the batch path on the skewed workload, from
# one ncu capture per kernel on a smaller index (see the summary beside it); the file
# records a digest of the sources the captures were taken with.
KERNEL_PROFILE = os.path.join(ROOT, "profiles", "kernels_skewed.json")

WORKLOADS = {
    "skewed": dict(fn=wl.skewed, n=1 << 27, q=1 << 22,
                   desc="plain PI, skewed: 2^27 uint64 keys/values, p=1/4, batches of 2^22 Zipf(0.99) "
                        "queries, 90% search / 5% insert / 5% delete, rebuild after each batch"),
    "mid": dict(fn=wl.mid, n=1 << 24, q=1 << 20,
                desc="plain PI, mid: 2^24 uint64 keys, p=1/4, batches of 2^20 queries, 50% search / "
                     "50% insert of new uniform keys, rebuild after each batch"),
    "tiny": dict(fn=wl.tiny, n=1 << 16, q=1 << 14,
                 desc="plain PI, tiny: 2^16 uint64 keys, p=1/2, one batch of 2^14 searches (half hits)"),
    "batching": dict(fn=wl.batching, n=None, q=None,
                     desc="batching: 256 independent indices, sizes log-uniform in [2^10,2^20] uint64 keys "
                          "(p=1/4), each with its own batch of log-uniform [2^8,2^16] queries, 80% search "
                          "(half hits) / 20% insert of new uniform keys; one CUDA-graph launch per step"),
    "serving": dict(fn=wl.serving, n=1 << 26, q=None,
                    desc="serving: resident 2^26-key uint64 index (p=1/4); Poisson-arrival requests of 1..4096 "
                         "queries (log-uniform), 95% search / 5% insert, Zipf 0.9 keys; coalesced batches of at "
                         "most 2^20 queries, 3 in flight; p50/p99 request latency at 50% and 90% of the measured capacity"),
    "range": dict(fn=None, n=1 << 24, q=None,
                  desc="range search: 2^24 distinct uniform uint64 keys (p=1/4); batches of 2^16 range queries "
                       "whose spans hold on average g = 1, 10, 100, 1000 keys (the paper's granularity); "
                       "value at g = 100"),
}
TUNING = os.path.join(ROOT, "paper_1601_00159_gb300", "multi_tuning.json")


def tuned_classes():
    """The size-class table the autotuner wrote, or None (built-in table)."""
    try:
        with open(TUNING) as f:
            return [tuple(c) for c in json.load(f)["classes"]]
    except Exception:
        return None


def tuned_lowest(nodes):
    """The batching form's tuned lowest built level for an index of `nodes` keys (its size
    class's), or 0 (the library's automatic choice)."""
    try:
        with open(TUNING) as f:
            d = json.load(f)
        lg = max(0, int(np.ceil(np.log2(max(nodes, 1)))))
        for hi in sorted(int(h) for h in d.get("lowest_level", {})):
            if lg <= hi:
                return int(d["lowest_level"][str(hi)])
    except Exception:
        pass
    return 0


PLAIN_TUNING = os.path.join(ROOT, "paper_1601_00159_gb300", "plain_tuning.json")


def tuned_plain(keys):
    """The plain path's tuned configuration for an index of `keys` keys: the class of the
    nearest tuned size, or {} (defaults)."""
    try:
        with open(PLAIN_TUNING) as f:
            cl = json.load(f)["classes"]
        lg = float(np.log2(max(keys, 1)))
        best = min(cl, key=lambda c: abs(c["log2_keys"] - lg))
        return dict(best["chosen"]) if abs(best["log2_keys"] - lg) <= 1 else {}
    except Exception:
        return {}


# The sources of the single-index batch path (the kernels a capture of the skewed
# workload measures, and the host code that launches them).
BATCH_PATH_SOURCES = ("common.cuh", "sort.cu", "descend.cu", "apply.cu", "rebuild.cu", "relevel.cu", "pi.cu")


def source_digest():
    """sha256 prefix of the batch path's CUDA sources and the C header: a DRAM capture
    counts only for the kernels it measured."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1601_00159_gb300", "csrc")
    for name in BATCH_PATH_SOURCES:
        h.update(name.encode())
        h.update(open(os.path.join(csrc, name), "rb").read())
    h.update(open(os.path.join(ROOT, "include", "pi.h"), "rb").read())
    return h.hexdigest()[:16]


def kernel_profile(workload, keys, queries):
    """(DRAM bytes per batch scaled to this run, per-kernel table, note) from the committed
    per-kernel ncu captures of this workload, or (None, None, why). Kernels whose traffic
    follows the index size (the rebuild's and the merge's) are scaled by the key count,
    the others by the batch size; the capture's smaller index keeps more of itself in L2,
    so the scaled sum is a lower bound of the traffic at this size."""
    try:
        d = json.load(open(KERNEL_PROFILE))
    except (OSError, ValueError):
        return None, None, "no per-kernel ncu capture"
    if d.get("workload") != workload:
        return None, None, f"the captures are of workload {d.get('workload')}"
    if d.get("digest") != source_digest():
        return None, None, "kernel sources changed since the ncu captures"
    ck, cq = d["capture"]["keys"], d["capture"]["batch"]
    total = 0.0
    for k in d["kernels"].values():
        f = keys / ck if k["scales_with"] == "index" else queries / cq
        total += k["dram_bytes"] * k["launches_per_batch"] * f
    return total, d["kernels"], (f"per-kernel ncu captures at {ck} keys and batches of {cq}, scaled "
                                 f"to this run (a lower bound: the smaller index is more L2-resident)")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------------
# Algorithmic bytes (the method's own traffic, counted per batch from its inputs and
# the index sizes; one 32-byte sector per random access).
def algorithmic_bytes(q, q_ins, distinct, hits, writes, live_after, level_sizes, l2_bytes, p):
    """The method's own bytes per batch, by the model of the paper's Section 5 as the
    hot-path table states it (one 32-byte sector per random access): batch I/O; one key
    and one down sector per distinct key and index level too large to stay in L2 (every
    level from 2 up, as the paper lays the index out); one key sector per distinct key
    and a value sector per hit in the storage layer, plus key, value and meta sectors per
    written key; and the paper's full rebuild: a 9-byte scan of every node and 12 bytes
    per index entry written, N' p / (1 - p) entries for N' live keys."""
    io = q * (1 + 8 + 16) + q_ins * 8
    trav = sum(distinct * 64 for l, n_l in enumerate(level_sizes) if l >= 2 and 12 * n_l > l2_bytes / 2)
    store = distinct * 32 + hits * 32 + writes * 96
    rebuild = 9 * live_after + 12 * live_after * p / (1 - p)
    return dict(io=io, traversal=trav, storage=store, rebuild=rebuild, total=io + trav + store + rebuild)


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    def __init__(self, gpu_index: int, period_ms: int = 100):
        self.gpu = gpu_index
        self.period = period_ms
        self.proc = None
        self.path = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", f"-lms={self.period}"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = np.array([float(r[1]) for r in rows])
        mx = float(rows[0][2])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = sm[sm > 0.5 * mx] if (sm > 0.5 * mx).any() else sm
        return {"sm_mhz": float(np.median(loaded)), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3] not in ("", "[N/A]"))}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------------
def cpu_baseline(w, batch0, budget_s: float = 20.0):
    """Time the oracle (single-threaded, as it stands) on a bounded sample: build over the
    full initial key set (untimed), then apply the first queries of the first batch."""
    import oracle
    oracle.build()
    t0 = time.time()
    orc = oracle.Oracle(w.keys, w.vals, w.promote_p, w.hash_seed)
    build_s = time.time() - t0
    q = len(batch0)
    done, elapsed, chunk = 0, 0.0, 1 << 14
    while done < q and elapsed < budget_s:
        c = min(chunk, q - done)
        t = time.perf_counter()
        orc.execute(batch0.ops[done:done + c], batch0.keys[done:done + c], batch0.vals[done:done + c])
        elapsed += time.perf_counter() - t
        done += c
        chunk = min(chunk * 2, 1 << 20)
    orc.close()
    return {"value": done / elapsed / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {done} queries of batch 0 on the full {len(w.keys)}-key index "
                      f"({elapsed:.1f} s timed; oracle build {build_s:.1f} s untimed)"}


def run_reference_batching(args):
    """The oracle on the batching workload: the first indices (bounded sample, built
    untimed), each step applying one round of their batches."""
    import oracle
    oracle.build()
    spec = WORKLOADS["batching"]
    w = wl.batching()
    take = 8
    orcs = [oracle.Oracle(w.keys[i], w.vals[i], w.promote_p, w.hash_seeds[i]) for i in range(take)]
    # a fresh round per step (its inserts are new keys), as in the GPU arm; at most 64
    n_rounds = min(args.warmup + args.steps, 64)
    rounds = [w.batches(r)[:take] for r in range(n_rounds)]
    for s_ in range(args.warmup):
        for o, b in zip(orcs, rounds[s_ % n_rounds]):
            o.execute(b.ops, b.keys, b.vals)
    t = time.perf_counter()
    done = 0
    for s_ in range(args.steps):
        for o, b in zip(orcs, rounds[(args.warmup + s_) % n_rounds]):
            o.execute(b.ops, b.keys, b.vals)
            done += len(b)
    el = time.perf_counter() - t
    v = done / el / 1e6
    for o in orcs:
        o.close()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": "batching", "desc": spec["desc"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"the batches of the first {take} of {len(w.keys)} indices per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_serving(args):
    """The oracle on the serving workload: built over the 2^26 keys (untimed), each step
    applying one bounded slice of the request stream in arrival order."""
    import oracle
    oracle.build()
    spec = WORKLOADS["serving"]
    w = wl.serving(nreq=4000)
    orc = oracle.Oracle(w.keys, w.vals, w.promote_p, w.hash_seed)
    per = min(len(w.ops) // max(args.steps + args.warmup, 1), 1 << 18)
    t = None
    for s_ in range(args.warmup + args.steps):
        if s_ == args.warmup:
            t = time.perf_counter()
        a = s_ * per
        orc.execute(w.ops[a:a + per], w.qkeys[a:a + per], w.qvals[a:a + per])
    el = time.perf_counter() - t
    v = args.steps * per / el / 1e6
    orc.close()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": "serving", "desc": spec["desc"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{per} queries of the request stream per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference_range(args):
    """The oracle on the range workload: ranges of granularity 100 over the 2^24 keys
    (built untimed), a bounded slice of 4096 ranges per step."""
    import oracle
    oracle.build()
    keys = np.sort(wl.distinct_keys(6, np.arange(1 << 24)))
    orc = oracle.Oracle(keys, wl.splitmix64(keys), 0.25, 6)
    lo, hi = range_bounds(keys, 4096 * (args.warmup + args.steps), 100, 107)
    t = None
    for s_ in range(args.warmup + args.steps):
        if s_ == args.warmup:
            t = time.perf_counter()
        orc.range(lo[s_ * 4096:(s_ + 1) * 4096], hi[s_ * 4096:(s_ + 1) * 4096])
    el = time.perf_counter() - t
    v = args.steps * 4096 / el / 1e6
    orc.close()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mranges/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": "range", "desc": WORKLOADS["range"]["desc"]},
            "cpu_baseline": {"value": v, "unit": "Mranges/s", "cores": 1, "kind": "oracle",
                             "sample": "4096 ranges of granularity 100 per step"},
            "e2e": {"value": v, "unit": "Mranges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference(args, ws, rank):
    if rank != 0:
        return
    if args.workload == "batching":
        return run_reference_batching(args)
    if args.workload == "serving":
        return run_reference_serving(args)
    if args.workload == "range":
        return run_reference_range(args)
    spec = WORKLOADS[args.workload]
    w = spec["fn"]()
    batches = list(w.batches()) if callable(w.batches) else list(w.batches)
    import oracle
    oracle.build()
    orc = oracle.Oracle(w.keys, w.vals, w.promote_p, w.hash_seed)
    per_step = min(len(batches[0]), 1 << 18)  # bounded sample per step
    for s in range(args.warmup):
        b = batches[s % len(batches)]
        orc.execute(b.ops[:per_step], b.keys[:per_step], b.vals[:per_step])
    t = time.perf_counter()
    for s in range(args.steps):
        b = batches[(args.warmup + s) % len(batches)]
        orc.execute(b.ops[:per_step], b.keys[:per_step], b.vals[:per_step])
    el = time.perf_counter() - t
    v = args.steps * per_step / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": args.workload, "desc": spec["desc"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} queries of each batch, applied in arrival order"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batching(args, ws, rank, local):
    """The batching workload: one pi_multi_execute per step over every index's batch, beside the same
    batches run by looping the single-index path over the indices."""
    import torch
    from paper_1601_00159_gb300 import Index, MultiSet, build, load_library
    build.build()
    load_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec = WORKLOADS["batching"]
    t_gen = time.time()
    w = wl.batching(seed=4 + rank)
    # Every call takes a round of batches no call has applied before, so its 20% inserts
    # of uniform keys are new keys (a merge and a rebuild for every index), as the
    # configuration states: the timed calls, then the plain-path loop, then the
    # host-buffer calls. Runs longer than kMaxRounds distinct rounds reuse the timed ones.
    kMaxRounds = 64
    loop_steps = 2
    e2e_steps = max(3, min(args.steps, 10))
    timed_rounds = min(args.warmup + args.steps, kMaxRounds)
    first_loop = timed_rounds
    first_e2e = first_loop + 1 + loop_steps
    n_rounds = first_e2e + 2 + e2e_steps
    host_rounds = [w.batches(r) for r in range(n_rounds)]
    gen_s = time.time() - t_gen
    count = len(w.keys)
    qs = [len(b) for b in host_rounds[0]]
    qtot = int(sum(qs))
    total_rounds = n_rounds + max(0, args.warmup + args.steps - timed_rounds)
    idxs = []
    t = time.time()
    for i in range(count):
        k = torch.from_numpy(w.keys[i].view(np.int64)).to(dev)
        v = torch.from_numpy(w.vals[i].view(np.int64)).to(dev)
        cap = len(w.keys[i]) + qs[i] * total_rounds // 4 + 4096
        cfg = {"storage_capacity": cap}
        low = tuned_lowest(len(w.keys[i]))
        if low:
            cfg["lowest_level"] = low
        idxs.append(Index(k, v, w.promote_p, w.hash_seeds[i], cfg))
    create_s = time.time() - t
    classes = tuned_classes()
    ms = MultiSet(idxs, classes)

    def pack(rnd):
        ops = np.concatenate([b.ops for b in rnd])
        keys = np.concatenate([b.keys for b in rnd]).view(np.int64)
        vals = np.concatenate([b.vals for b in rnd]).view(np.int64)
        return ops, keys, vals

    offs = np.concatenate([[0], np.cumsum(qs)])
    def upload(rnd):
        o, k, v = pack(rnd)
        return torch.from_numpy(o).to(dev), torch.from_numpy(k).to(dev), torch.from_numpy(v).to(dev)

    dev_rounds = [upload(rnd) for rnd in host_rounds[:timed_rounds]]
    results = torch.empty((qtot, 2), dtype=torch.int64, device=dev)

    def descs(o, k, v, res):
        return [(i, o[offs[i]:offs[i + 1]], k[offs[i]:offs[i + 1]], v[offs[i]:offs[i + 1]],
                 res[offs[i]:offs[i + 1]]) for i in range(count)]

    stream = torch.cuda.current_stream()
    # descriptor arrays built (and checked) once per round, outside the timed region
    step_descs = [ms.prepare(descs(*dr, results)) for dr in dev_rounds]
    for s_ in range(args.warmup):
        ms.execute(step_descs[s_ % timed_rounds])
    torch.cuda.synchronize()
    launches_per_call = ms.kernels_per_call()
    barrier(ws)
    with ClockSampler(local) as clk:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for s_ in range(args.steps):
            ms.execute(step_descs[(args.warmup + s_) % timed_rounds])
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    ms_total = reduce_max(ev0.elapsed_time(ev1), ws)
    ms_step = ms_total / args.steps
    value = ws * qtot * args.steps / (ms_total * 1e-3) / 1e6

    del step_descs, dev_rounds
    # fresh rounds through the single-index path, one index after another
    loop_descs = [descs(*upload(host_rounds[first_loop + j]), results) for j in range(1 + loop_steps)]
    for (i, o, k, v, r) in loop_descs[0]:
        idxs[i].execute(o, k, v, r)
    torch.cuda.synchronize()
    l0 = [ix.info()["kernel_launches"] for ix in idxs]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s_ in range(loop_steps):
        for (i, o, k, v, r) in loop_descs[1 + s_]:
            idxs[i].execute(o, k, v, r)
    for ix in idxs:
        ix.flush(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    loop_ms = reduce_max(e0.elapsed_time(e1), ws) / loop_steps
    loop_launches = (sum(ix.info()["kernel_launches"] for ix in idxs) - sum(l0)) // loop_steps
    loop_value = ws * qtot / (loop_ms * 1e-3) / 1e6

    del loop_descs
    # e2e: each step copies its packed (fresh) round from pinned host memory and reads the
    # results back, double-buffered: step s + 1's inputs go in on a copy stream while step s
    # runs, and step s's results come out on another while step s + 1 runs (the pattern the
    # plain path's host-buffer entry point uses inside the library)
    hp = []
    for rnd in host_rounds[first_e2e:]:
        o, k, v = pack(rnd)
        hp.append((torch.from_numpy(o).pin_memory(), torch.from_numpy(k.copy()).pin_memory(),
                   torch.from_numpy(v.copy()).pin_memory()))
    hres = [torch.empty((qtot, 2), dtype=torch.int64).pin_memory() for _ in range(2)]
    dbuf = [[torch.empty(qtot, dtype=torch.uint8, device=dev), torch.empty(qtot, dtype=torch.int64, device=dev),
             torch.empty(qtot, dtype=torch.int64, device=dev)] for _ in range(2)]
    dres = [results, torch.empty_like(results)]
    e2e_descs = [ms.prepare(descs(dbuf[j][0], dbuf[j][1], dbuf[j][2], dres[j])) for j in range(2)]
    cin, cout = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    for j in range(2):
        ev_done[j].record(stream)
        ev_out[j].record(stream)

    def e2e_step(s_, src):
        j = s_ & 1
        with torch.cuda.stream(cin):
            cin.wait_event(ev_done[j])  # the slot's inputs were read by its previous call
            for t in range(3):
                dbuf[j][t].copy_(src[t], non_blocking=True)
            ev_in[j].record(cin)
        stream.wait_event(ev_in[j])
        stream.wait_event(ev_out[j])  # the slot's previous results were copied out
        ms.execute(e2e_descs[j], stream=stream)
        ev_done[j].record(stream)
        with torch.cuda.stream(cout):
            cout.wait_event(ev_done[j])
            hres[j].copy_(dres[j], non_blocking=True)
            ev_out[j].record(cout)

    for s_ in range(2):
        e2e_step(s_, hp[s_])
    torch.cuda.synchronize()
    e0.record(stream)
    for s_ in range(e2e_steps):
        e2e_step(s_, hp[2 + s_])
    for j in range(2):
        stream.wait_event(ev_out[j])
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = reduce_max(e0.elapsed_time(e1), ws) / e2e_steps
    e2e_value = ws * qtot / (e2e_ms * 1e-3) / 1e6

    # algorithmic bytes of one step (every index: batch I/O, storage accesses, merge of the
    # new nodes, rebuild), after the timed steps
    hbm, peak_kind = measured_peaks()
    infos = [ix.info() for ix in idxs]
    ins = sum(int((b.ops == wl.OP_INSERT).sum()) for b in host_rounds[0])
    nodes = sum(inf["size"] for inf in infos)
    entries = sum(sum(inf["level_size"][inf["bottom_built"]:]) for inf in infos)
    io = qtot * (1 + 8 + 16) + ins * 8
    store = qtot * 32 + ins * 96
    merge = 2 * 17 * nodes
    rebuild = 9 * nodes + 12 * entries
    ab = io + store + merge + rebuild
    achieved = ab / (ms_step * 1e-3) / 1e9
    for ix in idxs:
        assert ix.status() == 0, "device error status"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "batching", "desc": spec["desc"], "indices": count, "queries_per_step": qtot,
                   "keys_total": int(sum(len(k) for k in w.keys)), "classes": classes or "built-in",
                   "distinct_rounds": n_rounds, "timed_rounds_distinct": timed_rounds,
                   "inserts": "new keys in every call (each call takes a round not applied before)",
                   "parallelism": f"replicas{ws}" if ws > 1 else "single",
                   "l2_flush": "none: the indices (0.7 GB of storage) and the rounds exceed L2"},
        "roofline": {"bound": "hbm", "kernel": "k_multi", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_source": peak_kind, "traffic": None,
                     "launches_per_step": launches_per_call, "ms_per_launch": ms_step,
                     "algorithmic_bytes_per_launch": ab,
                     "bytes_model": "per index: Q*25 + Q_ins*8 I/O, Q*32 + Q_ins*96 storage, "
                                    "2*17 B per node merge, 9 B per node + 12 B per index entry rebuild"},
        "plain_loop": {"value": loop_value, "unit": UNIT, "ms_per_step": loop_ms,
                       "gpu_launches_per_step": loop_launches,
                       "note": "the same batches, pi_execute_batch index after index on one stream"},
        "speedup_vs_plain_loop": value / loop_value,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": qtot * 17, "d2h_bytes_per_step": qtot * 16,
                "steps": e2e_steps, "pattern": "two buffer slots: copies in and out on their own streams, "
                                               "overlapping the neighbouring calls"},
        "gpu_launches": launches_per_call * args.steps,
        "clocks": clk.summary(),
        "index": {"nodes": nodes, "index_entries": entries, "create_s": create_s, "gen_s": gen_s},
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_multi(w, host_rounds[0], args.cpu_budget)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ms.close()
    for ix in idxs:
        ix.close()


def run_serving(args, ws, rank, local):
    """The serving workload: the server under a saturating burst (capacity), then under Poisson
    arrivals at 50% and 90% of that capacity (latency), beside one request per
    pi_execute_batch."""
    import torch
    from paper_1601_00159_gb300 import Index, Server, build, load_library
    build.build()
    load_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec = WORKLOADS["serving"]
    t = time.time()
    nreq = 40000
    w = wl.serving(seed=5 + rank, nreq=nreq)
    gen_s = time.time() - t
    offs = np.concatenate([[0], np.cumsum(w.sizes.astype(np.int64))])
    t = time.time()
    idx = Index(torch.from_numpy(w.keys.view(np.int64)).to(dev), torch.from_numpy(w.vals.view(np.int64)).to(dev),
                w.promote_p, w.hash_seed)
    torch.cuda.synchronize()
    create_s = time.time() - t
    srv = Server(idx, max_batch=1 << 20, slots=3)
    # warm-up, then capacity: every request arrives at once
    warm = 2000
    srv.replay(w.ops, w.qkeys, w.qvals, w.sizes[:warm], np.zeros(warm), want_results=False)
    srv.stats(reset=True)
    half = nreq // 2
    a, b = offs[warm], offs[warm + half]
    t = time.perf_counter()
    srv.replay(w.ops[a:b], w.qkeys[a:b], w.qvals[a:b], w.sizes[warm:warm + half], np.zeros(half), want_results=False)
    sat_s = time.perf_counter() - t
    sat = srv.stats(reset=True)
    capacity = (b - a) / sat_s / 1e6
    # latency: Poisson arrivals at 50% and then 90% of capacity, each on half the rest
    rest = nreq - warm - half
    l0 = idx.info()["kernel_launches"]
    runs = {}
    r0 = warm + half
    with ClockSampler(local) as clk:
        for frac, r1 in ((0.5, warm + half + rest // 2), (0.9, nreq)):
            a2, b2 = offs[r0], offs[r1]
            rate = frac * capacity * 1e6 / float(w.sizes[r0:r1].mean())  # requests per second
            gaps = -np.log(np.maximum(wl.uniform01(wl.stream_seed(5, 77 + int(frac * 10)), 0, r1 - r0), 1e-12)) / rate
            t = time.perf_counter()
            _, lat = srv.replay(w.ops[a2:b2], w.qkeys[a2:b2], w.qvals[a2:b2], w.sizes[r0:r1], np.cumsum(gaps),
                                want_results=False)
            run_s = time.perf_counter() - t
            st = srv.stats(reset=True)
            runs[frac] = dict(value=(b2 - a2) / run_s / 1e6, requests=r1 - r0, queries=int(b2 - a2), rate=rate,
                              run_s=run_s, p50_ms=float(np.percentile(lat, 50)) * 1e3,
                              p99_ms=float(np.percentile(lat, 99)) * 1e3, max_ms=float(lat.max()) * 1e3,
                              batches=st["batches"], mean_batch=st["mean_batch"], max_in_flight=st["max_in_flight"])
            r0 = r1
    srv.close()
    launches = idx.info()["kernel_launches"] - l0
    hi = runs[0.9]
    value = hi["value"]
    # the plain path without coalescing: one request per batch, host buffers, synchronous
    sample = 300
    hres = torch.empty((4096, 2), dtype=torch.int64).pin_memory()
    pops = torch.from_numpy(w.ops[:offs[sample]].copy()).pin_memory()
    pkeys = torch.from_numpy(w.qkeys[:offs[sample]].view(np.int64).copy()).pin_memory()
    pvals = torch.from_numpy(w.qvals[:offs[sample]].view(np.int64).copy()).pin_memory()
    plat = []
    t = time.perf_counter()
    for i in range(sample):
        x, y = offs[i], offs[i + 1]
        t1 = time.perf_counter()
        idx.execute_host(pops[x:y], pkeys[x:y], pvals[x:y], hres[: y - x])
        torch.cuda.synchronize()
        plat.append(time.perf_counter() - t1)
    per_req_s = time.perf_counter() - t
    per_req_value = offs[sample] / per_req_s / 1e6
    # the plain path on batches of the size the server coalesced under the burst: the same
    # request stream cut into batches of that many queries, through the host-buffer entry
    # point (which overlaps one batch's copies with the next one's kernels)
    cb = int(max(1, round(sat["mean_batch"])))
    nb_c = max(3, min(20, int(offs[-1] // cb) - 1))
    cops = torch.from_numpy(w.ops[:cb * (nb_c + 2)].copy()).pin_memory()
    ckeys = torch.from_numpy(w.qkeys[:cb * (nb_c + 2)].view(np.int64).copy()).pin_memory()
    cvals = torch.from_numpy(w.qvals[:cb * (nb_c + 2)].view(np.int64).copy()).pin_memory()
    cres = torch.empty((cb * (nb_c + 2), 2), dtype=torch.int64).pin_memory()
    for j in range(2):
        idx.execute_host(cops[j * cb:(j + 1) * cb], ckeys[j * cb:(j + 1) * cb], cvals[j * cb:(j + 1) * cb],
                         cres[j * cb:(j + 1) * cb])
    torch.cuda.synchronize()
    t = time.perf_counter()
    for j in range(2, nb_c + 2):
        idx.execute_host(cops[j * cb:(j + 1) * cb], ckeys[j * cb:(j + 1) * cb], cvals[j * cb:(j + 1) * cb],
                         cres[j * cb:(j + 1) * cb])
    idx.flush()
    torch.cuda.synchronize()
    coalesced_value = nb_c * cb / (time.perf_counter() - t) / 1e6
    hbm, peak_kind = measured_peaks()
    info = idx.info()
    assert idx.status() == 0
    idx.close()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": int(hi["requests"]),
        "warmup": warm, "ms_per_step": hi["run_s"] / hi["requests"] * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "serving", "desc": spec["desc"], "keys": len(w.keys), "requests": int(hi["requests"]),
                   "queries": hi["queries"], "mean_request": float(w.sizes.mean()), "arrival_rate_per_s": hi["rate"],
                   "load": "90% of the capacity measured under a burst (value); 50% in latency_50",
                   "step": "one request", "parallelism": f"replicas{ws}" if ws > 1 else "single",
                   "l2_flush": "none: the 2^26-key index (1.1 GB storage) exceeds L2"},
        "latency": {"p50_ms": hi["p50_ms"], "p99_ms": hi["p99_ms"], "max_ms": hi["max_ms"], "batches": hi["batches"],
                    "mean_batch": hi["mean_batch"], "max_in_flight": hi["max_in_flight"], "load": 0.9,
                    "measured_from": "scheduled arrival to results in host memory"},
        "latency_50": dict(runs[0.5], load=0.5),
        "capacity": {"value": capacity, "unit": UNIT, "batches": sat["batches"], "mean_batch": sat["mean_batch"],
                     "p99_ms": sat["p99_s"] * 1e3, "note": "every request arriving at once"},
        "plain_coalesced": {"value": coalesced_value, "unit": UNIT, "batch": cb, "batches": nb_c,
                            "note": "pi_execute_batch_host on the request stream cut into batches of the size the "
                                    "server coalesced under the burst (host arrays, pipelined copies)"},
        "plain_per_request": {"value": per_req_value, "unit": UNIT, "requests": sample,
                              "p50_ms": float(np.percentile(plat, 50)) * 1e3,
                              "p99_ms": float(np.percentile(plat, 99)) * 1e3,
                              "note": "pi_execute_batch_host per request, no coalescing, synchronous"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": float(w.sizes.mean()) * 17,
                "d2h_bytes_per_step": float(w.sizes.mean()) * 16,
                "note": "the server path is end to end: host requests in, host results out"},
        "roofline": None,
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "index": {"size": info["size"], "live": info["live"], "create_s": create_s, "gen_s": gen_s},
    }
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t = time.time()
        orc = oracle.Oracle(w.keys, w.vals, w.promote_p, w.hash_seed)
        build_s = time.time() - t
        done, el = 0, 0.0
        while done < offs[-1] and el < args.cpu_budget:
            c = int(min(1 << 18, offs[-1] - done))
            t = time.perf_counter()
            orc.execute(w.ops[done:done + c], w.qkeys[done:done + c], w.qvals[done:done + c])
            el += time.perf_counter() - t
            done += c
        orc.close()
        line["cpu_baseline"] = {"value": done / el / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"the first {done} queries of the request stream in arrival order "
                                          f"({el:.1f} s timed; oracle build {build_s:.1f} s untimed)"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def range_bounds(keys_sorted, q, g, seed):
    """q ranges whose span covers about g consecutive keys: lo uniform over the key space,
    hi = lo + g * (2^63 / n)."""
    s = wl.stream_seed(seed, 61)
    lo = wl.u64_stream(s, 0, q) >> np.uint64(1)
    span = np.uint64(max(1, int(g * (1 << 63) // len(keys_sorted))))
    return lo, lo + span


def run_range(args, ws, rank, local):
    """Range search (Section 3.2.5, the paper's granularity experiment): pi_range_search
    on batches of range queries over a 2^24-key index."""
    import torch
    from paper_1601_00159_gb300 import Index, build, load_library
    build.build()
    load_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = 1 << 24
    keys = np.sort(wl.distinct_keys(6, np.arange(n)))
    vals = wl.splitmix64(keys)
    idx = Index(torch.from_numpy(keys.view(np.int64)).to(dev), torch.from_numpy(vals.view(np.int64)).to(dev),
                0.25, 6)
    stream = torch.cuda.current_stream()
    grid = {}
    for q in (8192, 1 << 16):
        for g in (1, 10, 100, 1000):
            lo, hi = range_bounds(keys, q, g, 7 + g)
            dlo = torch.from_numpy(lo.view(np.int64)).to(dev)
            dhi = torch.from_numpy(hi.view(np.int64)).to(dev)
            cap = q * g * 2 + 4096
            offs = torch.empty(q + 1, dtype=torch.int64, device=dev)
            ko = torch.empty(cap, dtype=torch.int64, device=dev)
            vo = torch.empty(cap, dtype=torch.int64, device=dev)

            def call():
                rc = idx.lib.pi_range_search(idx._h, dlo.data_ptr(), dhi.data_ptr(), q, offs.data_ptr(),
                                             ko.data_ptr(), vo.data_ptr(), cap, ctypes_stream(stream))
                assert rc == 0
            for _ in range(args.warmup):
                call()
            torch.cuda.synchronize()
            steps = max(3, min(args.steps, 200))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                call()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            total = int(offs[q].item())
            assert total <= cap
            grid[f"q{q}_g{g}"] = {"ms_per_batch": ms, "Mranges_per_s": q / (ms * 1e-3) / 1e6,
                                  "Mresults_per_s": total / (ms * 1e-3) / 1e6, "results_per_range": total / q}
    head = grid["q65536_g100"]
    hbm, peak_kind = measured_peaks()
    res = head["results_per_range"] * (1 << 16)
    ab = res * (16 + 16 + 1) + (1 << 17) * (8 + 8 + 1)  # read pairs + meta, write pairs; bounds in
    achieved = ab / (head["ms_per_batch"] * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": head["Mranges_per_s"], "unit": "Mranges/s", "n_gpus": ws,
        "steps": max(3, min(args.steps, 200)), "warmup": args.warmup, "ms_per_step": head["ms_per_batch"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "range", "desc": WORKLOADS["range"]["desc"], "keys": n,
                   "l2_flush": "none: the 2^24-key index (285 MB storage) exceeds L2"},
        "grid": grid,
        "roofline": {"bound": "hbm", "kernel": "pi_range_search call", "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": achieved / hbm, "peak_source": peak_kind, "traffic": None,
                     "bytes_model": "per result: 8+8 B read, 1 B meta, 16 B written; per range: its two bounds"},
        "gpu_launches": None,
    }
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        orc = oracle.Oracle(keys, vals, 0.25, 6)
        lo, hi = range_bounds(keys, 1 << 16, 100, 107)
        t = time.perf_counter()
        done = 0
        while done < len(lo) and time.perf_counter() - t < args.cpu_budget:
            orc.range(lo[done:done + 4096], hi[done:done + 4096])
            done += 4096
        el = time.perf_counter() - t
        orc.close()
        line["cpu_baseline"] = {"value": done / el / 1e6, "unit": "Mranges/s", "cores": 1, "kind": "oracle",
                                "sample": f"{done} ranges of granularity 100 ({el:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    idx.close()


def ctypes_stream(stream):
    import ctypes
    return ctypes.c_void_p(stream.cuda_stream)


def cpu_baseline_multi(w, rnd, budget_s: float = 20.0):
    """The oracle on a bounded sample of the batching workload: indices in order, each
    built (untimed) and then given its batch (timed), until the budget is spent."""
    import oracle
    oracle.build()
    done, elapsed, used = 0, 0.0, 0
    for i, b in enumerate(rnd):
        if elapsed >= budget_s:
            break
        orc = oracle.Oracle(w.keys[i], w.vals[i], w.promote_p, w.hash_seeds[i])
        t = time.perf_counter()
        orc.execute(b.ops, b.keys, b.vals)
        elapsed += time.perf_counter() - t
        done += len(b)
        used += 1
        orc.close()
    return {"value": done / elapsed / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"the batches of the first {used} of {len(rnd)} indices ({done} queries, "
                      f"{elapsed:.1f} s timed; builds untimed)"}


def run_ours(args, ws, rank, local):
    import torch
    from paper_1601_00159_gb300 import Index, build, load_library
    build.build()
    load_library()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec = WORKLOADS[args.workload]
    t_gen = time.time()
    kw = {}
    if args.keys_log2:
        kw["n" if args.workload != "mid" else "n0"] = 1 << args.keys_log2
    if args.batch_log2:
        kw["q"] = 1 << args.batch_log2
    n_distinct_batches = 1 if args.workload == "tiny" else min(args.steps + args.warmup, args.batches)
    # the stage profile runs on further batches after the timed region: the mid workload's
    # inserts must be new keys there too, so it gets batches of its own
    prof_steps = min(args.steps, 16)
    n_prof_batches = prof_steps if args.workload == "mid" else 0
    if args.workload in ("mid", "skewed"):
        kw["n_batches"] = max(n_distinct_batches + n_prof_batches, 2)
    w = spec["fn"](**kw)
    gen = w.batches() if callable(w.batches) else iter(w.batches)
    host_batches = [next(gen) for _ in range(n_distinct_batches)]
    prof_host = [next(gen) for _ in range(n_prof_batches)]
    gen_s = time.time() - t_gen
    q = len(host_batches[0])

    def dev_batch(b):
        return (torch.from_numpy(b.ops).to(dev), torch.from_numpy(b.keys.view(np.int64)).to(dev),
                torch.from_numpy(b.vals.view(np.int64)).to(dev))

    dbatches = [dev_batch(b) for b in host_batches]
    results = torch.empty((q, 2), dtype=torch.int64, device=dev)
    keys_d = torch.from_numpy(w.keys.view(np.int64)).to(dev)
    vals_d = torch.from_numpy(w.vals.view(np.int64)).to(dev)
    total_steps = args.warmup + args.steps
    cfg = {"storage_capacity": len(w.keys) + q * (total_steps + n_prof_batches + 4) if args.workload == "mid" else 0,
           "rebuild_policy": 1 if args.rebuild == "deferred" else 0}
    cfg = {k: v for k, v in cfg.items() if v}
    tuned = tuned_plain(len(w.keys)) if args.workload == "skewed" else {}
    cfg.update(tuned)
    torch.cuda.synchronize()
    t = time.time()
    idx = Index(keys_d, vals_d, w.promote_p, w.hash_seed, cfg or None)
    create_s = time.time() - t
    del keys_d, vals_d
    stream = torch.cuda.current_stream()
    l2_bytes = torch.cuda.get_device_properties(dev).L2_cache_size

    for s in range(args.warmup):
        o, k, v = dbatches[s % len(dbatches)]
        idx.execute(o, k, v, results)
    torch.cuda.synchronize()
    info0 = idx.info()
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for s in range(args.steps):
            o, k, v = dbatches[(args.warmup + s) % len(dbatches)]
            idx.execute(o, k, v, results)
        idx.flush(stream)  # the last batch's background rebuild is inside the timed region
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    ms_total = ev0.elapsed_time(ev1)
    info1 = idx.info()
    routed = info1["routed_batches"] - info0["routed_batches"]
    # Stage times on further batches after the timed region (the events between stages
    # cost host time; a profiled batch also keeps the level-synchronous pipeline, so a run
    # whose batches took the small-batch route reports none).
    stage_ms, nb = {}, 0
    if routed < args.steps:
        prof_batches = [dev_batch(b) for b in prof_host] or dbatches
        idx.profile(True)
        for s in range(prof_steps):
            o, k, v = prof_batches[(s if prof_host else args.warmup + args.steps + s) % len(prof_batches)]
            idx.execute(o, k, v, results)
        idx.flush(stream)
        stage_ms, nb = idx.profile_read()  # stage times exclude the wait for the previous rebuild
        idx.profile(False)
    kernel_ms = None
    if args.kernel_times:
        # per-kernel times on extra batches after the timed region (events around every
        # launch serialise the launches, so these batches are not part of the value)
        idx.profile(2)
        for s in range(args.kernel_times):
            o, k, v = dbatches[(args.warmup + args.steps + s) % len(dbatches)]
            idx.execute(o, k, v, results)
        kt = idx.profile_kernels()
        idx.profile(False)
        kernel_ms = {name: {"launches_per_batch": c / args.kernel_times, "us_per_batch": 1e3 * ms / args.kernel_times}
                     for name, (c, ms) in kt.items()}
    assert idx.status() == 0, "device error status after the timed region"
    ms_total = reduce_max(ms_total, ws)
    ms_step = ms_total / args.steps
    value = ws * q * args.steps / (ms_total * 1e-3) / 1e6

    # e2e: host (pinned) buffers through pi_execute_batch_host, copies inside the timed region.
    # The mid workload's batches insert new keys, so replaying them on the same index would
    # skip their merges: its host-buffer run starts from a fresh index built from the same
    # keys and replays the same warm-up and batch sequence as the device-buffer run.
    e2e_steps = max(3, min(args.steps, 200))
    fresh = args.workload == "mid"
    if fresh:
        idx.close()
        keys_d = torch.from_numpy(w.keys.view(np.int64)).to(dev)
        vals_d = torch.from_numpy(w.vals.view(np.int64)).to(dev)
        idx = Index(keys_d, vals_d, w.promote_p, w.hash_seed, cfg or None)
        del keys_d, vals_d
        for s in range(args.warmup):
            o, k, v = dbatches[s % len(dbatches)]
            idx.execute(o, k, v, results)
        order = [(args.warmup + s) % len(host_batches) for s in range(e2e_steps)]
    else:
        order = [s % min(len(host_batches), 8) for s in range(e2e_steps)]
    hp = {}
    for i in sorted(set(order)):
        b = host_batches[i]
        hp[i] = (torch.from_numpy(b.ops.copy()).pin_memory(), torch.from_numpy(b.keys.view(np.int64).copy()).pin_memory(),
                 torch.from_numpy(b.vals.view(np.int64).copy()).pin_memory())
    hres = torch.empty((q, 2), dtype=torch.int64).pin_memory()
    if not fresh:
        for s in range(2):
            o, k, v = hp[order[s % len(order)]]
            idx.execute_host(o, k, v, hres)
    torch.cuda.synchronize()
    barrier(ws)
    t = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(e2e_steps):
        o, k, v = hp[order[s]]
        idx.execute_host(o, k, v, hres)
    idx.flush(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = reduce_max(e0.elapsed_time(e1), ws)
    e2e_value = ws * q * e2e_steps / (e2e_ms * 1e-3) / 1e6

    # The roofline of the whole batch (every kernel of one pi_execute_batch): the method's
    # bytes by the model of the paper's Section 5 (algorithmic_bytes), or the DRAM bytes
    # the kernels were measured to move by ncu if fewer, over the step time. Distinct,
    # written and inserted keys are counted exactly from the timed batches; every key of
    # the skewed workload is drawn from the key set, so each distinct key counts as a hit
    # (the delete-flagged few excepted, which the model then overstates by a value sector).
    hbm, peak_kind = measured_peaks()
    per_stage = {k: v / max(nb, 1) for k, v in stage_ms.items()}
    used = [host_batches[(args.warmup + s) % len(host_batches)] for s in range(min(args.steps, len(host_batches)))]
    distinct = float(np.mean([len(np.unique(b.keys)) for b in used]))
    writes = float(np.mean([len(np.unique(b.keys[b.ops != wl.OP_SEARCH])) for b in used]))
    ins = float(np.mean([int((b.ops == wl.OP_INSERT).sum()) for b in used]))
    sizes = info1["level_size"]
    lowest = info1["bottom_built"]
    ab = algorithmic_bytes(q, ins, distinct, distinct, writes, info1["live"], sizes, l2_bytes, w.promote_p)
    default_run = not (args.keys_log2 or args.batch_log2) and args.rebuild == "each"
    traffic, kprof, traffic_note = (kernel_profile(args.workload, len(w.keys), q) if default_run else
                                    (None, None, "no ncu capture of this configuration"))
    step_s = ms_step * 1e-3
    batch_low = min(ab["total"], traffic) if traffic is not None else ab["total"]
    # The storage locate (k_locate), the largest launch: it searches the lowest built index
    # level and then the storage layer. By the same model, per distinct key: a key and a
    # down sector on every level from 2 up to the lowest built one that is not
    # L2-resident (the paper's layout descends level 2 too; here the storage search
    # crosses that gap), a storage key sector and a value sector; plus the 25 B it streams
    # (query key and start position in; node position, state and prior value out).
    trav_levels = [l for l in range(2, lowest + 1) if sizes[l] and 12 * sizes[l] > l2_bytes / 2]
    loc_per_key = 64 * len(trav_levels) + 32 + 32 + 25
    loc_bytes = distinct * loc_per_key
    loc_ms = per_stage.get("locate")
    loc_traffic = None
    if kprof and "k_locate" in kprof:
        kl = kprof["k_locate"]
        loc_traffic = kl["dram_bytes"] * q / json.load(open(KERNEL_PROFILE))["capture"]["batch"]
    # The rebuild's writer: the incremental one reads and writes each built entry (8 B key
    # + 4 B down) once; the full one scans the storage layer's keys and meta and writes
    # every built entry.
    writer_ms = per_stage.get("rebuild_write")
    inc_region = info1["incremental_rebuilds"] - info0["incremental_rebuilds"]
    rebuilds_region = info1["rebuilds"] - info0["rebuilds"]
    entries = sum(sizes[lowest:])
    if rebuilds_region and inc_region == rebuilds_region:
        wkernel, wbytes = "k_relevel_write", 24 * entries
        wmodel = "12 B read + 12 B written per built index entry (incremental rebuild)"
    else:
        wkernel, wbytes = "k_rebuild_write", 9 * info1["size"] + 12 * entries
        wmodel = "9 B per storage node (key + meta scan) + 12 B per built index entry"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": (args.workload if not (args.keys_log2 or args.batch_log2) else
                                f"{args.workload}-keys{len(w.keys)}-batch{q}")
                               + ("-deferred-rebuild" if args.rebuild == "deferred" else ""),
                   "desc": spec["desc"] + ("; index rebuilt only when the updates since the last rebuild "
                                           "exceed 15% of the storage layer" if args.rebuild == "deferred" else ""),
                   "rebuild_policy": args.rebuild, "keys": len(w.keys), "batch": q,
                   "tuned": tuned or "defaults (the tuner's choice for this size, or no table)",
                   "distinct_batches_cycled": len(dbatches), "parallelism": f"replicas{ws}" if ws > 1 else "single",
                   "l2_flush": "none: storage layer and cycled batch inputs exceed L2"},
        "roofline": {"bound": "hbm", "kernel": "whole batch: every kernel of one pi_execute_batch",
                     "achieved": batch_low / step_s / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": batch_low / step_s / 1e9 / hbm, "peak_source": peak_kind,
                     "traffic": traffic, "traffic_note": traffic_note,
                     "algorithmic_bytes_per_launch": ab["total"], "bytes": "the smaller of the model and the traffic",
                     "frac_model": ab["total"] / step_s / 1e9 / hbm,
                     "frac_traffic": traffic / step_s / 1e9 / hbm if traffic is not None else None,
                     "frac_of_nominal_8tbs": batch_low / step_s / 1e9 / 8000.0,
                     "launches_per_step": (info1["kernel_launches"] - info0["kernel_launches"]) / args.steps,
                     "ms_per_launch": ms_step,
                     "model_parts": {k: v for k, v in ab.items() if k != "total"},
                     "bytes_model": "per batch: Q*25 + Q_ins*8 I/O; 64 B per distinct key and index level "
                                    "(from 2) too large for L2; 32 B key sector per distinct key, 32 B value "
                                    "sector per hit, 96 B per written key; full rebuild 9 N' + 12 N' p/(1-p)",
                     "distinct_keys_per_batch": distinct, "written_keys_per_batch": writes,
                     "k_locate": ({"ms_per_launch": loc_ms, "share_of_step": loc_ms / ms_step,
                                   "algorithmic_bytes_per_launch": loc_bytes,
                                   "achieved": loc_bytes / (loc_ms * 1e-3) / 1e9,
                                   "frac": loc_bytes / (loc_ms * 1e-3) / 1e9 / hbm,
                                   "traffic": loc_traffic,
                                   "bytes_model": f"{loc_per_key} B per distinct key: key and down sectors "
                                                  f"(64 B) on levels {trav_levels}, storage key and value "
                                                  "sectors (32 B each), 25 B streamed",
                                   "lowest_built_level": lowest} if loc_ms else
                                  {"note": "no k_locate launch: every timed batch took the small-batch "
                                           "route (one thread-block-cluster launch)"})},
        "rebuild_writer": {"kernel": wkernel, "ms_per_launch": writer_ms,
                           "algorithmic_bytes_per_launch": wbytes, "bytes_model": wmodel,
                           "achieved_gbs": wbytes / (writer_ms * 1e-3) / 1e9 if writer_ms else None,
                           "traffic": (kprof[wkernel]["dram_bytes"] * len(w.keys) /
                                       json.load(open(KERNEL_PROFILE))["capture"]["keys"])
                           if kprof and wkernel in kprof else None,
                           "incremental_rebuilds": inc_region, "rebuilds": rebuilds_region,
                           "note": "runs on the rebuild stream, overlapping the next batch's sort"},
        "stages_ms": per_stage,
        "kernel_us": kernel_ms,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": q * 17, "d2h_bytes_per_step": q * 16,
                "steps": e2e_steps, "index": "fresh, same batch sequence" if fresh else "the timed index"},
        "gpu_launches": info1["kernel_launches"] - info0["kernel_launches"],
        "routed_batches": routed,
        "clocks": clk.summary(),
        "index": {"size": info1["size"], "live": info1["live"], "tombstones": info1["tombstones"],
                  "top_level": info1["top_level"], "rebuilds_in_region": info1["rebuilds"] - info0["rebuilds"],
                  "create_s": create_s, "gen_s": gen_s, "distinct_keys_per_batch": distinct},
    }
    if args.rebuild == "deferred":
        # most batches skip the rebuild, so the writer's per-batch average is not one launch
        line["rebuild_writer"] = {"kernel": "k_rebuild_write", "ms_per_launch": None,
                                  "note": "deferred rebuild: the writer runs in "
                                          f"{rebuilds_region} of {args.steps} timed batches"}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, host_batches[0], args.cpu_budget)
    if rank == 0:
        print(json.dumps(line), flush=True)
    idx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="skewed", choices=sorted(WORKLOADS))
    ap.add_argument("--batches", type=int, default=32, help="distinct batches generated and cycled")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--keys-log2", type=int, default=0, help="override the index size (profiling runs)")
    ap.add_argument("--batch-log2", type=int, default=0, help="override the batch size (profiling runs)")
    ap.add_argument("--kernel-times", type=int, default=0,
                    help="after the timed region, time every kernel of this many more batches")
    ap.add_argument("--rebuild", default="each", choices=["each", "deferred"],
                    help="index rebuild after every batch, or deferred until the updates since the last "
                         "rebuild exceed 15%% of the storage layer (the paper's setting)")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        run_reference(args, ws, rank)
    elif args.workload == "batching":
        run_batching(args, ws, rank, local)
    elif args.workload == "serving":
        run_serving(args, ws, rank, local)
    elif args.workload == "range":
        run_range(args, ws, rank, local)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
