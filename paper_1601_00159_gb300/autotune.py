"""Autotuner of the batching form's kernel variants (run on the GPU that will serve).

The batching form (pi_multi_execute) runs each size class of indices with its own
persistent kernel. This script times every variant -- 8, 16 or 32 warps per index, 4- or
8-bit radix digits -- on the indices of each class of the batching workload and writes
the fastest per class to multi_tuning.json beside it, which bench.py and MultiSet
callers pass to pi_multi_create.

    python -m paper_1601_00159_gb300.autotune [--calls 8]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "multi_tuning.json")
BOUNDS = [14, 17, 32]  # class upper bounds (log2 of the storage size)
VARIANTS = [(w, b) for w in (8, 16, 32) for b in (4, 8)]


def main():
    import torch
    from . import Index, MultiSet, build, load_library
    from . import workloads as wl
    ap = argparse.ArgumentParser()
    ap.add_argument("--calls", type=int, default=8)
    ap.add_argument("--out", default=OUT)
    ap.add_argument("--only", default="", help="time one variant, e.g. 32x8 (profiling runs)")
    args = ap.parse_args()
    variants = VARIANTS
    if args.only:
        wv, bv = (int(x) for x in args.only.split("x"))
        variants = [(wv, bv)]
    build.build()
    load_library()
    dev = torch.device("cuda")
    w = wl.batching()
    # every call takes a round no call has applied before, so its inserts are new keys
    # (every index merges and rebuilds), as in the batching workload itself
    nr = 2 + args.calls
    rounds = [w.batches(r) for r in range(nr)]
    rnd = rounds[0]
    sizes = np.array([len(k) for k in w.keys])
    lg = np.ceil(np.log2(np.maximum(sizes, 1))).astype(int)
    chosen, table = [], {}
    lo = -1
    for c, hi in enumerate(BOUNDS):
        members = [i for i in range(len(sizes)) if lo < lg[i] <= hi]
        lo = hi
        if not members:
            chosen.append((hi, 16, 8))
            continue
        batches = [[(torch.from_numpy(rd[i].ops).to(dev), torch.from_numpy(rd[i].keys.view(np.int64)).to(dev),
                     torch.from_numpy(rd[i].vals.view(np.int64)).to(dev),
                     torch.empty((len(rd[i]), 2), dtype=torch.int64, device=dev)) for i in members] for rd in rounds]
        timings = {}
        for (wp, bits) in variants:
            idxs = []
            for i in members:
                k = torch.from_numpy(w.keys[i].view(np.int64)).to(dev)
                v = torch.from_numpy(w.vals[i].view(np.int64)).to(dev)
                cap = len(w.keys[i]) + len(rnd[i]) * (nr + 4)
                idxs.append(Index(k, v, w.promote_p, w.hash_seeds[i], {"storage_capacity": cap}))
            ms = MultiSet(idxs, [(32, wp, bits)])
            descs = [[(j, *bj[j]) for j in range(len(members))] for bj in batches]
            for r in range(2):
                ms.execute(descs[r])
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for r in range(args.calls):
                ms.execute(descs[2 + r])
            e1.record()
            torch.cuda.synchronize()
            timings[f"{wp}x{bits}"] = e0.elapsed_time(e1) / args.calls
            ms.close()
            for ix in idxs:
                ix.close()
        best = min(timings, key=timings.get)
        wp, bits = (int(x) for x in best.split("x"))
        chosen.append((hi, wp, bits))
        table[f"class{c} (log2 size <= {hi}, {len(members)} indices)"] = timings
        print(f"class {c}: {len(members)} indices, ms per call {timings} -> {best}", flush=True)
    # The classes run concurrently in one call and share the SMs, so the per-class winners
    # are checked jointly: every table whose classes take one of the two fastest variants
    # of their class is timed on the whole workload, and the fastest table is kept.
    joint = {}
    if not args.only:
        import itertools
        tops = []
        for c, hi in enumerate(BOUNDS):
            key = next((k for k in table if k.startswith(f"class{c} ")), None)
            ranked = sorted(table[key], key=table[key].get)[:2] if key else [f"{chosen[c][1]}x{chosen[c][2]}"]
            tops.append([tuple(int(x) for x in r.split("x")) for r in ranked])
        all_batches = [[(i, torch.from_numpy(b.ops).to(dev), torch.from_numpy(b.keys.view(np.int64)).to(dev),
                         torch.from_numpy(b.vals.view(np.int64)).to(dev),
                         torch.empty((len(b), 2), dtype=torch.int64, device=dev)) for i, b in enumerate(rd)]
                       for rd in rounds]
        for combo in itertools.product(*tops):
            cls = [(BOUNDS[c], combo[c][0], combo[c][1]) for c in range(len(BOUNDS))]
            idxs = []
            for i in range(len(sizes)):
                k = torch.from_numpy(w.keys[i].view(np.int64)).to(dev)
                v = torch.from_numpy(w.vals[i].view(np.int64)).to(dev)
                cap = len(w.keys[i]) + len(rnd[i]) * (nr + 4)
                idxs.append(Index(k, v, w.promote_p, w.hash_seeds[i], {"storage_capacity": cap}))
            ms = MultiSet(idxs, cls)
            for r in range(2):
                ms.execute(all_batches[r])
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for r in range(args.calls):
                ms.execute(all_batches[2 + r])
            e1.record()
            torch.cuda.synchronize()
            joint[json.dumps(cls)] = e0.elapsed_time(e1) / args.calls
            ms.close()
            for ix in idxs:
                ix.close()
            print(f"joint {cls}: {joint[json.dumps(cls)]:.3f} ms per call", flush=True)
        best = min(joint, key=joint.get)
        chosen = [tuple(c) for c in json.loads(best)]
    out = {"classes": chosen, "ms_per_call": table, "joint_ms_per_call": joint,
           "device": torch.cuda.get_device_name(),
           "workload": "batching (seed 4): indices of each class; every call a fresh round of batches "
                       "(inserts are new keys)",
           "calls_timed": args.calls, "date": time.strftime("%Y-%m-%d")}
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out["classes"]))


if __name__ == "__main__":
    main()
