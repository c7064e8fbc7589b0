"""Autotuner of the batch path's variants (run on the GPU that will serve).

Batching form (default mode): pi_multi_execute runs each size class of indices with its
own persistent kernel. This mode times every variant -- 8, 16 or 32 warps per index, 4-
or 8-bit radix digits, and for 16 or 32 warps with 8-bit digits thread-block clusters of
2, 4, 8 or 16 CTAs per batch -- on the indices of each class of the batching workload, then the
node fan-out of each class (the lowest built index level, i.e. the storage nodes one
entry of the lowest level spans), and writes the fastest per class to multi_tuning.json
beside it, which bench.py and MultiSet callers pass to pi_multi_create / pi_create_ex.

Plain path (--plain): for each index size of the skewed workload (batches of 2^22 Zipf
queries), the fan-out (lowest built level) together with the entries pinned in shared
memory, then the radix passes per batch with the fastest of those; every variant's
results and final key/value set must equal the default configuration's, bit for bit.
Writes plain_tuning.json beside this file, which bench.py reads.

    python -m paper_1601_00159_gb300.autotune [--calls 8]
    python -m paper_1601_00159_gb300.autotune --plain [--sizes 24 26 27] [--calls 6]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "multi_tuning.json")
PLAIN_OUT = os.path.join(HERE, "plain_tuning.json")
BOUNDS = [14, 17, 32]  # class upper bounds (log2 of the storage size)
VARIANTS = [(w, b, 1) for w in (8, 16, 32) for b in (4, 8)] + [(w, 8, c) for w in (16, 32) for c in (2, 4, 8, 16)]


def kernel_name(v):
    """'32x8' for one CTA per batch, '32x8c4' for clusters of 4 CTAs."""
    w, b, c = v
    return f"{w}x{b}" + (f"c{c}" if c > 1 else "")


def parse_kernel(name):
    wb, _, c = name.partition("c")
    w, b = (int(x) for x in wb.split("x"))
    return (w, b, int(c) if c else 1)


def variant_name(cfg):
    return ",".join(f"{k}={v}" for k, v in sorted(cfg.items())) or "default"


def tune_plain(args):
    """The plain path's tunables on the skewed workload, one index size at a time."""
    import torch
    from . import Index, build, load_library
    from . import workloads as wl
    build.build()
    load_library()
    dev = torch.device("cuda")
    classes = []
    for logn in args.sizes:
        w = wl.skewed(n=1 << logn, n_batches=args.calls + 2)
        gen = w.batches()
        dbs = []
        for _ in range(args.calls + 2):
            b = next(gen)
            dbs.append((torch.from_numpy(b.ops).to(dev), torch.from_numpy(b.keys.view(np.int64)).to(dev),
                        torch.from_numpy(b.vals.view(np.int64)).to(dev)))
        keys_d = torch.from_numpy(w.keys.view(np.int64)).to(dev)
        vals_d = torch.from_numpy(w.vals.view(np.int64)).to(dev)
        ref = {}

        def run(cfg):
            idx = Index(keys_d, vals_d, w.promote_p, w.hash_seed, cfg or None)
            outs = [torch.empty((len(d[0]), 2), dtype=torch.int64, device=dev) for d in dbs]
            for i in range(2):
                idx.execute(*dbs[i], outs[i])
            idx.flush()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for i in range(2, len(dbs)):
                idx.execute(*dbs[i], outs[i])
            idx.flush()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.calls
            state = idx.export()
            info = idx.info()
            assert idx.status() == 0
            idx.close()
            if not ref:  # the default configuration is the reference
                ref.update(outs=outs, state=state)
            else:
                for i, (a, b) in enumerate(zip(outs, ref["outs"])):
                    assert torch.equal(a, b), f"{variant_name(cfg)}: batch {i} results differ from the default's"
                assert torch.equal(state[0], ref["state"][0]) and torch.equal(state[1], ref["state"][1]), \
                    f"{variant_name(cfg)}: final key/value set differs from the default's"
            return ms, info

        timings, shapes = {}, {}
        ms, info = run({})
        timings["default"] = ms
        shapes["default"] = {"lowest_built": info["bottom_built"], "pinned_from_level": info["smem_low_level"]}
        fan = [{"lowest_level": lo, "smem_top_entries": sm} for lo in (2, 3, 4) for sm in (2048, 12288)]
        for cfg in fan:
            ms, info = run(cfg)
            timings[variant_name(cfg)] = ms
            shapes[variant_name(cfg)] = {"lowest_built": info["bottom_built"], "pinned_from_level": info["smem_low_level"]}
            print(f"2^{logn}: {variant_name(cfg)}: {ms:.4f} ms per batch", flush=True)
        best_fan = min(fan, key=lambda c: timings[variant_name(c)])
        for sp in (3, 4, 8):
            cfg = dict(best_fan, sort_passes=sp)
            ms, _ = run(cfg)
            timings[variant_name(cfg)] = ms
            print(f"2^{logn}: {variant_name(cfg)}: {ms:.4f} ms per batch", flush=True)
        cands = [c for c in [dict(best_fan, sort_passes=sp) for sp in (3, 4, 8)] + [dict(c) for c in fan]]
        best = min(cands, key=lambda c: timings[variant_name(c)])
        if timings["default"] <= timings[variant_name(best)]:
            best = {}
        classes.append({"log2_keys": logn, "chosen": best, "ms_per_batch": timings, "shape": shapes,
                        "fanout_storage_nodes": {variant_name(c): 4 ** (shapes[variant_name(c)]["lowest_built"] - 1)
                                                 for c in fan}})
        print(f"2^{logn}: chosen {variant_name(best)} ({timings[variant_name(best)]:.4f} ms vs default "
              f"{timings['default']:.4f})", flush=True)
        del dbs, keys_d, vals_d, ref
        torch.cuda.empty_cache()
    out = {"classes": classes, "device": torch.cuda.get_device_name(),
           "workload": "skewed: batches of 2^22 Zipf(0.99) queries, 90/5/5 search/insert/delete, P = 1/4",
           "calls_timed": args.calls, "date": time.strftime("%Y-%m-%d"),
           "checked": "every variant's results and final key/value set equal the default configuration's"}
    with open(args.plain_out, "w") as f:
        json.dump(out, f, indent=1)


def main():
    import torch
    from . import Index, MultiSet, build, load_library
    from . import workloads as wl
    ap = argparse.ArgumentParser()
    ap.add_argument("--calls", type=int, default=8)
    ap.add_argument("--warm", type=int, default=16,
                    help="untimed calls first: every call inserts new keys, so the indices grow "
                         "towards the sizes a long run reaches")
    ap.add_argument("--out", default=OUT)
    ap.add_argument("--only", default="", help="time one variant, e.g. 32x8 or 32x8c8 (profiling runs)")
    ap.add_argument("--plain", action="store_true", help="tune the plain path instead of the batching form")
    ap.add_argument("--sizes", type=int, nargs="*", default=[24, 26, 27], help="--plain: log2 index sizes")
    ap.add_argument("--plain-out", default=PLAIN_OUT)
    args = ap.parse_args()
    if args.plain:
        return tune_plain(args)
    variants = VARIANTS
    if args.only:
        variants = [parse_kernel(args.only)]
    build.build()
    load_library()
    dev = torch.device("cuda")
    w = wl.batching()
    # every call takes a round no call has applied before, so its inserts are new keys
    # (every index merges and rebuilds), as in the batching workload itself
    nw = args.warm
    nr = nw + args.calls
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
            chosen.append((hi, 16, 8, 1))
            continue
        batches = [[(torch.from_numpy(rd[i].ops).to(dev), torch.from_numpy(rd[i].keys.view(np.int64)).to(dev),
                     torch.from_numpy(rd[i].vals.view(np.int64)).to(dev),
                     torch.empty((len(rd[i]), 2), dtype=torch.int64, device=dev)) for i in members] for rd in rounds]
        timings = {}
        for var in variants:
            idxs = []
            for i in members:
                k = torch.from_numpy(w.keys[i].view(np.int64)).to(dev)
                v = torch.from_numpy(w.vals[i].view(np.int64)).to(dev)
                cap = len(w.keys[i]) + len(rnd[i]) * (nr + 4)
                idxs.append(Index(k, v, w.promote_p, w.hash_seeds[i], {"storage_capacity": cap}))
            ms = MultiSet(idxs, [(32, *var)])
            descs = [ms.prepare([(j, *bj[j]) for j in range(len(members))]) for bj in batches]
            for r in range(nw):
                ms.execute(descs[r])
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for r in range(args.calls):
                ms.execute(descs[nw + r])
            e1.record()
            torch.cuda.synchronize()
            timings[kernel_name(var)] = e0.elapsed_time(e1) / args.calls
            ms.close()
            for ix in idxs:
                ix.close()
        best = min(timings, key=timings.get)
        chosen.append((hi, *parse_kernel(best)))
        table[f"class{c} (log2 size <= {hi}, {len(members)} indices)"] = timings
        print(f"class {c}: {len(members)} indices, ms per call {timings} -> {best}", flush=True)
    # The classes run concurrently in one call and share the SMs, so the per-class winners
    # are checked jointly on the whole workload: every table whose classes take one of the
    # three fastest variants of their class, and the tables with fewer classes (two classes
    # split at 2^14 or 2^17 nodes, or one) whose classes take one of the fastest variants
    # of the classes they merge. The fastest table is kept.
    joint = {}
    if not args.only:
        import itertools
        tops = []
        for c, hi in enumerate(BOUNDS):
            key = next((k for k in table if k.startswith(f"class{c} ")), None)
            ranked = sorted(table[key], key=table[key].get)[:3] if key else [kernel_name(chosen[c][1:])]
            tops.append([parse_kernel(r) for r in ranked])
        all_batches = [[(i, torch.from_numpy(b.ops).to(dev), torch.from_numpy(b.keys.view(np.int64)).to(dev),
                         torch.from_numpy(b.vals.view(np.int64)).to(dev),
                         torch.empty((len(b), 2), dtype=torch.int64, device=dev)) for i, b in enumerate(rd)]
                       for rd in rounds]

        def merged(cs):  # the fastest variants of the classes cs, without repeats
            out = []
            for c in cs:
                for v in tops[c]:
                    if v not in out:
                        out.append(v)
            return out

        tables = [[(BOUNDS[c], *combo[c]) for c in range(len(BOUNDS))] for combo in itertools.product(*tops)]
        for split in range(len(BOUNDS) - 1):  # two classes: [0, split] and (split, last]
            for lo_v in merged(range(split + 1)):
                for hi_v in merged(range(split + 1, len(BOUNDS))):
                    tables.append([(BOUNDS[split], *lo_v), (BOUNDS[-1], *hi_v)])
        for v in merged(range(len(BOUNDS))):
            tables.append([(BOUNDS[-1], *v)])
        for cls in tables:
            idxs = []
            for i in range(len(sizes)):
                k = torch.from_numpy(w.keys[i].view(np.int64)).to(dev)
                v = torch.from_numpy(w.vals[i].view(np.int64)).to(dev)
                cap = len(w.keys[i]) + len(rnd[i]) * (nr + 4)
                idxs.append(Index(k, v, w.promote_p, w.hash_seeds[i], {"storage_capacity": cap}))
            ms = MultiSet(idxs, cls)
            prepared = [ms.prepare(b) for b in all_batches]
            for r in range(nw):
                ms.execute(prepared[r])
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for r in range(args.calls):
                ms.execute(prepared[nw + r])
            e1.record()
            torch.cuda.synchronize()
            joint[json.dumps(cls)] = e0.elapsed_time(e1) / args.calls
            ms.close()
            for ix in idxs:
                ix.close()
            print(f"joint {cls}: {joint[json.dumps(cls)]:.3f} ms per call", flush=True)
        best = min(joint, key=joint.get)
        chosen = [tuple(c) for c in json.loads(best)]
    # Node fan-out per class: the lowest built index level (at P = 1/4 an entry of level l
    # spans 4^(l-1) storage nodes), timed with the class's chosen kernel variant on the
    # class's indices; 0 is the library's automatic choice.
    fanout, lowest = {}, {}
    lo = -1
    for c, hi in enumerate(cb[0] for cb in chosen):
        members = [i for i in range(len(sizes)) if lo < lg[i] <= hi or (c == len(chosen) - 1 and lg[i] > hi)]
        lo = hi
        if not members or args.only:
            continue
        batches = [[(j, torch.from_numpy(rd[i].ops).to(dev), torch.from_numpy(rd[i].keys.view(np.int64)).to(dev),
                     torch.from_numpy(rd[i].vals.view(np.int64)).to(dev),
                     torch.empty((len(rd[i]), 2), dtype=torch.int64, device=dev)) for j, i in enumerate(members)]
                   for rd in rounds]
        times = {}
        for low in (0, 2, 3, 4):
            idxs = []
            for i in members:
                k = torch.from_numpy(w.keys[i].view(np.int64)).to(dev)
                v = torch.from_numpy(w.vals[i].view(np.int64)).to(dev)
                cap = len(w.keys[i]) + len(rnd[i]) * (nr + 4)
                cfg = {"storage_capacity": cap}
                if low:
                    cfg["lowest_level"] = low
                idxs.append(Index(k, v, w.promote_p, w.hash_seeds[i], cfg))
            ms = MultiSet(idxs, [(32, *chosen[c][1:])])
            prepared = [ms.prepare(b) for b in batches]
            for r in range(nw):
                ms.execute(prepared[r])
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for r in range(args.calls):
                ms.execute(prepared[nw + r])
            e1.record()
            torch.cuda.synchronize()
            times[f"lowest_level={low or 'auto'}"] = e0.elapsed_time(e1) / args.calls
            ms.close()
            for ix in idxs:
                ix.close()
        key = min(times, key=times.get)
        lowest[str(hi)] = 0 if key.endswith("auto") else int(key.split("=")[1])
        fanout[f"class{c} (log2 size <= {hi}, {len(members)} indices)"] = times
        print(f"class {c} fan-out: {times} -> {key}", flush=True)
    out = {"classes": chosen, "lowest_level": lowest, "fanout_ms_per_call": fanout,
           "ms_per_call": table, "joint_ms_per_call": joint,
           "device": torch.cuda.get_device_name(),
           "workload": "batching (seed 4): indices of each class; every call a fresh round of batches "
                       "(inserts are new keys)",
           "calls_timed": args.calls, "date": time.strftime("%Y-%m-%d")}
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out["classes"]))


if __name__ == "__main__":
    main()
