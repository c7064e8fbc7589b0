"""Batching form (pi_multi_execute) against one oracle per index, bit for bit.

A set of independent indices of uneven sizes (p = 1/4) gets one batch each per call, of
uneven lengths: searches (half hits), inserts of new and of existing keys, deletes, a
few invalid queries and a hot key. Every result and every index's final state (live
pairs and built levels) must equal its oracle's. The class tables cover every kernel
variant (8, 16 and 32 warps per index; 4- and 8-bit radix digits), and the indices
stay usable by the single-index batch path before and after.
"""
import numpy as np
import pytest

from paper_1601_00159_gb300 import workloads as wl
from tests.parity import assert_results_equal, assert_state_equal, make_index, results_np, to_dev

pytestmark = pytest.mark.gpu

TABLES = {
    "default": None,
    "a": [(12, 8, 4), (15, 16, 8), (32, 32, 4)],
    "b": [(12, 8, 8), (15, 16, 4), (32, 32, 8)],
    # thread-block clusters: 2, 4, 8 and 16 CTAs per batch
    "c": [(12, 8, 4), (15, 32, 8, 2), (32, 32, 8, 8)],
    "d": [(14, 32, 8, 4), (32, 32, 8, 16)],
    "e": [(12, 16, 8, 8), (32, 16, 8, 2)],
}


@pytest.fixture(scope="module")
def orc_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    from paper_1601_00159_gb300 import build, load_library
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return load_library()


def log_uniform(seed, tag, count, lo_log, hi_log):
    u = wl.uniform01(wl.stream_seed(seed, tag), 0, count)
    return np.floor(2.0 ** (lo_log + u * (hi_log - lo_log))).astype(np.int64)


def make_batch(seed, keys, q):
    s = wl.stream_seed(seed, 77)
    kind = wl.bounded(s, 0, q, 20)
    hit = keys[wl.bounded(s, q, q, max(len(keys), 1))] if len(keys) else wl.u64_stream(s, q, q) >> np.uint64(1)
    miss = wl.u64_stream(s, 2 * q, q) >> np.uint64(1)
    bkeys = np.where(kind % 2 == 0, hit, miss)
    bkeys = np.where(kind == 19, hit[0], bkeys)  # a hot key
    ops = np.where(kind < 12, 0, np.where(kind < 16, 1, 2)).astype(np.uint8)
    ops = np.where(kind == 13, np.uint8(5), ops)  # invalid op code
    bkeys = np.where(kind == 15, wl.RESERVED_KEY, bkeys)  # the reserved key
    return wl.Batch(ops.astype(np.uint8), bkeys.astype(np.uint64), wl.u64_stream(s, 3 * q, q))


def build_set(orc_mod, seed, count, lo_log, hi_log, big=None, configs=None):
    sizes = log_uniform(seed, 1, count, lo_log, hi_log)
    if big:
        sizes[0] = big
    idxs, orcs, keysets = [], [], []
    for i, n in enumerate(sizes):
        keys = wl.distinct_keys(seed * 1000 + i, np.arange(int(n)))
        vals = wl.splitmix64(keys)
        hs = int(wl.stream_seed(seed, 500 + i))
        idxs.append(make_index(keys, vals, 0.25, hs, (configs or {}).get(i)))
        orcs.append(orc_mod.Oracle(keys, vals, 0.25, hs))
        keysets.append(keys)
    return idxs, orcs, keysets


def run_rounds(ms, idxs, orcs, keysets, seed, rounds, qlo_log, qhi_log, skip=()):
    import torch
    for r in range(rounds):
        qs = log_uniform(seed, 100 + r, len(idxs), qlo_log, qhi_log)
        batches, host = [], []
        for i, q in enumerate(qs):
            if i in skip:
                continue
            b = make_batch(seed * 7919 + r * 131 + i, keysets[i], int(q))
            res = torch.full((len(b.ops), 2), -1, dtype=torch.int64, device="cuda")
            batches.append((i, to_dev(b.ops, torch.uint8), to_dev(b.keys, torch.int64),
                            to_dev(b.vals, torch.int64), res))
            host.append((i, b, res))
        ms.execute(batches)
        torch.cuda.synchronize()
        for i, b, res in host:
            exp = orcs[i].execute(b.ops, b.keys, b.vals)
            assert_results_equal(results_np(res), exp, f"round {r} index {i}")


@pytest.mark.parametrize("table", sorted(TABLES))
def test_multi_matches_oracle_per_index(orc_mod, table):
    from paper_1601_00159_gb300 import MultiSet
    seed = 3 + len(table)
    idxs, orcs, keysets = build_set(orc_mod, seed, 20, 6, 16, big=(1 << 18) + 5)
    ms = MultiSet(idxs, TABLES[table])
    run_rounds(ms, idxs, orcs, keysets, seed, 3, 0, 12)
    for i, (ix, orc) in enumerate(zip(idxs, orcs)):
        assert_state_equal(ix, orc, f"index {i}")
    ms.close()
    for ix, orc in zip(idxs, orcs):
        ix.close()
        orc.close()


def test_multi_mixed_with_plain_path_and_subsets(orc_mod):
    """Rounds that leave some indices out, empty batches, the single-index path on the
    same indices in between, and an index whose storage must grow."""
    import torch
    from paper_1601_00159_gb300 import MultiSet
    from tests.parity import run_batch
    seed = 17
    idxs, orcs, keysets = build_set(orc_mod, seed, 9, 4, 13)
    ms = MultiSet(idxs)
    run_rounds(ms, idxs, orcs, keysets, seed, 2, 0, 11, skip=(2, 5))
    for i in (0, 2, 7):  # the plain path after the batching form
        b = make_batch(900 + i, keysets[i], 3000)
        assert_results_equal(run_batch(idxs[i], b), orcs[i].execute(b.ops, b.keys, b.vals), f"plain {i}")
    # an empty batch for index 1 and many new keys for index 3 (its storage grows)
    empty = (1, torch.zeros(0, dtype=torch.uint8, device="cuda"), torch.zeros(0, dtype=torch.int64, device="cuda"),
             torch.zeros(0, dtype=torch.int64, device="cuda"), torch.zeros((0, 2), dtype=torch.int64, device="cuda"))
    q = 20000
    s = wl.stream_seed(seed, 3)
    ins = wl.Batch(np.ones(q, np.uint8), wl.u64_stream(s, 0, q) >> np.uint64(1), wl.u64_stream(s, q, q))
    res = torch.full((q, 2), -1, dtype=torch.int64, device="cuda")
    ms.execute([empty, (3, to_dev(ins.ops, torch.uint8), to_dev(ins.keys, torch.int64),
                        to_dev(ins.vals, torch.int64), res)])
    torch.cuda.synchronize()
    assert_results_equal(results_np(res), orcs[3].execute(ins.ops, ins.keys, ins.vals), "growth")
    run_rounds(ms, idxs, orcs, keysets, seed + 1, 2, 0, 11)
    for i, (ix, orc) in enumerate(zip(idxs, orcs)):
        assert_state_equal(ix, orc, f"index {i}")
    ms.close()


def test_multi_after_the_plain_path_grew_an_index(orc_mod):
    """A plain batch of new keys grows an index's storage (its arrays are reallocated);
    the set's next calls must use the new arrays."""
    from paper_1601_00159_gb300 import MultiSet
    from tests.parity import run_batch
    seed = 29
    # index 2 builds every level (lowest level 2), so the burst of new keys below also
    # outgrows its index layer's capacity
    idxs, orcs, keysets = build_set(orc_mod, seed, 6, 4, 12, configs={2: {"lowest_level": 2}})
    ms = MultiSet(idxs)
    run_rounds(ms, idxs, orcs, keysets, seed, 1, 0, 10)
    cap0 = idxs[2].info()["storage_capacity"]
    q = 90000  # more new keys than the storage layer's headroom
    s = wl.stream_seed(seed, 5)
    ins = wl.Batch(np.ones(q, np.uint8), wl.u64_stream(s, 0, q) >> np.uint64(1), wl.u64_stream(s, q, q))
    icap0 = idxs[2].info()["index_capacity"]
    assert_results_equal(run_batch(idxs[2], ins), orcs[2].execute(ins.ops, ins.keys, ins.vals), "plain growth")
    # the next plain batch grows the index layer the larger storage layer needs
    b = make_batch(31, keysets[2], 500)
    assert_results_equal(run_batch(idxs[2], b), orcs[2].execute(b.ops, b.keys, b.vals), "plain after growth")
    info = idxs[2].info()
    assert info["storage_capacity"] > cap0 and info["index_capacity"] > icap0
    run_rounds(ms, idxs, orcs, keysets, seed + 1, 3, 0, 12)
    for i, (ix, orc) in enumerate(zip(idxs, orcs)):
        assert_state_equal(ix, orc, f"index {i}")
    ms.close()


def test_multi_rejects_bad_sets_and_batches():
    import torch
    from paper_1601_00159_gb300 import MultiSet, PiError, PI_ERR_INVALID_ARG
    keys = wl.distinct_keys(5, np.arange(100))
    a = make_index(keys, keys, 0.25, 1)
    with pytest.raises(PiError) as e:
        MultiSet([a, a])
    assert e.value.code == PI_ERR_INVALID_ARG
    with pytest.raises(PiError):
        MultiSet([a], classes=[(12, 12, 8)])
    with pytest.raises(PiError):
        MultiSet([a], classes=[(32, 8, 8, 4)])  # a cluster takes 16- or 32-warp CTAs
    with pytest.raises(PiError):
        MultiSet([a], classes=[(32, 32, 8, 3)])  # cluster sizes 2, 4, 8, 16
    ms = MultiSet([a])
    z = torch.zeros(4, dtype=torch.int64, device="cuda")
    ops = torch.zeros(4, dtype=torch.uint8, device="cuda")
    r = torch.zeros((4, 2), dtype=torch.int64, device="cuda")
    with pytest.raises(PiError):
        ms.execute([(1, ops, z, z, r)])  # no such index
    with pytest.raises(PiError):
        ms.execute([(0, ops, z, z, r), (0, ops, z, z, r)])  # twice in one call
    ms.close()
    a.close()


@pytest.mark.parametrize("kind", ["few_segments", "overflow"])
def test_multi_prefix_fixup(orc_mod, kind):
    """Keys whose four leading varying bytes collide: a few segments of different keys
    (ordered by the in-CTA fix-up), or so many that the CTA packs the batch again and
    sorts it with every pass. Exact per index either way."""
    import torch
    from paper_1601_00159_gb300 import MultiSet
    idxs, orcs, batches, host = [], [], [], []
    for i in range(6):
        s = wl.stream_seed(70 + i, 1)
        n, q = 3000 + 500 * i, 20000 + 3000 * i
        if kind == "few_segments":  # bytes 0..4 vary, byte 4 holds 4 bits: 28-bit prefixes
            mk = lambda st, o, c: wl.u64_stream(st, o, c) & np.uint64((1 << 36) - 1)
        else:  # bytes 0 and 4..7 vary, bytes 4..7 take 16 values: every prefix is shared
            mk = lambda st, o, c: ((wl.u64_stream(st, o, c) & np.uint64(0xFF))
                                   | ((wl.bounded(st, o + c, c, 16).astype(np.uint64) * np.uint64(0x01010101)) << np.uint64(32)))
        keys = np.unique(mk(s, 0, n))
        vals = wl.splitmix64(keys)
        hs = 900 + i
        idxs.append(make_index(keys, vals, 0.25, hs))
        orcs.append(orc_mod.Oracle(keys, vals, 0.25, hs))
        sb = wl.stream_seed(80 + i, 2)
        ops = wl.bounded(sb, 0, q, 3).astype(np.uint8)
        bk = np.where(wl.bounded(sb, q, q, 2) == 0, keys[wl.bounded(sb, 2 * q, q, len(keys))], mk(sb, 3 * q, q))
        b = wl.Batch(ops, bk.astype(np.uint64), wl.u64_stream(sb, 5 * q, q))
        res = torch.full((q, 2), -1, dtype=torch.int64, device="cuda")
        batches.append((i, to_dev(b.ops, torch.uint8), to_dev(b.keys, torch.int64), to_dev(b.vals, torch.int64), res))
        host.append((i, b, res))
    for table in (None, [(32, 16, 4)], [(32, 32, 8, 4)]):
        ms = MultiSet(idxs, table)
        ms.execute(batches)
        torch.cuda.synchronize()
        for i, b, res in host:
            assert_results_equal(results_np(res), orcs[i].execute(b.ops, b.keys, b.vals), f"{kind} {table} {i}")
        ms.close()
    for i, (ix, orc) in enumerate(zip(idxs, orcs)):
        assert_state_equal(ix, orc, f"{kind} index {i}")


def test_multi_full_batching_workload(orc_mod):
    """The batching workload at full size: 256 indices of 2^10..2^20 keys, batches of
    2^8..2^16 queries (20% inserts of new keys), two rounds through the tuned class table
    (thread-block clusters for the largest class), against 256 oracles; then every
    index's live pairs and levels."""
    import json
    import os
    import torch
    from paper_1601_00159_gb300 import MultiSet
    w = wl.batching()
    root = os.path.join(os.path.dirname(__file__), "..", "paper_1601_00159_gb300", "multi_tuning.json")
    with open(root) as f:
        tuning = json.load(f)
    classes = [tuple(c) for c in tuning["classes"]]
    lowest = {int(h): int(l) for h, l in tuning.get("lowest_level", {}).items()}
    idxs, orcs = [], []
    for i, keys in enumerate(w.keys):
        lg = int(np.ceil(np.log2(max(len(keys), 1))))
        low = next((lowest[h] for h in sorted(lowest) if lg <= h), 0)
        cfg = {"storage_capacity": len(keys) + 4 * int(w.batch_sizes[i]) + 4096}
        if low:
            cfg["lowest_level"] = low
        idxs.append(make_index(keys, w.vals[i], w.promote_p, w.hash_seeds[i], cfg))
        orcs.append(orc_mod.Oracle(keys, w.vals[i], w.promote_p, w.hash_seeds[i]))
    ms = MultiSet(idxs, classes)
    for r in range(2):
        rnd = w.batches(r)
        batches = []
        for i, b in enumerate(rnd):
            res = torch.full((len(b), 2), -1, dtype=torch.int64, device="cuda")
            batches.append((i, to_dev(b.ops, torch.uint8), to_dev(b.keys, torch.int64), to_dev(b.vals, torch.int64),
                            res))
        ms.execute(batches)
        torch.cuda.synchronize()
        for i, b in enumerate(rnd):
            assert_results_equal(results_np(batches[i][4]), orcs[i].execute(b.ops, b.keys, b.vals),
                                 f"round {r} index {i} ({len(w.keys[i])} keys, {len(b)} queries)")
    for i, (ix, orc) in enumerate(zip(idxs, orcs)):
        assert_state_equal(ix, orc, f"index {i}")
    ms.close()
    for ix, orc in zip(idxs, orcs):
        ix.close()
        orc.close()
