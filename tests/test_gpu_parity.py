"""GPU path vs oracle, bit for bit: per-query results (arrival order), final live
(key, value) set, and every built index level with its down pointers.

Integer work throughout, so the bar is exact equality. Sizes span several tiles of
every kernel (sort 4096, apply 2048, rebuild 4096 queries or nodes) with ragged tails.
"""
import numpy as np
import pytest

from paper_1601_00159_gb300 import workloads as wl
from tests.parity import (assert_results_equal, assert_state_equal, make_index, run_batch, to_dev,
                          results_np)

pytestmark = pytest.mark.gpu


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


def run_workload(orc_mod, w, config=None, check_levels_every=1, batches=None, check_levels=True, route=False):
    idx = make_index(w.keys, w.vals, w.promote_p, w.hash_seed, config, route=route)
    orc = orc_mod.Oracle(w.keys, w.vals, w.promote_p, w.hash_seed)
    assert_state_equal(idx, orc, f"{w.name} after create")
    bl = w.batches() if callable(w.batches) else w.batches
    for b, batch in enumerate(bl):
        if batches is not None and b >= batches:
            break
        got = run_batch(idx, batch)
        exp = orc.execute(batch.ops, batch.keys, batch.vals)
        assert_results_equal(got, exp, f"{w.name} batch {b}")
        if (b + 1) % check_levels_every == 0:
            assert_state_equal(idx, orc, f"{w.name} batch {b}", check_levels)
    info = assert_state_equal(idx, orc, f"{w.name} end", check_levels)
    idx.close()
    orc.close()
    return info


@pytest.mark.parametrize("route", [False, True])
def test_tiny_config_full_size(orc_mod, route):
    """2^16 keys, p = 1/2, one all-search batch of 2^14 (half hits, half misses); on the
    level-synchronous pipeline and on the small-batch route."""
    w = wl.tiny()
    info = run_workload(orc_mod, w, route=route)
    assert info["rebuilds"] == 1  # only the initial build: a search batch changes nothing


@pytest.mark.parametrize("route", [False, True])
@pytest.mark.parametrize("seed", range(40))
def test_random_small_dense(orc_mod, seed, route):
    """Tiny key ranges: long same-key runs, revivals, delete/insert chains, invalid ops;
    on the level-synchronous pipeline and on the small-batch route (one cluster launch)."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 3000))
    q = int(rng.integers(1, 9000))
    kr = int(rng.choice([5, 64, 700, 5000, 1 << 40]))
    p = float(rng.choice([0.5, 0.25, 0.125, 0.0625]))
    w = wl.random_small(1000 + seed, n, q, kr, p=p, n_batches=4)
    run_workload(orc_mod, w, route=route)


def test_mid_shape_scaled(orc_mod):
    w = wl.mid(seed=11, n0=1 << 18, q=1 << 15, n_batches=6)
    run_workload(orc_mod, w)


def test_skewed_shape_scaled(orc_mod):
    w = wl.skewed(seed=12, n=1 << 20, q=1 << 17, n_batches=6)
    info = run_workload(orc_mod, w)
    assert info["tombstones"] > 0  # deletes keep flagged nodes in place


@pytest.mark.parametrize("policy", [0, 1])
def test_rebuild_policy_does_not_change_results(orc_mod, policy):
    w = wl.random_small(77, 20000, 30000, 1 << 20, p=0.25, n_batches=5)
    # levels are defined right after a rebuild; the deferred policy may leave them stale
    run_workload(orc_mod, w, config={"rebuild_policy": policy, "rebuild_threshold_pct": 50},
                 check_levels_every=1, check_levels=(policy == 0))


@pytest.mark.parametrize("cfg", [{"test_flags": 1}, {"smem_top_entries": 1}, {"smem_top_entries": 40},
                                 {"test_flags": 1, "smem_top_entries": 200}])
def test_descent_paths_give_identical_results(orc_mod, cfg):
    """The in-kernel level walk, no pinned levels, and few pinned levels all reach
    the same interceptions as the default launch plan."""
    w = wl.random_small(88, 60000, 40000, 1 << 40, p=0.25, n_batches=3)
    run_workload(orc_mod, w, config=cfg)
    w2 = wl.skewed(seed=5, n=1 << 18, q=1 << 15, n_batches=3)
    run_workload(orc_mod, w2, config=cfg)


def test_index_capacity_overflow_keeps_results_exact(orc_mod):
    """An index layer that does not fit drops its lowest levels (the descent then walks
    longer storage gaps); results stay exact and the capacity grows afterwards."""
    w = wl.random_small(5, 50000, 20000, 1 << 30, p=0.5, n_batches=4)
    idx = make_index(w.keys, w.vals, w.promote_p, w.hash_seed, {"index_capacity": 3000, "lowest_level": 2})
    orc = orc_mod.Oracle(w.keys, w.vals, w.promote_p, w.hash_seed)
    info0 = idx.info()
    assert info0["bottom_built"] > 2
    for b, batch in enumerate(w.batches):
        assert_results_equal(run_batch(idx, batch), orc.execute(batch.ops, batch.keys, batch.vals), f"b{b}")
    info = assert_state_equal(idx, orc, "overflow end")
    assert info["bottom_built"] == 2 and info["index_capacity"] > 3000


@pytest.mark.parametrize("route", [False, True])
@pytest.mark.parametrize("lowest", [0, 2, 3, 5])
@pytest.mark.parametrize("p", [0.5, 0.25])
def test_lowest_built_level(orc_mod, lowest, p, route):
    """Index layers whose lowest materialised level is 2 (every level, as in the paper),
    3, 5 or the automatic choice: results, live pairs and the built levels stay exact,
    and the descent scans the longer storage gaps below the lowest level."""
    w = wl.random_small(60 + lowest, 30000, 20000, 1 << 40, p=p, n_batches=3)
    cfg = {"lowest_level": lowest} if lowest else None
    info = run_workload(orc_mod, w, cfg, route=route)
    auto = 4 if p == 0.25 else 6  # the lowest level whose expected storage gap is >= 32 nodes
    assert info["bottom_built"] == (lowest or auto)


@pytest.mark.parametrize("route", [False, True])
def test_edge_cases(orc_mod, route):
    import torch
    M = (1 << 64) - 1
    # empty index, then inserts; empty batch; all-invalid batch; extreme keys
    idx = make_index(np.zeros(0, np.uint64), np.zeros(0, np.uint64), 0.25, 3, route=route)
    orc = orc_mod.Oracle(np.zeros(0, np.uint64), np.zeros(0, np.uint64), 0.25, 3)
    assert_state_equal(idx, orc, "empty")
    empty = torch.empty(0, dtype=torch.int64, device="cuda")
    idx.execute(torch.empty(0, dtype=torch.uint8, device="cuda"), empty, empty)
    cases = [
        (np.array([0, 1, 0, 2, 0], np.uint8), np.array([0, 0, 0, 0, 0], np.uint64), np.arange(5, dtype=np.uint64)),
        (np.array([1, 1, 0, 0], np.uint8), np.array([M - 1, 1 << 63, M - 1, M], np.uint64),
         np.array([7, 8, 9, 10], np.uint64)),
        (np.array([3, 200, 1], np.uint8), np.array([5, 5, M], np.uint64), np.array([1, 2, 3], np.uint64)),
        (np.full(10000, 1, np.uint8), np.full(10000, 42, np.uint64), np.arange(10000, dtype=np.uint64)),
        (np.array([2] * 5000 + [0] * 5000, np.uint8), np.full(10000, 42, np.uint64), np.zeros(10000, np.uint64)),
    ]
    for c, (ops, keys, vals) in enumerate(cases):
        b = wl.Batch(ops, keys, vals)
        assert_results_equal(run_batch(idx, b), orc.execute(ops, keys, vals), f"case {c}")
        assert_state_equal(idx, orc, f"case {c}")


def test_one_hot_key_spans_many_tiles(orc_mod):
    """One key receives 2^18 interleaved queries (sort, scan and apply tiles all split
    the run): the owner is the run's last query and every result sees the prior ones."""
    n = 1 << 12
    keys = wl.distinct_keys(3, np.arange(n))
    vals = wl.splitmix64(keys)
    idx = make_index(keys, vals, 0.25, 9)
    orc = orc_mod.Oracle(keys, vals, 0.25, 9)
    q = (1 << 18) + 123
    s = wl.stream_seed(3, 9)
    ops = wl.bounded(s, 0, q, 3).astype(np.uint8)
    bkeys = np.where(wl.bounded(s, q, q, 4) == 0, keys[wl.bounded(s, 2 * q, q, n)], keys[17])
    bvals = wl.u64_stream(s, 3 * q, q)
    b = wl.Batch(ops, bkeys.astype(np.uint64), bvals)
    assert_results_equal(run_batch(idx, b), orc.execute(b.ops, b.keys, b.vals), "hot")
    assert_state_equal(idx, orc, "hot")


def test_host_entry_point_matches_device_entry_point(orc_mod):
    import torch
    w = wl.random_small(31, 4000, 5000, 3000, p=0.25, n_batches=2)
    a = make_index(w.keys, w.vals, w.promote_p, w.hash_seed)
    b = make_index(w.keys, w.vals, w.promote_p, w.hash_seed)
    for batch in w.batches:
        ra = results_np(a.execute(to_dev(batch.ops, torch.uint8), to_dev(batch.keys, torch.int64),
                                  to_dev(batch.vals, torch.int64)))
        ops = torch.from_numpy(batch.ops.copy()).pin_memory()
        ks = torch.from_numpy(batch.keys.view(np.int64).copy()).pin_memory()
        vs = torch.from_numpy(batch.vals.view(np.int64).copy()).pin_memory()
        out = torch.empty((len(batch), 2), dtype=torch.int64).pin_memory()
        b.execute_host(ops, ks, vs, out)
        torch.cuda.current_stream().synchronize()
        rb = results_np(out)
        assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])


@pytest.mark.parametrize("route", [False, True])
def test_host_entry_point_pipelined_and_mixed_with_other_streams(orc_mod, route):
    """Host-buffer batches run on the library's own streams, two in flight: several are
    issued back to back with no synchronisation, then a device-buffer batch on another
    stream, a range search and more host-buffer batches. Each must see the effect of every
    batch issued before it on the index (arrival order across calls), and each result
    buffer must be complete once the caller's stream completes."""
    import torch
    w = wl.random_small(77, 20000, 30000, 40000, p=0.25, n_batches=8)  # dense keys: long dependency chains
    orc = orc_mod.Oracle(w.keys, w.vals, w.promote_p, w.hash_seed)
    idx = make_index(w.keys, w.vals, w.promote_p, w.hash_seed, route=route)
    side = torch.cuda.Stream()
    expected, outs = [], []
    for b, batch in enumerate(w.batches):
        expected.append(orc.execute(batch.ops, batch.keys, batch.vals))
        if b == 4:  # a device-buffer batch on another stream, between host-buffer ones
            with torch.cuda.stream(side):
                res = idx.execute(to_dev(batch.ops, torch.uint8), to_dev(batch.keys, torch.int64),
                                  to_dev(batch.vals, torch.int64), stream=side)
            outs.append((res, side))
            continue
        ops = torch.from_numpy(batch.ops.copy()).pin_memory()
        ks = torch.from_numpy(batch.keys.view(np.int64).copy()).pin_memory()
        vs = torch.from_numpy(batch.vals.view(np.int64).copy()).pin_memory()
        out = torch.empty((len(batch), 2), dtype=torch.int64).pin_memory()
        idx.execute_host(ops, ks, vs, out)
        outs.append((out, (ops, ks, vs)))  # the inputs stay referenced until their copies ran
    torch.cuda.current_stream().synchronize()
    side.synchronize()
    for b, ((out, st), exp) in enumerate(zip(outs, expected)):
        assert_results_equal(results_np(out), exp, f"pipelined batch {b}")
    assert_state_equal(idx, orc, "after pipelined host batches")
    idx.close()
    orc.close()


def test_create_rejects_bad_arguments():
    import torch
    from paper_1601_00159_gb300 import Index, PiError, PI_ERR_INVALID_ARG
    k = to_dev(np.array([1, (1 << 64) - 1], np.uint64), torch.int64)
    v = to_dev(np.array([1, 2], np.uint64), torch.int64)
    with pytest.raises(PiError) as e:
        Index(k, v, 0.25, 1)
    assert e.value.code == PI_ERR_INVALID_ARG
    k2 = to_dev(np.array([1, 2], np.uint64), torch.int64)
    with pytest.raises(PiError):
        Index(k2, v, 0.3, 1)


@pytest.mark.parametrize("lowest,p", [(2, 0.5), (3, 0.25), (0, 0.25)])
def test_incremental_level_rebuild(orc_mod, lowest, p):
    """Batches that only delete, revive and overwrite existing keys leave the storage
    layout alone until delete-flagged nodes pass 1/8 of it, so most rebuilds update the
    previous levels with the batch's membership changes. Every batch's results, live
    pairs and built levels (with down pointers) must equal the oracle's."""
    n = 40000
    keys = wl.distinct_keys(77, np.arange(n))
    vals = wl.splitmix64(keys)
    cfg = {"lowest_level": lowest} if lowest else None
    idx = make_index(keys, vals, p, 12, cfg)
    orc = orc_mod.Oracle(keys, vals, p, 12)
    for b in range(8):
        s = wl.stream_seed(77, 100 + b)
        q = 9000
        u = wl.bounded(s, 0, q, 100)
        ops = np.where(u < 5, 2, np.where(u < 45, 1, 0)).astype(np.uint8)  # 5% delete, 40% (re)insert
        bk = keys[wl.bounded(s, q, q, n)]
        batch = wl.Batch(ops, bk.astype(np.uint64), wl.u64_stream(s, 2 * q, q))
        assert_results_equal(run_batch(idx, batch), orc.execute(batch.ops, batch.keys, batch.vals), f"b{b}")
        assert_state_equal(idx, orc, f"b{b}")
    info = idx.info()
    assert info["incremental_rebuilds"] >= 4, info["incremental_rebuilds"]
    idx.close()
    orc.close()


def _distinct_writes(batches):
    """Distinct keys written (valid inserts and deletes) per batch, summed."""
    total = 0
    for b in batches:
        valid = (b.ops == wl.OP_INSERT) | (b.ops == wl.OP_DELETE)
        valid &= b.keys != np.uint64(0xFFFFFFFFFFFFFFFF)
        total += len(np.unique(b.keys[valid]))
    return total


@pytest.mark.parametrize("kr", [16, 700, 1 << 40])
def test_single_owner_per_storage_node(orc_mod, kr):
    """Section 3.2.4: every storage node is modified by exactly one owner per batch. The
    debug check counts the writes to every node; a second write would leave a sticky
    error that the state comparison (pi_status) reports."""
    from paper_1601_00159_gb300 import PI_TEST_OWNER_CHECK
    w = wl.random_small(60 + kr % 89, 3000, 30000, kr, p=0.25, n_batches=4)
    info = run_workload(orc_mod, w, config={"test_flags": PI_TEST_OWNER_CHECK})
    assert 0 < info["owner_checked_writes"] <= _distinct_writes(w.batches)
    w2 = wl.skewed(seed=9, n=1 << 18, q=1 << 16, n_batches=3)  # Zipf hot keys: long same-key runs
    info2 = run_workload(orc_mod, w2, config={"test_flags": PI_TEST_OWNER_CHECK})
    w2b = w2.batches() if callable(w2.batches) else w2.batches
    assert 0 < info2["owner_checked_writes"] <= _distinct_writes(list(w2b)[:3])


def _capped_workload(b: int, seed: int):
    """Keys whose hash reaches the height cap (built by inverting splitmix64), among
    random keys, then batches that insert more of them (new keys: a re-layout and a full
    rebuild), delete some (delete-flagged nodes at the top levels: an incremental
    rebuild), and revive them."""
    from tests.hashkeys import hash_with_trailing_zeros, key_with_hash
    mix = int(wl.splitmix64(np.uint64(seed)))
    hmax = min(32, 64 // b)
    tz_near = [64, 63, b * (hmax - 1), b * (hmax - 1) - 1, b * (hmax - 2)]
    capped = []
    for j, tz in enumerate(tz_near * 4):
        k = key_with_hash(hash_with_trailing_zeros(tz, 1000 * j + b), mix)
        if k != (1 << 64) - 1 and k not in capped:
            capped.append(k)
    base = [int(k) for k in wl.distinct_keys(b + 50, np.arange(3000))]
    init = np.array(sorted(set(base + capped[: len(capped) // 2])), np.uint64)
    later = np.array(capped[len(capped) // 2:], np.uint64)
    early = np.array(capped[: len(capped) // 2], np.uint64)
    z = np.zeros
    b1 = wl.Batch(np.ones(len(later), np.uint8), later, np.arange(len(later), dtype=np.uint64) + 7)
    b2 = wl.Batch(np.full(len(early), 2, np.uint8), early, z(len(early), np.uint64))
    rev = early[:3]
    b3 = wl.Batch(np.concatenate([np.ones(len(rev), np.uint8), z(len(capped), np.uint8)]),
                  np.concatenate([rev, np.array(capped, np.uint64)]),
                  np.concatenate([np.arange(len(rev), dtype=np.uint64) + 11, z(len(capped), np.uint64)]))
    return wl.Workload(f"capped-b{b}", init, wl.splitmix64(init), 2.0 ** -b, seed, [b1, b2, b3]), hmax


@pytest.mark.parametrize("b", [1, 2, 3, 4])
@pytest.mark.parametrize("lowest", [0, 2])
def test_height_cap_keys(orc_mod, b, lowest):
    """Keys at the height cap (hash 0, whose trailing-zero count is 64, and hashes with
    b * (Hmax - 1) or more trailing zeros) give an index of exactly Hmax levels; every
    level, its down pointers and the results match the oracle through create, insert,
    delete and revive batches."""
    w, hmax = _capped_workload(b, 900 + b)
    info = run_workload(orc_mod, w, config={"lowest_level": lowest} if lowest else None)
    assert info["top_level"] == hmax
    assert info["level_size"][hmax] >= 1


def test_small_route_alternates_with_plain_path(orc_mod):
    """One index takes routed batches (at most 2^16 queries, one cluster launch) and
    level-synchronous ones (larger batches) in turn, with a range search and a no-alloc
    batch between them, inserts that make it outgrow 2^20 keys (after which every batch
    takes the level-synchronous pipeline) and deletes past 1/8 of the storage layer.
    Every result, the live pairs and the built levels match the oracle throughout."""
    import torch
    n0 = (1 << 20) - 100000
    keys = wl.distinct_keys(41, np.arange(n0))
    vals = wl.splitmix64(keys)
    idx = make_index(keys, vals, 0.25, 41, route=True)
    orc = orc_mod.Oracle(keys, vals, 0.25, 41)
    s = wl.stream_seed(41, 7)
    off = 0
    for b, q in enumerate([1 << 14, 1 << 17, 60000, 5000, (1 << 16) + 1, 3000, 200000, 1 << 16, 1 << 15]):
        kind = wl.bounded(s, off, q, 10)
        old = keys[wl.bounded(s, off + q, q, len(keys))]
        new = wl.u64_stream(s, off + 2 * q, q) >> np.uint64(1)
        ops = np.where(kind < 3, 0, np.where(kind < 8, 1, 2)).astype(np.uint8)
        bk = np.where(kind % 2 == 0, old, new).astype(np.uint64)
        batch = wl.Batch(ops, bk, wl.u64_stream(s, off + 3 * q, q))
        off += 4 * q
        if b == 3:  # the no-alloc entry point between routed batches
            res = torch.full((q, 2), -1, dtype=torch.int64, device="cuda")
            idx.execute_noalloc(to_dev(batch.ops, torch.uint8), to_dev(batch.keys, torch.int64),
                                to_dev(batch.vals, torch.int64), res)
            got = results_np(res)
        else:
            got = run_batch(idx, batch)
        assert_results_equal(got, orc.execute(batch.ops, batch.keys, batch.vals), f"batch {b} ({q} queries)")
        assert_state_equal(idx, orc, f"batch {b}")
        if b == 4:  # a range search sees every batch before it
            lo = np.sort(keys[:64])
            hi = lo + np.uint64(1 << 40)
            offs, rk, rv = idx.range_search(to_dev(lo, torch.int64), to_dev(hi, torch.int64))
            ok, ov = orc.export()
            for j in range(len(lo)):
                sel = (ok >= lo[j]) & (ok <= hi[j])
                a, e = int(offs[j]), int(offs[j + 1])
                assert np.array_equal(rk[a:e].cpu().numpy().view(np.uint64), ok[sel]), f"range {j}"
    assert idx.info()["size"] > (1 << 20)
    idx.close()
    orc.close()
