"""Range search (pi_range_search) against the oracle, bit for bit.

Both bounds of every query go through the batch sort and descent; each query's pairs are
then read from its storage slice. The index carries delete-flagged nodes and merged new
nodes from earlier batches. Checked: every offset, every key and value, in key order;
empty ranges (lo > hi), single keys, the whole key space, the bound 2^64-1, thousands of
queries over several CTAs, all lowest-level layouts and sort variants, and the
capacity rule (a query's pairs are written only when they all fit).
"""
import numpy as np
import pytest

from paper_1601_00159_gb300 import workloads as wl
from tests.parity import assert_results_equal, make_index, run_batch, to_dev

pytestmark = pytest.mark.gpu
M64 = (1 << 64) - 1


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


def ranges(seed, keys, q, max_span):
    s = wl.stream_seed(seed, 31)
    anchor = keys[wl.bounded(s, 0, q, len(keys))]
    jitter = wl.bounded(s, q, q, 1 << 20).astype(np.uint64)
    lo = np.where(wl.bounded(s, 2 * q, q, 2) == 0, anchor, anchor - np.minimum(anchor, jitter))
    span = (wl.u64_stream(s, 3 * q, q) % np.uint64(max_span)).astype(np.uint64)
    hi = lo + span
    lo[:6] = [0, 9, keys[3], 0, keys[-1], M64]
    hi[:6] = [M64, 8, keys[3], 0, M64, M64]  # all, lo > hi, one key, [0, 0], tail, [max, max]
    return lo.astype(np.uint64), hi.astype(np.uint64)


def check(idx, orc, lo, hi, ctx, cap=None):
    import torch
    offs, k, v = idx.range_search(to_dev(lo, torch.int64), to_dev(hi, torch.int64), cap=cap)
    eo, ek, ev = orc.range(lo, hi)
    go = offs.cpu().numpy().view(np.uint64)
    assert np.array_equal(go, eo), f"{ctx}: offsets differ at {np.nonzero(go != eo)[0][:5]}"
    assert np.array_equal(k.cpu().numpy().view(np.uint64), ek), f"{ctx}: keys differ"
    assert np.array_equal(v.cpu().numpy().view(np.uint64), ev), f"{ctx}: values differ"
    return int(eo[-1])


@pytest.mark.parametrize("cfg", [None, {"lowest_level": 2}, {"lowest_level": 4}, {"test_flags": 1 << 4},
                                 {"test_flags": 2}])
def test_range_search_matches_oracle(orc_mod, cfg):
    n = 50000
    keys = np.sort(wl.distinct_keys(41, np.arange(n)))
    vals = wl.splitmix64(keys)
    idx = make_index(keys, vals, 0.25, 8, cfg)
    orc = orc_mod.Oracle(keys, vals, 0.25, 8)
    # deletes (delete-flagged nodes stay in storage) and new keys (merged)
    w = wl.random_small(42, 10, 30000, 1 << 63, p=0.25, n_batches=1)
    b = w.batches[0]
    bkeys = np.where(wl.bounded(wl.stream_seed(42, 1), 0, len(b), 2) == 0,
                     keys[wl.bounded(wl.stream_seed(42, 2), 0, len(b), n)], b.keys)
    batch = wl.Batch(b.ops, bkeys.astype(np.uint64), b.vals)
    assert_results_equal(run_batch(idx, batch), orc.execute(batch.ops, batch.keys, batch.vals), "setup")
    # a few deletes of existing keys: they stay as delete-flagged nodes (no re-layout)
    s = wl.stream_seed(42, 3)
    dk = keys[wl.bounded(s, 0, 2000, n)]
    dels = wl.Batch(np.full(2000, 2, np.uint8), dk.astype(np.uint64), np.zeros(2000, np.uint64))
    assert_results_equal(run_batch(idx, dels), orc.execute(dels.ops, dels.keys, dels.vals), "deletes")
    assert idx.info()["tombstones"] > 0
    for span, q in ((1 << 50, 3001), (1 << 58, 500), (1, 257)):
        lo, hi = ranges(int(span % 97) + q, keys, q, span)
        total = check(idx, orc, lo, hi, f"span {span}")
        assert total > 0
    idx.close()
    orc.close()


def test_range_search_capacity_and_empty(orc_mod):
    import torch
    keys = np.sort(wl.distinct_keys(43, np.arange(4000)))
    idx = make_index(keys, keys, 0.5, 2)
    orc = orc_mod.Oracle(keys, keys, 0.5, 2)
    lo, hi = ranges(5, keys, 300, 1 << 60)
    eo, ek, ev = orc.range(lo, hi)
    total = int(eo[-1])
    cap = total // 2
    offs = torch.empty(len(lo) + 1, dtype=torch.int64, device="cuda")
    kk = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    vv = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    dlo, dhi = to_dev(lo, torch.int64), to_dev(hi, torch.int64)  # kept alive across the call
    rc = idx.lib.pi_range_search(idx._h, dlo.data_ptr(), dhi.data_ptr(), len(lo), offs.data_ptr(), kk.data_ptr(),
                                 vv.data_ptr(), cap, None)
    torch.cuda.synchronize()
    assert rc == 0
    go = offs.cpu().numpy().view(np.uint64)
    assert np.array_equal(go, eo)
    gk = kk.cpu().numpy().view(np.uint64)
    for i in range(len(lo)):
        a, b = int(eo[i]), int(eo[i + 1])
        if b <= cap:  # fits: written
            assert np.array_equal(gk[a:b], ek[a:b]), i
    # n = 0 writes offsets[0] = 0
    z = torch.zeros(0, dtype=torch.int64, device="cuda")
    o1 = torch.full((1,), 7, dtype=torch.int64, device="cuda")
    assert idx.lib.pi_range_search(idx._h, z.data_ptr(), z.data_ptr(), 0, o1.data_ptr(), None, None, 0, None) == 0
    torch.cuda.synchronize()
    assert int(o1.item()) == 0
    idx.close()
    orc.close()
