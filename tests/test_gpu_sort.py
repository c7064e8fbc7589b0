"""The batch sort's prefix passes and fix-up, against the oracle.

By default a batch is sorted with radix passes on its four most significant varying key
bytes. Queries whose keys agree on those bytes then form segments in arrival order, and
a fix-up kernel orders each segment that holds different keys. test_flags can force 1-3
prefix passes, which makes such segments long and common, or all eight passes. Every
variant must give the same results and the same final index as the oracle. Invalid
queries (bad op code, or the reserved key 2^64-1) sort after every valid one.
"""
import numpy as np
import pytest

from paper_1601_00159_gb300 import workloads as wl
from tests.parity import assert_results_equal, assert_state_equal, make_index, run_batch

pytestmark = pytest.mark.gpu

FLAGS = [("full", 2), ("prefix1", 1 << 4), ("prefix2", 2 << 4), ("prefix3", 3 << 4), ("default", 0)]


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


def _run(orc_mod, w, flags, n_batches):
    idx = make_index(w.keys, w.vals, w.promote_p, w.hash_seed, {"test_flags": flags} if flags else None)
    orc = orc_mod.Oracle(w.keys, w.vals, w.promote_p, w.hash_seed)
    gen = w.batches() if callable(w.batches) else iter(w.batches)
    launches = []
    for b in range(n_batches):
        batch = next(gen)
        l0 = idx.info()["kernel_launches"]
        assert_results_equal(run_batch(idx, batch), orc.execute(batch.ops, batch.keys, batch.vals),
                             f"{w.name} flags {flags} batch {b}")
        launches.append(idx.info()["kernel_launches"] - l0)
    assert_state_equal(idx, orc, f"{w.name} flags {flags} end")
    idx.close()
    orc.close()
    return launches


@pytest.mark.parametrize("name,flags", FLAGS)
def test_wide_keys_with_invalid_queries(orc_mod, name, flags):
    """Keys spread over five bytes, 2% invalid queries: one to four prefix passes leave
    one to five bytes to the fix-up (segments of tens of thousands of queries under one
    pass, a few queries under three)."""
    w = wl.random_small(51, 20000, 30000, 1 << 40, p=0.25, n_batches=2)
    _run(orc_mod, w, flags, 2)


@pytest.mark.parametrize("name,flags", FLAGS)
def test_zipf_hot_keys(orc_mod, name, flags):
    """Zipf(0.99) over 2^14 uniform 63-bit keys, batches of 2^16 + 77: the hottest keys
    hold thousands of queries, so prefix collisions with them make long segments."""
    w = wl.skewed(seed=7, n=1 << 14, q=(1 << 16) + 77, n_batches=2)
    _run(orc_mod, w, flags, 2)


def test_low_spread_prefix_switches_to_full_sort(orc_mod):
    """Keys whose four leading varying bytes take only 16 values: four prefix passes
    leave 16 segments of thousands of different keys, ordered by the long-segment path.
    Once the host sees that, later batches take all eight passes (more launches).
    Every batch stays exact."""
    n, q = 8192, 40000
    s = wl.stream_seed(11, 1)

    def mk(start, count):
        bits = wl.bounded(s, start, count, 16).astype(np.uint64)
        low = wl.bounded(s, start + count, count, 1 << 24).astype(np.uint64)
        out = low
        for j, shift in enumerate((24, 32, 40, 48)):
            out = out | (((bits >> np.uint64(j)) & np.uint64(1)) << np.uint64(shift))
        return out

    keys = np.unique(mk(0, n))
    vals = wl.splitmix64(keys)
    batches = []
    for b in range(6):
        sb = wl.stream_seed(11, 10 + b)
        ops = wl.bounded(sb, 0, q, 3).astype(np.uint8)
        pick = wl.bounded(sb, q, q, 2) == 0
        bkeys = np.where(pick, keys[wl.bounded(sb, 2 * q, q, len(keys))], mk(10 ** 6 * (b + 1), q))
        batches.append(wl.Batch(ops, bkeys.astype(np.uint64), wl.u64_stream(sb, 3 * q, q)))
    w = wl.Workload("lowspread", keys, vals, 0.25, 5, batches, True)
    launches = _run(orc_mod, w, 0, 6)
    assert launches[-1] > launches[0], launches


@pytest.mark.parametrize("flags", [0, 1 << 4, 3 << 4])
def test_small_and_degenerate_batches(orc_mod, flags):
    """Batches of 1, 31, 33 and 2049 queries; one of all-invalid queries; one whose
    keys are all equal."""
    import oracle  # noqa: F401
    keys = wl.distinct_keys(4, np.arange(3000))
    vals = wl.splitmix64(keys)
    idx = make_index(keys, vals, 0.5, 2, {"test_flags": flags} if flags else None)
    orc = orc_mod.Oracle(keys, vals, 0.5, 2)
    s = wl.stream_seed(4, 3)
    cases = []
    for c, q in enumerate((1, 31, 33, 2049)):
        ops = wl.bounded(s, 10 * c, q, 3).astype(np.uint8)
        bk = np.where(wl.bounded(s, 10 * c + q, q, 2) == 0, keys[wl.bounded(s, 10 * c + 2 * q, q, 3000)],
                      wl.u64_stream(s, 10 * c + 3 * q, q) >> np.uint64(1))
        cases.append(wl.Batch(ops, bk.astype(np.uint64), wl.u64_stream(s, 10 * c + 4 * q, q)))
    q = 500
    cases.append(wl.Batch(np.full(q, 7, np.uint8), keys[:q].copy(), np.arange(q, dtype=np.uint64)))
    cases.append(wl.Batch(wl.bounded(s, 99999, q, 3).astype(np.uint8), np.full(q, keys[5], np.uint64),
                          np.arange(q, dtype=np.uint64)))
    for c, b in enumerate(cases):
        assert_results_equal(run_batch(idx, b), orc.execute(b.ops, b.keys, b.vals), f"case {c}")
        assert_state_equal(idx, orc, f"case {c}")
    idx.close()
    orc.close()
