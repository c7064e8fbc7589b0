"""The allocation-free batch entry point (pi_execute_batch_noalloc) against the regular
one (pi_execute_batch).

Some callers cannot allocate device memory while a batch runs -- a serving loop that
must not stall on the CUDA allocator, or a process whose memory budget is fixed up
front -- so the library offers a variant whose per-batch scratch lives in a fixed
device array. This file checks, through the C ABI, that two indices built from the same
pairs and fed the same two batches in a row, one through each entry point, return
identical results and end in identical states (the path is integer-exact, so the
tolerance is zero); the same for two indices whose calls alternate on one stream without
synchronisation, with a batch of exactly the size limit. It also checks the limit. It is named to run after every other
test, and it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

from paper_1601_00159_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch
    from paper_1601_00159_gb300 import build, load_library
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return load_library()


def _dev(a, dtype):
    import torch
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def test_noalloc_matches_regular_entry_point_on_two_calls():
    import torch
    from paper_1601_00159_gb300 import Index
    w = wl.random_small(4242, 30000, 50000, 1 << 40, p=0.25, n_batches=2)
    # both indices get room for the new keys, so neither batch needs the storage to grow
    cfg = {"storage_capacity": 200000}
    regular = Index(_dev(w.keys, torch.int64), _dev(w.vals, torch.int64), w.promote_p, w.hash_seed, cfg)
    static = Index(_dev(w.keys, torch.int64), _dev(w.vals, torch.int64), w.promote_p, w.hash_seed, cfg)
    for b, batch in enumerate(w.batches):
        ops, keys, vals = _dev(batch.ops, torch.uint8), _dev(batch.keys, torch.int64), _dev(batch.vals, torch.int64)
        r1 = regular.execute(ops, keys, vals)
        r2 = torch.full_like(r1, -1)
        static.execute_noalloc(ops, keys, vals, r2)
        torch.cuda.synchronize()
        assert torch.equal(r1, r2), f"call {b}: results differ"
        assert regular.status() == 0 and static.status() == 0
        k1, v1 = regular.export()
        k2, v2 = static.export()
        assert torch.equal(k1, k2) and torch.equal(v1, v2), f"call {b}: final states differ"
        i1, i2 = regular.info(), static.info()
        assert i1["level_size"] == i2["level_size"] and i1["top_level"] == i2["top_level"]
    regular.close()
    static.close()


def test_noalloc_alternating_indices_on_one_stream():
    """Calls that alternate between two indices on one stream, with no synchronisation
    between them, share the one scratch array while each index's background rebuild still
    reads its part of it. Batch sizes include exactly PI_NOALLOC_MAX_BATCH. Results and
    final states must equal those of the regular entry point on twin indices."""
    import torch
    from paper_1601_00159_gb300 import Index, PI_NOALLOC_MAX_BATCH
    wa = wl.random_small(51, 40000, PI_NOALLOC_MAX_BATCH, 1 << 40, p=0.25, n_batches=3)
    wb = wl.random_small(52, 20000, 30000, 1 << 20, p=0.5, n_batches=3)
    cfg = {"storage_capacity": 400000}

    def twins(w):
        mk = lambda: Index(_dev(w.keys, torch.int64), _dev(w.vals, torch.int64), w.promote_p, w.hash_seed, cfg)
        return mk(), mk()

    (ra, sa), (rb, sb) = twins(wa), twins(wb)
    assert len(wa.batches[0]) == PI_NOALLOC_MAX_BATCH
    inputs = []
    for j in range(3):
        for w in (wa, wb):
            bt = w.batches[j]
            inputs.append((_dev(bt.ops, torch.uint8), _dev(bt.keys, torch.int64), _dev(bt.vals, torch.int64)))
    torch.cuda.synchronize()
    outs = []
    for c, (ops, keys, vals) in enumerate(inputs):  # A1 B1 A2 B2 A3 B3, one stream, no sync
        out = torch.full((ops.numel(), 2), -1, dtype=torch.int64, device="cuda")
        (sa if c % 2 == 0 else sb).execute_noalloc(ops, keys, vals, out)
        outs.append(out)
    expected = [(ra if c % 2 == 0 else rb).execute(*inp) for c, inp in enumerate(inputs)]
    torch.cuda.synchronize()
    for c, (got, exp) in enumerate(zip(outs, expected)):
        assert torch.equal(got, exp), f"call {c}: results differ"
    for reg, sta in ((ra, sa), (rb, sb)):
        assert reg.status() == 0 and sta.status() == 0
        k1, v1 = reg.export()
        k2, v2 = sta.export()
        assert torch.equal(k1, k2) and torch.equal(v1, v2), "final states differ"
        reg.close()
        sta.close()


def test_noalloc_rejects_batches_over_the_limit():
    import torch
    from paper_1601_00159_gb300 import Index, PiError, PI_ERR_INVALID_ARG, PI_NOALLOC_MAX_BATCH
    keys = _dev(wl.distinct_keys(1, np.arange(1000)), torch.int64)
    idx = Index(keys, keys.clone(), 0.5, 3)
    n = PI_NOALLOC_MAX_BATCH + 1
    ops = torch.zeros(n, dtype=torch.uint8, device="cuda")
    q = torch.zeros(n, dtype=torch.int64, device="cuda")
    out = torch.empty((n, 2), dtype=torch.int64, device="cuda")
    with pytest.raises(PiError) as e:
        idx.execute_noalloc(ops, q, q, out)
    assert e.value.code == PI_ERR_INVALID_ARG
    assert idx.status() == 0
    idx.close()
