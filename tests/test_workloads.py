"""The workload generators keep the properties the measurements rely on (CPU only, at
reduced sizes): inserts that the configurations call new are new in every call,
skewed and serving queries stay on the key set, and the request sizes stay in range."""
import numpy as np

from paper_1601_00159_gb300 import workloads as wl


def test_batching_inserts_are_new_keys_in_every_round():
    """Every round's inserts are keys no index holds and no earlier round inserted, so a
    bench that gives every call a fresh round merges and rebuilds every index every call."""
    w = wl.batching(count=12, hi_log=12, qhi_log=10)
    seen = [set(k.tolist()) for k in w.keys]
    for r in range(5):
        for i, b in enumerate(w.batches(r)):
            ins = b.keys[b.ops == wl.OP_INSERT]
            assert len(np.unique(ins)) == len(ins), (r, i)
            assert not (set(ins.tolist()) & seen[i]), (r, i)
            seen[i] |= set(ins.tolist())
            assert (b.keys < np.uint64(1 << 63)).all()


def test_mid_inserts_are_new_and_hits_are_live():
    w = wl.mid(n0=1 << 12, q=1 << 10, n_batches=4)
    live = set(w.keys.tolist())
    for b in w.batches():
        ins = b.keys[b.ops == wl.OP_INSERT]
        assert not (set(ins.tolist()) & live) and len(np.unique(ins)) == len(ins)
        srch = b.keys[b.ops == wl.OP_SEARCH].tolist()
        hits = sum(k in live for k in srch)
        assert 0.35 * len(srch) < hits < 0.65 * len(srch)  # half hits, half misses
        live |= set(ins.tolist())


def test_skewed_queries_stay_on_the_key_set_with_a_hot_head():
    """Inserts are overwrites or revivals and deletes hit stored keys; the hottest key
    takes about 1/zeta(n, 0.99) of the queries."""
    n, q = 1 << 14, 1 << 14
    w = wl.skewed(n=n, q=q, n_batches=2)
    keyset = set(w.keys.tolist())
    for b in w.batches():
        assert set(b.keys.tolist()) <= keyset
        fr = np.bincount(b.ops, minlength=3) / q
        assert abs(fr[0] - 0.9) < 0.02 and abs(fr[1] - 0.05) < 0.01 and abs(fr[2] - 0.05) < 0.01
        _, counts = np.unique(b.keys, return_counts=True)
        top = counts.max() / q
        expect = 1.0 / wl.zeta(n, 0.99)
        assert 0.7 * expect < top < 1.3 * expect


def test_serving_request_stream_shape():
    w = wl.serving(n=1 << 12, nreq=3000)
    assert w.sizes.min() >= 1 and w.sizes.max() <= 4096
    assert int(w.sizes.sum()) == len(w.ops) == len(w.qkeys) == len(w.qvals)
    assert set(w.qkeys.tolist()) <= set(w.keys.tolist())
    fr_ins = float((w.ops == wl.OP_INSERT).mean())
    assert abs(fr_ins - 0.05) < 0.01
    # log-uniform sizes in [1, 4096]: the median is near 2^6
    assert 32 <= float(np.median(w.sizes)) <= 128
