"""Shared harness of the GPU parity tests: run the same seeded batches through the
CUDA path (via the C ABI binding) and through the oracle, and compare bit for bit."""
from __future__ import annotations

import numpy as np


def to_dev(a: np.ndarray, dtype):
    import torch
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def results_np(res):
    r = res.cpu().numpy()
    vals = r[:, 0].view(np.uint64)
    status = (r[:, 1].view(np.uint64) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    reserved = (r[:, 1].view(np.uint64) >> np.uint64(32)).astype(np.uint32)
    return vals, status, reserved


def make_index(keys, vals, p, seed, config=None, route=False):
    """An index on the GPU (the library's defaults: every batch on the level-synchronous
    pipeline). route=True sets small_batches = 1: batches of at most 2^16 queries on
    indices of at most 2^20 keys then run as one thread-block-cluster launch."""
    import torch
    from paper_1601_00159_gb300 import Index
    cfg = dict(config or {})
    if route:
        cfg.setdefault("small_batches", 1)
    return Index(to_dev(keys, torch.int64), to_dev(vals, torch.int64), p, seed, cfg or None)


def run_batch(idx, batch):
    import torch
    res = idx.execute(to_dev(batch.ops, torch.uint8), to_dev(batch.keys, torch.int64),
                      to_dev(batch.vals, torch.int64))
    return results_np(res)


def assert_results_equal(got, expected, ctx=""):
    gv, gs, gr = got
    ev, es = expected
    assert gs.shape == es.shape
    bad = np.nonzero((gs != es) | (gv != ev))[0]
    assert len(bad) == 0, (f"{ctx}: {len(bad)} of {len(es)} results differ; first at {bad[:5]}: "
                           f"gpu {list(zip(gs[bad[:5]], gv[bad[:5]]))} oracle {list(zip(es[bad[:5]], ev[bad[:5]]))}")
    assert not gr.any(), f"{ctx}: reserved field not zero"


def assert_state_equal(idx, orc, ctx="", check_levels=True):
    k, v = idx.export()
    gk = k.cpu().numpy().view(np.uint64)
    gv = v.cpu().numpy().view(np.uint64)
    ok, ov = orc.export()
    assert len(gk) == len(ok), f"{ctx}: {len(gk)} live keys on GPU, oracle {len(ok)}"
    assert np.array_equal(gk, ok), f"{ctx}: live key sets differ"
    assert np.array_equal(gv, ov), f"{ctx}: values differ"
    info = idx.info()
    assert info["live"] == len(ok)
    assert idx.size() == len(ok), f"{ctx}: pi_size {idx.size()} vs oracle {len(ok)}"
    assert idx.status() == 0, f"{ctx}: device error status {idx.status()}"
    # The storage layer as stored: sorted, its live nodes exactly the oracle's keys, and
    # as many delete-flagged nodes as pi_info reports.
    st_k, st_m = idx.export_storage()
    sk = st_k.cpu().numpy().view(np.uint64)
    sm = st_m.cpu().numpy()
    assert len(sk) == info["size"], f"{ctx}: storage export size"
    assert np.all(sk[1:] > sk[:-1]), f"{ctx}: storage layer not strictly increasing"
    live = (sm & 0x80) == 0
    assert int((~live).sum()) == info["tombstones"], f"{ctx}: delete-flagged node count"
    assert np.array_equal(sk[live], ok), f"{ctx}: live storage nodes differ from the oracle's keys"
    del live, sm
    if not check_levels:
        return info
    top = orc.num_levels()
    assert info["top_level"] == max(top, 1), f"{ctx}: top level {info['top_level']} vs {top}"
    assert idx.num_levels() == max(top, 1), f"{ctx}: pi_num_levels {idx.num_levels()} vs {top}"
    prev_keys = ok
    for level in range(2, top + 1):
        lv = idx.export_level(level)
        exp = orc.level(level)
        assert info["level_size"][level] == len(exp)
        if lv is None:
            assert level < info["bottom_built"], f"{ctx}: level {level} missing"
            prev_keys = exp
            continue
        lk = lv[0].cpu().numpy().view(np.uint64)
        ld = lv[1].cpu().numpy().astype(np.int64)
        assert np.array_equal(lk, exp), f"{ctx}: level {level} differs"
        if level > info["bottom_built"]:
            assert np.array_equal(prev_keys[ld], lk), f"{ctx}: down pointers of level {level} wrong"
        else:
            # the lowest built level points at storage positions, delete-flagged nodes
            # included (Section 3.1: each level a subsequence of the one below)
            assert np.array_equal(sk[ld], lk), f"{ctx}: storage down pointers of level {level} wrong"
        prev_keys = exp
    return info
