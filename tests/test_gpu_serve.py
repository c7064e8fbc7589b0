"""Serving form (pi_server_*): continuous batching gives every request the result it
gets alone.

Requests of log-uniform sizes (Zipf keys over the index, searches, inserts of existing
and new keys, deletes, a few invalid queries) go through the server, which coalesces
them into batches and keeps several in flight. Each request's results must equal (a)
the results of running the requests one by one through pi_execute_batch on a twin
index, and (b) the oracle's. The final states must agree too. Exact equality: the path
is integer-only.
"""
import numpy as np
import pytest

from paper_1601_00159_gb300 import workloads as wl
from tests.parity import assert_results_equal, assert_state_equal, make_index, results_np, to_dev

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


def host_results(r):
    vals = r[:, 0].view(np.uint64)
    status = (r[:, 1].view(np.uint64) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    reserved = (r[:, 1].view(np.uint64) >> np.uint64(32)).astype(np.uint32)
    return vals, status, reserved


def request_stream(seed, keys, nreq, max_size):
    s = wl.stream_seed(seed, 1)
    u = wl.uniform01(s, 0, nreq)
    sizes = np.maximum(1, np.floor(2.0 ** (u * np.log2(max_size)))).astype(np.uint32)
    q = int(sizes.sum())
    z = wl.Zipf(len(keys), 0.9)
    hot = keys[wl.scramble(z.ranks(wl.uniform01(s, nreq, q)), len(keys), seed)]
    kind = wl.bounded(s, nreq + q, q, 100)
    new = wl.u64_stream(s, nreq + 2 * q, q) >> np.uint64(1)
    bkeys = np.where(kind < 85, hot, np.where(kind < 95, new, hot))
    ops = np.where(kind < 80, 0, np.where(kind < 95, 1, 2)).astype(np.uint8)
    ops = np.where(kind == 99, np.uint8(9), ops)
    return sizes, ops, bkeys.astype(np.uint64), wl.u64_stream(s, nreq + 3 * q, q)


def test_results_alone_equal_results_in_the_mix(orc_mod):
    import torch
    from paper_1601_00159_gb300 import Server
    n = 1 << 15
    keys = wl.distinct_keys(21, np.arange(n))
    vals = wl.splitmix64(keys)
    alone = make_index(keys, vals, 0.25, 77)
    mixed = make_index(keys, vals, 0.25, 77)
    orc = orc_mod.Oracle(keys, vals, 0.25, 77)
    sizes, ops, bkeys, bvals = request_stream(21, keys, 400, 2048)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    # (a) one request per batch, in arrival order
    got_alone = []
    for i in range(len(sizes)):
        a, b = offs[i], offs[i + 1]
        res = alone.execute(to_dev(ops[a:b], torch.uint8), to_dev(bkeys[a:b], torch.int64),
                            to_dev(bvals[a:b], torch.int64))
        got_alone.append(results_np(res))
    # (b) the server: every arrival at t = 0, so requests coalesce and batches overlap
    srv = Server(mixed, max_batch=4096, slots=3)
    res, lat = srv.replay(ops, bkeys, bvals, sizes, np.zeros(len(sizes)))
    st = srv.stats()
    srv.close()
    exp_v, exp_s = orc.execute(ops, bkeys, bvals)
    mv, ms_, mr = host_results(res)
    for i in range(len(sizes)):
        a, b = offs[i], offs[i + 1]
        assert_results_equal(got_alone[i], (exp_v[a:b], exp_s[a:b]), f"alone request {i}")
        assert_results_equal((mv[a:b], ms_[a:b], mr[a:b]), (exp_v[a:b], exp_s[a:b]), f"mixed request {i}")
    assert st["requests"] == len(sizes) and st["queries"] == int(sizes.sum())
    assert st["batches"] < len(sizes), st          # requests were coalesced
    assert st["max_in_flight"] >= 2, st            # batches overlapped on the device
    assert (lat > 0).all() and st["p99_s"] >= st["p50_s"] > 0
    assert_state_equal(alone, orc, "alone end")
    assert_state_equal(mixed, orc, "mixed end")


def test_poisson_replay_and_admission(orc_mod):
    """Poisson arrivals through a ring that holds only two batches: submissions wait for
    space, and every result is still exact."""
    from paper_1601_00159_gb300 import Server
    n = 1 << 14
    keys = wl.distinct_keys(22, np.arange(n))
    vals = wl.splitmix64(keys)
    idx = make_index(keys, vals, 0.25, 78)
    orc = orc_mod.Oracle(keys, vals, 0.25, 78)
    sizes, ops, bkeys, bvals = request_stream(22, keys, 600, 4096)
    gaps = -np.log(np.maximum(wl.uniform01(wl.stream_seed(22, 9), 0, len(sizes)), 1e-12)) * 20e-6
    srv = Server(idx, max_batch=8192, slots=2, ring_queries=16384)
    res, lat = srv.replay(ops, bkeys, bvals, sizes, np.cumsum(gaps))
    st = srv.stats(reset=True)
    assert st["requests"] == len(sizes)
    srv.close()
    exp_v, exp_s = orc.execute(ops, bkeys, bvals)
    assert_results_equal(host_results(res), (exp_v, exp_s), "poisson")
    assert_state_equal(idx, orc, "poisson end")


def test_server_submit_and_wait_by_hand(orc_mod):
    from paper_1601_00159_gb300 import PiError, Server
    keys = wl.distinct_keys(23, np.arange(5000))
    idx = make_index(keys, keys, 0.5, 3)
    orc = orc_mod.Oracle(keys, keys, 0.5, 3)
    # the ring holds every request of this single-threaded test: submit waits while it
    # is full, and only a later wait would free it
    srv = Server(idx, max_batch=1000, slots=2, ring_queries=1 << 15)
    with pytest.raises(PiError):
        srv.submit(np.zeros(1001, np.uint8), np.zeros(1001, np.uint64), np.zeros(1001, np.uint64))
    reqs = []
    for i in range(30):
        q = 1 + (i * 37) % 700
        s = wl.stream_seed(23, 100 + i)
        o = wl.bounded(s, 0, q, 3).astype(np.uint8)
        k = np.where(wl.bounded(s, q, q, 2) == 0, keys[wl.bounded(s, 2 * q, q, 5000)], wl.u64_stream(s, 3 * q, q) >> np.uint64(2))
        v = wl.u64_stream(s, 4 * q, q)
        reqs.append((srv.submit(o, k, v), o, k.astype(np.uint64), v))
    with pytest.raises(PiError):
        srv.wait(reqs[1][0], len(reqs[1][1]))  # not the oldest
    for t, o, k, v in reqs:
        r, lat = srv.wait(t, len(o))
        assert lat > 0
        ev, es = orc.execute(o, k, v)
        assert_results_equal(host_results(r), (ev, es), f"ticket {t}")
    srv.close()
    assert_state_equal(idx, orc, "by hand end")
