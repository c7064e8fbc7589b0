"""Pins for the oracle (CPU only): each test checks it against something other than
itself, so that a dropped term, a wrong sign or index or a swapped operand fails.

* published SplitMix64 outputs (tests/golden/splitmix64.txt);
* the paper's worked example and a hand-derived same-key chain (tests/golden/);
* brute force: a Python dict replay of the batch in arrival order, which is the
  serializability definition of Section 4.2, on thousands of tiny dense inputs;
* structure invariants of Section 3.1 (levels sorted, each a subset of the one below);
* closed forms of Section 5.1: P(height >= l) = p^(l-1), top height ~ log_{1/p} N,
  mean gap 1/p between consecutive keys of the next level.
"""
import math
import os

import numpy as np
import pytest

from paper_1601_00159_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M64 = (1 << 64) - 1


def read_golden_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def read_example(name):
    init, queries, final = [], [], []
    for row in read_golden_table(name):
        tag, vals = row[0], [int(x) for x in row[1:]]
        {"initial": init, "query": queries, "final": final}[tag].append(vals)
    return init, queries, final


def replay(init_keys, init_vals, batches):
    """Brute force: a dict, queries applied one at a time in arrival order."""
    d = {}
    for k, v in zip(init_keys.tolist(), init_vals.tolist()):
        d[k] = v
    out = []
    for b in batches:
        rv = np.zeros(len(b), np.uint64)
        rs = np.zeros(len(b), np.uint32)
        for i, (op, k, v) in enumerate(zip(b.ops.tolist(), b.keys.tolist(), b.vals.tolist())):
            if op > 2 or k == M64:
                rs[i] = 2
                continue
            if k in d:
                rs[i], rv[i] = 1, d[k]
            if op == 1:
                d[k] = v
            elif op == 2:
                d.pop(k, None)
        out.append((rv, rs))
    return out, d


def test_splitmix64_golden(oracle_mod):
    gamma = 0x9E3779B97F4A7C15
    for idx, hexval in read_golden_table("splitmix64.txt"):
        x = (int(idx) * gamma) & M64
        assert oracle_mod.splitmix64(x) == int(hexval, 16)
        assert int(wl.splitmix64(np.uint64(x))) == int(hexval, 16)


@pytest.mark.parametrize("name", ["paper_example.txt", "same_key_chain.txt"])
def test_worked_examples(oracle_mod, name):
    init, queries, final = read_example(name)
    ik = np.array([r[0] for r in init], np.uint64)
    iv = np.array([r[1] for r in init], np.uint64)
    o = oracle_mod.Oracle(ik, iv, 0.5, 12345)
    ops = np.array([q[0] for q in queries], np.uint8)
    keys = np.array([q[1] for q in queries], np.uint64)
    vals = np.array([q[2] for q in queries], np.uint64)
    rv, rs = o.execute(ops, keys, vals)
    assert rs.tolist() == [q[3] for q in queries]
    assert rv.tolist() == [q[4] for q in queries]
    fk, fv = o.export()
    assert fk.tolist() == [r[0] for r in final]
    assert fv.tolist() == [r[1] for r in final]


def _levels_from_definition(oracle_mod, keys, seed, b):
    """Level l = live keys with height >= l (Definition 1 / Section 3.1)."""
    hs = np.array([oracle_mod.height(seed, b, int(k)) for k in keys.tolist()], np.int64)
    top = int(hs.max()) if len(hs) else 0
    return [keys[hs >= l] for l in range(1, top + 1)]


def _check_structure(oracle_mod, o, seed, b, live_keys):
    levels = [o.level(l) for l in range(1, o.num_levels() + 1)]
    expect = _levels_from_definition(oracle_mod, np.sort(live_keys), seed, b)
    assert len(levels) == len(expect)
    for got, exp in zip(levels, expect):
        assert np.array_equal(got, exp)
    for l, lev in enumerate(levels):
        assert np.all(lev[1:] > lev[:-1]), "level not strictly increasing"
        if l > 0:
            assert np.all(np.isin(lev, levels[l - 1])), "level not a subset of the level below"


def test_bruteforce_replay_many_seeds(oracle_mod):
    rng = np.random.default_rng(0)
    for seed in range(1500):
        n = int(rng.integers(0, 40))
        q = int(rng.integers(0, 120))
        key_range = int(rng.choice([3, 8, 32, 64]))
        p = float(rng.choice([0.5, 0.25, 0.125, 0.0625]))
        w = wl.random_small(seed, n, q, key_range, p=p, n_batches=3)
        o = oracle_mod.Oracle(w.keys, w.vals, w.promote_p, w.hash_seed)
        expected, final = replay(w.keys, w.vals, w.batches)
        for batch, (ev, es) in zip(w.batches, expected):
            rv, rs = o.execute(batch.ops, batch.keys, batch.vals)
            assert np.array_equal(rs, es), f"seed {seed}: status mismatch"
            assert np.array_equal(rv, ev), f"seed {seed}: value mismatch"
        fk, fv = o.export()
        assert fk.tolist() == sorted(final)
        assert fv.tolist() == [final[k] for k in sorted(final)]
        if seed % 10 == 0:
            _check_structure(oracle_mod, o, w.hash_seed, o.b, fk)


def test_structure_after_mixed_batches(oracle_mod):
    seed = 77
    n = 1 << 13
    keys = wl.distinct_keys(seed, np.arange(n))
    vals = wl.u64_stream(np.uint64(5), 0, n)
    o = oracle_mod.Oracle(keys, vals, 0.25, 999)
    live = dict(zip(keys.tolist(), vals.tolist()))
    for b in range(3):
        s = wl.stream_seed(seed, b)
        q = 4096
        ops = wl.bounded(s, 0, q, 3).astype(np.uint8)
        pick = wl.bounded(s, q, q, n + 2048)
        bkeys = wl.distinct_keys(seed, pick)
        bvals = wl.u64_stream(s, 2 * q, q)
        batch = wl.Batch(ops, bkeys, bvals)
        (ev, es), = replay(np.array(list(live.keys()), np.uint64),
                           np.array(list(live.values()), np.uint64), [batch])[0]
        rv, rs = o.execute(ops, bkeys, bvals)
        assert np.array_equal(rs, es) and np.array_equal(rv, ev)
        _, live = replay(np.array(list(live.keys()), np.uint64),
                         np.array(list(live.values()), np.uint64), [batch])
        fk, _ = o.export()
        assert fk.tolist() == sorted(live)
        _check_structure(oracle_mod, o, 999, 2, fk)


@pytest.mark.parametrize("b", [1, 2, 3, 4])
def test_height_distribution_closed_form(oracle_mod, b):
    """P(height >= l) = p^(l-1) (Definition 1; Section 5.1), within 6 sigma."""
    n = 1 << 16
    p = 2.0 ** -b
    o = oracle_mod.Oracle(wl.distinct_keys(b, np.arange(n)), np.zeros(n, np.uint64), p, 4242 + b)
    hmax = min(32, 64 // b)
    assert o.num_levels() <= hmax
    for l in range(2, 6):
        cnt = len(o.level(l))
        mu = n * p ** (l - 1)
        sd = math.sqrt(mu * (1 - p ** (l - 1)))
        assert abs(cnt - mu) <= 6 * sd + 1, (l, cnt, mu)


@pytest.mark.parametrize("b,logn", [(1, 14), (2, 16), (2, 18), (3, 15)])
def test_top_height_and_gap_closed_form(oracle_mod, b, logn):
    """H ~ ceil(-log_P N) (Section 5.1) and mean gap 1/P between next-level keys."""
    n = 1 << logn
    p = 2.0 ** -b
    o = oracle_mod.Oracle(wl.distinct_keys(logn, np.arange(n)), np.zeros(n, np.uint64), p, 31 * b)
    h_model = math.ceil(math.log(n) / math.log(1 / p))
    assert abs(o.num_levels() - h_model) <= 3
    l1, l2 = o.level(1), o.level(2)
    pos = np.searchsorted(l1, l2)
    gaps = np.diff(pos)
    assert abs(gaps.mean() - 1 / p) < 6 * math.sqrt((1 - p) / p ** 2 / len(gaps)) + 0.01


def test_height_known_structure(oracle_mod):
    """The height depends on ctz of splitmix64(key ^ splitmix64(seed)) divided by b.
    Pins the trailing-zero reading against the leading-zero one: find keys whose hash
    has many trailing zeros and no leading zeros, and check their heights."""
    seed = 2024
    sm = oracle_mod.splitmix64
    mix = sm(seed)
    found = 0
    for key in range(200000):
        h = sm(key ^ mix)
        tz = (h & -h).bit_length() - 1
        if tz >= 4 and (h >> 63) == 1:
            assert oracle_mod.height(seed, 1, key) == 1 + tz
            assert oracle_mod.height(seed, 2, key) == 1 + tz // 2
            assert oracle_mod.height(seed, 4, key) == 1 + tz // 4
            found += 1
        if tz == 0:
            assert oracle_mod.height(seed, 1, key) == 1
    assert found > 100


def test_height_cap_known_answers(oracle_mod):
    """The cap of the height rule: Hmax - 1 levels above the storage level at most, and a
    hash of 0 counted as 64 trailing zeros. The keys are built to hit chosen hashes by
    inverting splitmix64 (tests/hashkeys.py), and the expected heights are the
    hand-derived table tests/golden/height_cap.txt."""
    from tests.hashkeys import hash_with_trailing_zeros, key_with_hash, splitmix64_inverse
    sm = oracle_mod.splitmix64
    rows = [tuple(int(x) for x in r) for r in read_golden_table("height_cap.txt")]
    assert len(rows) >= 20
    for seed in (0, 7, 2024):
        mix = sm(seed)
        for b, tz, expected in rows:
            for salt in (0, 12345, M64 >> 3):
                h = hash_with_trailing_zeros(tz, salt)
                assert sm(splitmix64_inverse(h)) == h
                key = key_with_hash(h, mix)
                assert sm(key ^ mix) == h
                if key == M64:
                    continue
                assert oracle_mod.height(seed, b, key) == expected, (seed, b, tz, salt)
    # Built into an index, such keys set its number of levels: Hmax for every b.
    for b, hmax in ((1, 32), (2, 32), (3, 21), (4, 16)):
        seed = 100 + b
        mix = sm(seed)
        capped = sorted({key_with_hash(0, mix), key_with_hash(1 << 63, mix)} - {M64})
        keys = capped + [int(k) for k in wl.distinct_keys(b, np.arange(200))]
        keys = np.array(sorted(set(keys)), np.uint64)
        o = oracle_mod.Oracle(keys, np.arange(len(keys), dtype=np.uint64), 2.0 ** -b, seed)
        assert o.num_levels() == hmax
        assert o.level(hmax).tolist() == capped
        o.close()


def test_create_duplicates_last_wins_and_rejects_reserved(oracle_mod):
    keys = np.array([5, 3, 5, 9, 3, 5], np.uint64)
    vals = np.array([1, 2, 3, 4, 5, 6], np.uint64)
    o = oracle_mod.Oracle(keys, vals, 0.5, 1)
    k, v = o.export()
    assert k.tolist() == [3, 5, 9] and v.tolist() == [5, 6, 4]
    with pytest.raises(ValueError):
        oracle_mod.Oracle(np.array([1, M64], np.uint64), np.zeros(2, np.uint64), 0.5, 1)
    with pytest.raises(ValueError):
        oracle_mod.Oracle(keys, vals, 0.3, 1)


def test_special_cases(oracle_mod):
    n = 1000
    keys = wl.distinct_keys(9, np.arange(n))
    vals = wl.splitmix64(keys)
    o = oracle_mod.Oracle(keys, vals, 0.25, 7)
    before = [o.level(l) for l in range(1, o.num_levels() + 1)]
    # an all-search batch changes nothing
    q = np.concatenate([keys[:50], wl.distinct_keys(9, np.arange(n, n + 50))])
    rv, rs = o.execute(np.zeros(100, np.uint8), q, np.zeros(100, np.uint64))
    assert rs[:50].tolist() == [1] * 50 and rs[50:].tolist() == [0] * 50
    assert np.array_equal(rv[:50], vals[:50])
    after = [o.level(l) for l in range(1, o.num_levels() + 1)]
    assert all(np.array_equal(a, b) for a, b in zip(before, after)) and len(before) == len(after)
    # a key below every stored key, insert then search, delete then insert revives
    lo = int(keys.min())
    if lo > 0:
        rv, rs = o.execute(np.array([0, 1, 0], np.uint8), np.array([lo - 1] * 3, np.uint64),
                           np.array([0, 11, 0], np.uint64))
        assert rs.tolist() == [0, 0, 1] and rv.tolist() == [0, 0, 11]
    k0 = int(keys[0])
    rv, rs = o.execute(np.array([2, 0, 1, 0], np.uint8), np.array([k0] * 4, np.uint64),
                       np.array([0, 0, 77, 0], np.uint64))
    assert rs.tolist() == [1, 0, 0, 1] and rv.tolist() == [int(vals[0]), 0, 0, 77]


def test_zipf_generator_rank0_frequency():
    """Gray et al.'s generator puts mass 1/zeta(n, theta) on rank 0 exactly."""
    for n, theta in [(1 << 16, 0.99), (1 << 20, 0.9), (1000, 0.5)]:
        z = wl.Zipf(n, theta)
        u = wl.uniform01(np.uint64(n), 0, 1 << 20)
        r = z.ranks(u)
        assert r.min() >= 0 and r.max() < n
        f = float(np.mean(r == 0))
        mu = 1 / z.zetan
        assert abs(f - mu) < 6 * math.sqrt(mu * (1 - mu) / len(u))
    assert wl.zeta(1000, 0.0) == 1000.0
    assert abs(wl.zeta(1 << 20, 2.0) - (math.pi ** 2 / 6 - 1.0 / (1 << 20))) < 1e-9


def test_distinct_keys_are_distinct_and_below_2_63():
    idx = np.concatenate([np.arange(1 << 18), (1 << 62) + np.arange(1 << 16)])
    k = wl.distinct_keys(5, idx)
    assert len(np.unique(k)) == len(idx)
    assert int(k.max()) < (1 << 63)


def test_range_search_brute_force(oracle_mod):
    """Range search (Section 3.2.5) against a brute-force filter of a Python dict that
    replays the same queries: for every range, the live pairs with lo <= key <= hi in key
    order. Ranges include empty ones (lo > hi), single keys, the whole key space, bounds at
    0 and 2^64-1, and bounds inside and outside the key set."""
    rng = np.random.default_rng(11)
    for trial in range(60):
        n = int(rng.integers(0, 300))
        keys = np.unique(rng.integers(0, 1 << 12, n, dtype=np.uint64))
        vals = rng.integers(0, 1 << 62, len(keys), dtype=np.uint64)
        b = wl.random_small(trial, 1, 200, 1 << 12, p=0.5, n_batches=1).batches[0]
        orc = oracle_mod.Oracle(keys, vals, 0.25 if trial % 2 else 0.5, trial)
        orc.execute(b.ops, b.keys, b.vals)
        _, d = replay(keys, vals, [b])
        live = sorted(d)
        q = 40
        lo = rng.integers(0, 1 << 12, q, dtype=np.uint64)
        width = rng.integers(0, 300, q, dtype=np.uint64)
        hi = lo + width
        lo[:4] = [0, 5, 7, 0]
        hi[:4] = [M64, 4, 7, 0]          # everything, lo > hi, a single key, [0, 0]
        if live:
            lo[4] = hi[4] = live[len(live) // 2]  # exactly one live key
        offs, rk, rv = orc.range(lo, hi)
        assert offs[0] == 0 and len(offs) == q + 1
        for i in range(q):
            exp = [k for k in live if int(lo[i]) <= k <= int(hi[i])]
            got = rk[offs[i]:offs[i + 1]].tolist()
            assert got == exp, (trial, i, int(lo[i]), int(hi[i]))
            assert rv[offs[i]:offs[i + 1]].tolist() == [d[k] for k in exp]
        orc.close()
