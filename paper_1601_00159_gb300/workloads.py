"""Seeded synthetic workloads shaped like the paper's experiments (Section 6, Table 2).

This module only draws inputs: keys, values, op codes and Zipf ranks. It holds none
of the index method's arithmetic (no tower heights, no ordering logic), so both the
CUDA path and the oracle can be fed from it without sharing any of the method.

The paper measures on YCSB-generated workloads (Section 6: uniform or Zipfian keys,
update ratios of YCSB A/B/C). YCSB is not available here; the generators below are
stand-ins with the same shapes, written from the published definitions:

* Random numbers: the SplitMix64 counter stream (Steele, Lea and Flood, "Fast
  splittable pseudorandom number generators", OOPSLA 2014): output i of a stream
  with seed ``s`` is ``mix64(s + (i + 1) * 0x9E3779B97F4A7C15)``. Counter based, so a
  whole array is one vectorised expression.
* Distinct keys: key ``i`` is ``F(i)`` for a seeded bijection ``F`` on [0, 2^63), built
  from steps that are each invertible modulo 2^63 (add, multiply by an odd constant,
  xor with a right shift). Distinct indices give distinct keys, so "new" keys and
  "miss" keys are drawn from index ranges that the initial set does not use.
* Zipf ranks: the method of Gray, Sundaresan, Englert, Baclawski and Weinberger,
  "Quickly generating billion-record synthetic databases" (SIGMOD 1994), the
  generator YCSB uses. Rank 0 is the hottest; ranks are scattered over the key set by
  a seeded affine bijection so hot keys are not clustered in key order.

Everything is numpy uint64 arithmetic, which wraps modulo 2^64.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
MASK63 = np.uint64((1 << 63) - 1)
RESERVED_KEY = np.uint64(0xFFFFFFFFFFFFFFFF)

OP_SEARCH, OP_INSERT, OP_DELETE = 0, 1, 2


def mix64(z: np.ndarray) -> np.ndarray:
    """The SplitMix64 output function applied elementwise (Steele et al. 2014)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def splitmix64(x) -> np.ndarray:
    """splitmix64(x) = mix64(x + gamma): one step of the generator from state x."""
    with np.errstate(over="ignore"):
        return mix64(np.asarray(x, dtype=np.uint64) + GAMMA)


def stream_seed(master: int, tag: int) -> np.uint64:
    """Derive an independent stream seed from a master seed and a purpose tag."""
    s = splitmix64(np.uint64(master & 0xFFFFFFFFFFFFFFFF))
    return splitmix64(s ^ np.uint64(tag & 0xFFFFFFFFFFFFFFFF))


def u64_stream(seed: np.uint64, start: int, count: int) -> np.ndarray:
    """Outputs start..start+count-1 of the SplitMix64 counter stream with this seed."""
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(np.uint64(seed) + i * GAMMA)


def uniform01(seed: np.uint64, start: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of the stream."""
    return (u64_stream(seed, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def bounded(seed: np.uint64, start: int, count: int, bound: int) -> np.ndarray:
    """Integers in [0, bound) by multiply-high of the top 32 bits (bias < 2^-32 * bound)."""
    hi = (u64_stream(seed, start, count) >> np.uint64(32)).astype(np.uint64)
    with np.errstate(over="ignore"):
        return ((hi * np.uint64(bound)) >> np.uint64(32)).astype(np.int64)


def distinct_keys(seed: int, idx: np.ndarray) -> np.ndarray:
    """F(idx): a seeded bijection of [0, 2^63) applied to key indices.

    Each step is invertible modulo 2^63: adding a constant, multiplying by an odd
    constant, and x ^ (x >> k). So distinct indices always map to distinct keys, and
    every key is below 2^63 (never the reserved key 2^64-1).
    """
    s = stream_seed(seed, 0xF00D)
    a = np.uint64((int(s) | 1) & int(MASK63))
    c = np.uint64(int(splitmix64(s)) & int(MASK63))
    x = np.asarray(idx, dtype=np.uint64) & MASK63
    with np.errstate(over="ignore"):
        x = (x + c) & MASK63
        x = (x * np.uint64(0xBF58476D1CE4E5B9)) & MASK63
        x = x ^ (x >> np.uint64(29))
        x = (x * a) & MASK63
        x = x ^ (x >> np.uint64(32))
        x = (x * np.uint64(0x94D049BB133111EB)) & MASK63
        x = x ^ (x >> np.uint64(31))
    return x


def zeta(n: int, theta: float) -> float:
    """sum_{i=1..n} i^-theta in float64, summed in chunks."""
    total = 0.0
    chunk = 1 << 22
    for lo in range(1, n + 1, chunk):
        hi = min(n, lo + chunk - 1)
        i = np.arange(lo, hi + 1, dtype=np.float64)
        total += float(np.sum(i ** (-theta)))
    return total


@dataclasses.dataclass
class Zipf:
    """Zipf(theta) ranks in [0, n) by Gray et al. (1994); rank 0 is the most frequent."""

    n: int
    theta: float

    def __post_init__(self):
        self.zetan = zeta(self.n, self.theta)
        self.zeta2 = 1.0 + 2.0 ** (-self.theta)
        self.alpha = 1.0 / (1.0 - self.theta)
        self.eta = (1.0 - (2.0 / self.n) ** (1.0 - self.theta)) / (1.0 - self.zeta2 / self.zetan)

    def ranks(self, u: np.ndarray) -> np.ndarray:
        uz = u * self.zetan
        r = np.floor(self.n * (self.eta * u - self.eta + 1.0) ** self.alpha)
        r = np.clip(r, 0, self.n - 1).astype(np.int64)
        r = np.where(uz < 1.0 + 0.5 ** self.theta, 1, r)
        r = np.where(uz < 1.0, 0, r)
        return r


def scramble(ranks: np.ndarray, n: int, seed: int) -> np.ndarray:
    """A seeded affine bijection of [0, n): r -> (a*r + c) mod n with gcd(a, n) = 1."""
    assert n <= (1 << 31)
    s = int(stream_seed(seed, 0x5C7A))
    a = (s | 1) % n or 1
    while math.gcd(a, n) != 1:
        a += 1
    c = (s >> 17) % n
    return (ranks.astype(np.int64) * a + c) % n


@dataclasses.dataclass
class Batch:
    ops: np.ndarray    # uint8[Q]
    keys: np.ndarray   # uint64[Q]
    vals: np.ndarray   # uint64[Q]; read only where ops == insert

    def __len__(self):
        return len(self.ops)


@dataclasses.dataclass
class Workload:
    name: str
    keys: np.ndarray       # initial keys (uint64)
    vals: np.ndarray       # initial values (uint64)
    promote_p: float
    hash_seed: int
    batches: list          # list[Batch] or a callable producing them lazily
    rebuild_each_batch: bool = True


def _mixed_ops(seed: np.uint64, start: int, q: int, fr_insert: float, fr_delete: float) -> np.ndarray:
    u = uniform01(seed, start, q)
    ops = np.full(q, OP_SEARCH, dtype=np.uint8)
    ops[u < fr_insert + fr_delete] = OP_DELETE
    ops[u < fr_insert] = OP_INSERT
    return ops


def tiny(seed: int = 1, n: int = 1 << 16, q: int = 1 << 14) -> Workload:
    """Plain PI, tiny: n distinct uniform keys in [0, 2^63), value = splitmix64(key),
    promotion p = 1/2; one all-search batch, half hits and half uniform misses."""
    keys = distinct_keys(seed, np.arange(n))
    vals = splitmix64(keys)
    s = stream_seed(seed, 1)
    hit = u64_stream(s, 0, q) & np.uint64(1)
    hit_idx = bounded(s, q, q, n)
    miss_idx = (np.uint64(1) << np.uint64(62)) + np.arange(q, dtype=np.uint64)
    bkeys = np.where(hit == 1, keys[hit_idx], distinct_keys(seed, miss_idx))
    batch = Batch(np.zeros(q, np.uint8), bkeys.astype(np.uint64), np.zeros(q, np.uint64))
    return Workload("tiny", keys, vals, 0.5, int(stream_seed(seed, 2)), [batch], True)


def mid(seed: int = 2, n0: int = 1 << 24, q: int = 1 << 20, n_batches: int = 16) -> Workload:
    """Plain PI, mid: n0 distinct uniform keys, p = 1/4; batches of q queries, 50% search
    (half hits over the live keys, half misses) / 50% insert of new uniform keys, ops
    interleaved at random; rebuild after each batch."""
    keys = distinct_keys(seed, np.arange(n0))
    vals = u64_stream(stream_seed(seed, 3), 0, n0)

    def batches():
        live = n0
        miss_base = 1 << 62
        for b in range(n_batches):
            s = stream_seed(seed, 100 + b)
            ops = np.where(uniform01(s, 0, q) < 0.5, OP_INSERT, OP_SEARCH).astype(np.uint8)
            ins = ops == OP_INSERT
            n_ins = int(ins.sum())
            bkeys = np.empty(q, np.uint64)
            bkeys[ins] = distinct_keys(seed, np.arange(live, live + n_ins))
            n_s = q - n_ins
            hit = (u64_stream(s, q, n_s) & np.uint64(1)) == 1
            hit_keys = distinct_keys(seed, bounded(s, 2 * q, n_s, live))
            miss_keys = distinct_keys(seed, np.arange(miss_base, miss_base + n_s))
            miss_base += n_s
            bkeys[~ins] = np.where(hit, hit_keys, miss_keys)
            bvals = u64_stream(s, 3 * q, q)
            live += n_ins
            yield Batch(ops, bkeys, bvals)

    return Workload("mid", keys, vals, 0.25, int(stream_seed(seed, 4)), batches, True)


def skewed(seed: int = 3, n: int = 1 << 27, q: int = 1 << 22, n_batches: int = 32,
           theta: float = 0.99) -> Workload:
    """Plain PI, skewed: n distinct uniform keys with value = splitmix64(key), p = 1/4;
    batches of q queries with Zipf(theta) keys over the initial key set (ranks
    scattered by a seeded bijection), 90% search / 5% insert / 5% delete."""
    keys = distinct_keys(seed, np.arange(n))
    vals = splitmix64(keys)
    z = Zipf(n, theta)

    def batches():
        for b in range(n_batches):
            s = stream_seed(seed, 200 + b)
            ops = _mixed_ops(s, 0, q, 0.05, 0.05)
            ranks = z.ranks(uniform01(s, q, q))
            bkeys = keys[scramble(ranks, n, seed)]
            bvals = u64_stream(s, 2 * q, q)
            yield Batch(ops, bkeys, bvals)

    return Workload("skewed", keys, vals, 0.25, int(stream_seed(seed, 5)), batches, True)


def random_small(seed: int, n: int, q: int, key_range: int, p: float = 0.5,
                 invalid_frac: float = 0.02, n_batches: int = 1) -> Workload:
    """Tiny dense workload for exhaustive checks: keys drawn from [0, key_range) so that
    same-key runs, revivals and delete-then-insert chains are frequent. Includes a few
    invalid queries (bad op code or the reserved key 2^64-1)."""
    s = stream_seed(seed, 7)
    keys = bounded(s, 0, n, key_range).astype(np.uint64)
    vals = u64_stream(s, n, n)
    out = []
    for b in range(n_batches):
        sb = stream_seed(seed, 300 + b)
        ops = bounded(sb, 0, q, 3).astype(np.uint8)
        bkeys = bounded(sb, q, q, key_range).astype(np.uint64)
        bvals = u64_stream(sb, 2 * q, q)
        bad = uniform01(sb, 3 * q, q) < invalid_frac
        which = bounded(sb, 4 * q, q, 2)
        ops = np.where(bad & (which == 0), np.uint8(3 + (b % 250)), ops).astype(np.uint8)
        bkeys = np.where(bad & (which == 1), RESERVED_KEY, bkeys)
        out.append(Batch(ops, bkeys, bvals))
    return Workload("random_small", keys, vals, p, int(stream_seed(seed, 8)), out, True)


@dataclasses.dataclass
class MultiWorkload:
    name: str
    keys: list             # per index: initial keys (uint64)
    vals: list             # per index: initial values (uint64)
    promote_p: float
    hash_seeds: list       # per index
    batch_sizes: np.ndarray
    batches: object        # callable(round) -> list[Batch], one per index


def batching(seed: int = 4, count: int = 256, lo_log: float = 10, hi_log: float = 20,
             qlo_log: float = 8, qhi_log: float = 16) -> MultiWorkload:
    """Batching: `count` independent indices with sizes log-uniform in [2^lo, 2^hi]
    (distinct uniform keys in [0, 2^63), value = splitmix64(key), p = 1/4); each has its
    own batch, of a size log-uniform in [2^qlo, 2^qhi] fixed per index, with 80% search
    (half hits over the initial keys, half misses) and 20% insert of new uniform keys."""
    s = stream_seed(seed, 40)
    sizes = np.floor(2.0 ** (lo_log + uniform01(s, 0, count) * (hi_log - lo_log))).astype(np.int64)
    qs = np.floor(2.0 ** (qlo_log + uniform01(s, count, count) * (qhi_log - qlo_log))).astype(np.int64)
    keys = [distinct_keys(seed * 100003 + i, np.arange(int(n))) for i, n in enumerate(sizes)]
    vals = [splitmix64(k) for k in keys]
    seeds = [int(stream_seed(seed, 1000 + i)) for i in range(count)]

    def batches(r: int):
        out = []
        for i in range(count):
            q, n = int(qs[i]), int(sizes[i])
            sb = stream_seed(seed * 7 + i, 10_000 + r)
            u = uniform01(sb, 0, q)
            ops = np.where(u < 0.2, OP_INSERT, OP_SEARCH).astype(np.uint8)
            hit = keys[i][bounded(sb, q, q, n)]
            new = distinct_keys(seed * 100003 + i, np.uint64(1 << 40) + np.uint64(r) * np.uint64(1 << 20)
                                + np.arange(q, dtype=np.uint64))
            half = bounded(sb, 2 * q, q, 2) == 0
            bkeys = np.where(ops == OP_INSERT, new, np.where(half, hit, new[::-1]))
            out.append(Batch(ops, bkeys.astype(np.uint64), u64_stream(sb, 3 * q, q)))
        return out

    return MultiWorkload("batching", keys, vals, 0.25, seeds, qs, batches)


@dataclasses.dataclass
class ServeWorkload:
    name: str
    keys: np.ndarray
    vals: np.ndarray
    promote_p: float
    hash_seed: int
    ops: np.ndarray        # the request stream's queries, back to back
    qkeys: np.ndarray
    qvals: np.ndarray
    sizes: np.ndarray      # uint32 request sizes (queries)


def serving(seed: int = 5, n: int = 1 << 26, nreq: int = 40000, max_size: int = 4096,
            theta: float = 0.9) -> ServeWorkload:
    """Serving: a resident index of n distinct uniform keys (value = splitmix64(key),
    p = 1/4) and a stream of nreq requests of log-uniform sizes in [1, max_size], their
    queries 95% search / 5% insert (overwrites) with Zipf(theta) keys over the index
    (ranks scattered by a seeded bijection). Arrival times are the caller's."""
    keys = distinct_keys(seed, np.arange(n))
    vals = splitmix64(keys)
    s = stream_seed(seed, 50)
    sizes = np.maximum(1, np.floor(2.0 ** (uniform01(s, 0, nreq) * np.log2(max_size)))).astype(np.uint32)
    q = int(sizes.sum())
    z = Zipf(n, theta)
    qkeys = keys[scramble(z.ranks(uniform01(s, nreq, q)), n, seed)]
    ops = np.where(uniform01(s, nreq + q, q) < 0.05, OP_INSERT, OP_SEARCH).astype(np.uint8)
    qvals = u64_stream(s, nreq + 2 * q, q)
    return ServeWorkload("serving", keys, vals, 0.25, int(stream_seed(seed, 51)), ops, qkeys, qvals, sizes)
