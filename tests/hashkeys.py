"""Keys whose height hash takes a chosen value, for tests that must reach the height cap.

The height rule hashes h = splitmix64(key ^ splitmix64(seed)). SplitMix64 (Steele, Lea
and Flood 2014) is a bijection on 64-bit words: an add of the odd gamma, two steps of
"xor with a right shift, then multiply by an odd constant", and a final xorshift. Each
step is invertible, so the key for any wanted h is
    key = splitmix64^-1(h) ^ splitmix64(seed).
The inverse below undoes the steps in reverse order from the published definition:
a right xorshift by s is undone by repeating y ^ (x >> s) until it is stable (each round
fixes s more high bits), and a multiply by an odd constant by the multiplicative inverse
mod 2^64. Callers check splitmix64(inverse(h)) == h with the oracle's own (pinned)
splitmix64 before using a key.
"""
from __future__ import annotations

M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
MUL1 = 0xBF58476D1CE4E5B9
MUL2 = 0x94D049BB133111EB


def _unxorshift(y: int, s: int) -> int:
    x = y
    for _ in range(64 // s + 1):
        x = y ^ (x >> s)
    return x & M64


def splitmix64_inverse(h: int) -> int:
    z = _unxorshift(h & M64, 31)
    z = (z * pow(MUL2, -1, 1 << 64)) & M64
    z = _unxorshift(z, 27)
    z = (z * pow(MUL1, -1, 1 << 64)) & M64
    z = _unxorshift(z, 30)
    return (z - GAMMA) & M64


def key_with_hash(h: int, seed_mix: int) -> int:
    """The key whose height hash is h, given splitmix64(seed)."""
    return splitmix64_inverse(h) ^ seed_mix


def hash_with_trailing_zeros(tz: int, salt: int) -> int:
    """A 64-bit word with exactly tz trailing zero bits (0 for tz = 64); the bits above
    the lowest set one come from salt."""
    if tz >= 64:
        return 0
    hi = (salt * 2 + 1) & M64  # odd
    return (hi << tz) & M64
