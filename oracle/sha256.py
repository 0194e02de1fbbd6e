"""SHA-256 written from FIPS 180-4 (oracle).

The round constants and initial hash value are derived here from their
definitions in FIPS 180-4 §4.2.2 and §5.3.3 (the first 32 bits of the
fractional parts of the cube roots of the first 64 primes, and of the square
roots of the first 8 primes), with exact integer arithmetic, instead of being
typed in.
"""
from __future__ import annotations

MASK = 0xFFFFFFFF


def _primes(n: int) -> list[int]:
    out = []
    k = 2
    while len(out) < n:
        if all(k % p for p in out if p * p <= k):
            out.append(k)
        k += 1
    return out


def _iroot(x: int, r: int) -> int:
    """floor(x ** (1/r)) for a non-negative integer x."""
    lo, hi = 0, 1
    while hi ** r <= x:
        hi *= 2
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if mid ** r <= x:
            lo = mid
        else:
            hi = mid
    return lo


def _frac_bits(p: int, r: int) -> int:
    """First 32 bits of the fractional part of p ** (1/r)."""
    return _iroot(p << (32 * r), r) & MASK


K = [_frac_bits(p, 3) for p in _primes(64)]
H0 = [_frac_bits(p, 2) for p in _primes(8)]


def _rotr(x: int, n: int) -> int:
    return ((x >> n) | (x << (32 - n))) & MASK


def compress(state: list[int], block: bytes) -> list[int]:
    """One application of the SHA-256 compression function (FIPS 180-4 §6.2.2)."""
    w = [int.from_bytes(block[4 * t:4 * t + 4], "big") for t in range(16)]
    for t in range(16, 64):
        s0 = _rotr(w[t - 15], 7) ^ _rotr(w[t - 15], 18) ^ (w[t - 15] >> 3)
        s1 = _rotr(w[t - 2], 17) ^ _rotr(w[t - 2], 19) ^ (w[t - 2] >> 10)
        w.append((w[t - 16] + s0 + w[t - 7] + s1) & MASK)
    a, b, c, d, e, f, g, h = state
    for t in range(64):
        S1 = _rotr(e, 6) ^ _rotr(e, 11) ^ _rotr(e, 25)
        ch = (e & f) ^ (~e & g)
        t1 = (h + S1 + ch + K[t] + w[t]) & MASK
        S0 = _rotr(a, 2) ^ _rotr(a, 13) ^ _rotr(a, 22)
        maj = (a & b) ^ (a & c) ^ (b & c)
        t2 = (S0 + maj) & MASK
        h, g, f, e, d, c, b, a = g, f, e, (d + t1) & MASK, c, b, a, (t1 + t2) & MASK
    return [(x + y) & MASK for x, y in zip(state, (a, b, c, d, e, f, g, h))]


def pad(message: bytes) -> bytes:
    """Message padding (FIPS 180-4 §5.1.1): 0x80, zeros, 64-bit big-endian bit length."""
    n = len(message)
    zeros = (55 - n) % 64
    return message + b"\x80" + b"\x00" * zeros + (8 * n).to_bytes(8, "big")


def sha256(message: bytes) -> bytes:
    padded = pad(message)
    state = list(H0)
    for i in range(0, len(padded), 64):
        state = compress(state, padded[i:i + 64])
    return b"".join(x.to_bytes(4, "big") for x in state)
