"""Pins for the oracle's SHA-256 (FIPS 180-4) and HMAC (RFC 2104).

The oracle computes both from scratch; these tests compare it with
independent implementations: Python's ``hashlib`` / ``hmac`` and the
``openssl`` command-line tool. Message lengths cross the 55/56/64-byte
padding edges; key lengths cover empty, short, exactly one block, and longer
than a block (which RFC 2104 hashes first).
"""
import hashlib
import hmac
import math
import shutil
import subprocess

import numpy as np
import pytest

from oracle import sha256 as S
from oracle.hmac_sha256 import hmac_sha256


def test_constants_match_their_definition_in_floating_point():
    # FIPS 180-4 §4.2.2 / §5.3.3 define the constants as fractional parts of
    # cube / square roots of primes; double precision agrees to ~20 bits.
    primes = [p for p in range(2, 400) if all(p % q for q in range(2, int(p ** 0.5) + 1))]
    for k, p in zip(S.K, primes[:64]):
        approx = (p ** (1.0 / 3.0)) % 1.0 * 2 ** 32
        assert abs(k - approx) < 2 ** 12
    for h, p in zip(S.H0, primes[:8]):
        approx = math.sqrt(p) % 1.0 * 2 ** 32
        assert abs(h - approx) < 2 ** 12
    assert len(set(S.K)) == 64


@pytest.mark.parametrize("n", list(range(0, 140)) + [191, 192, 255, 256, 300, 1000])
def test_sha256_matches_hashlib(n):
    rng = np.random.default_rng(n)
    msg = rng.integers(0, 256, size=n, dtype=np.uint8).tobytes()
    assert S.sha256(msg) == hashlib.sha256(msg).digest()


def test_padding_lengths():
    for n in range(0, 200):
        p = S.pad(b"x" * n)
        assert len(p) % 64 == 0
        assert len(p) - n >= 9 and len(p) - n <= 72


@pytest.mark.parametrize("klen", [0, 1, 31, 32, 63, 64, 65, 131])
def test_hmac_matches_stdlib(klen):
    rng = np.random.default_rng(1000 + klen)
    key = rng.integers(0, 256, size=klen, dtype=np.uint8).tobytes()
    for mlen in list(range(0, 70)) + [119, 120, 183, 184, 253, 300]:
        msg = rng.integers(0, 256, size=mlen, dtype=np.uint8).tobytes()
        assert hmac_sha256(key, msg) == hmac.new(key, msg, hashlib.sha256).digest()


@pytest.mark.skipif(shutil.which("openssl") is None, reason="openssl CLI not installed")
@pytest.mark.parametrize("klen,msg", [(1, b"100.111.20.23"), (64, b"CVE-2024-12345"), (70, b"")])
def test_hmac_matches_openssl_cli(klen, msg):
    key = bytes((7 * i + 3) % 256 for i in range(klen))
    r = subprocess.run(["openssl", "dgst", "-sha256", "-mac", "HMAC", "-macopt", f"hexkey:{key.hex()}"],
                       input=msg, capture_output=True, check=True)
    assert r.stdout.decode().strip().split()[-1] == hmac_sha256(key, msg).hex()


def test_wrong_constant_is_detected():
    """A planted mistake in one round constant changes the digest (the pins bite)."""
    saved = S.K[17]
    try:
        S.K[17] ^= 1
        assert S.sha256(b"abc") != hashlib.sha256(b"abc").digest()
    finally:
        S.K[17] = saved
    assert S.sha256(b"abc") == hashlib.sha256(b"abc").digest()
