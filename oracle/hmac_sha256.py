"""HMAC-SHA256 written from RFC 2104 on the oracle's own SHA-256 (oracle).

The paper replaces each entity with an HMAC-SHA256 slug computed under an
operator-defined secret key (§2 stage (3)). RFC 2104 with B = 64: a key
longer than 64 bytes is first hashed; the key is zero-padded to 64 bytes;
HMAC = H((K xor opad) || H((K xor ipad) || message)), ipad = 0x36 repeated,
opad = 0x5c repeated.
"""
from __future__ import annotations

from .sha256 import sha256

BLOCK = 64


def hmac_sha256(key: bytes, message: bytes) -> bytes:
    if len(key) > BLOCK:
        key = sha256(key)
    key = key + b"\x00" * (BLOCK - len(key))
    ikey = bytes(k ^ 0x36 for k in key)
    okey = bytes(k ^ 0x5C for k in key)
    return sha256(okey + sha256(ikey + message))
