"""Seeded synthetic subword vocabulary.

Id layout: 0 is padding; ids 1..256 stand for the single bytes 0x00..0xFF
(id = byte + 1); ids 257..size-1 are distinct alphanumeric strings of 2..12
bytes. The strings are data: the lexicon words in three casings, short
fragments of them, a few digit-bearing technical tokens, and seeded
pseudo-words to fill the table. Nothing here tokenizes anything.
"""
from __future__ import annotations

import numpy as np

from . import lexicon as lx

N_BYTE_IDS = 256
FIRST_WORD_ID = 257
MAX_PIECE = 12
MIN_PIECE = 2

_TECH = (
    "v1 v2 v3 x86 x64 tls10 tls11 tls12 tls13 ssl2 ssl3 sha1 sha256 sha512 md5 "
    "http2 ipv4 ipv6 aes128 aes256 rc4 des3 utf8 base64 win32 win64 amd64 arm64 "
    "i386 el7 el8 ubuntu1604 debian9 centos7 php7 php8 python3 java8 java11 "
    "node16 log4j smb1 smb2 smb3 snmpv1 snmpv2 ntlmv1 ntlmv2 rsa2048 rsa1024 ec256"
).split()

_CONS = "bcdfghjklmnprstvwz"
_VOWELS = "aeiou"


def _casings(w: str):
    yield w
    yield w[:1].upper() + w[1:]
    yield w.upper()


def make_vocab(size: int = 8192, seed: int = 2002) -> list[bytes]:
    """Return the strings for ids FIRST_WORD_ID..size-1 (size - 257 entries)."""
    n_words = size - FIRST_WORD_ID
    if n_words <= 0:
        raise ValueError("vocab size must exceed 257")
    rng = np.random.default_rng(seed)
    words: set[str] = set()
    base = (list(lx.SERVICES) + list(lx.NOUNS) + list(lx.VERBS) + list(lx.ADJECTIVES)
            + list(lx.FUNCTION_WORDS) + list(lx.SEVERITIES) + list(lx.PROTOCOLS)
            + list(lx.TLDS) + list(lx.HOST_WORDS) + list(lx.ORG_WORDS) + list(lx.FIELD_LABELS))
    for w in base:
        for c in _casings(w):
            if MIN_PIECE <= len(c) <= MAX_PIECE and c.isalnum() and c.isascii():
                words.add(c)
    for w in _TECH:
        words.add(w)
    # fragments: word prefixes and suffixes of 2..5 letters, so that unknown
    # words (host labels, pseudo names) split into several pieces
    for w in base:
        lw = w.lower()
        for k in range(2, 6):
            if len(lw) > k:
                words.add(lw[:k])
                words.add(lw[-k:])
    words = {w for w in words if MIN_PIECE <= len(w) <= MAX_PIECE and w.isascii() and w.isalnum()}
    chosen = sorted(words)
    if len(chosen) > n_words:
        keep = rng.permutation(len(chosen))[:n_words]
        chosen = sorted(chosen[i] for i in keep)
    # fill with seeded pseudo-words (consonant/vowel syllables)
    while len(chosen) < n_words:
        n_syl = int(rng.integers(1, 5))
        s = "".join(_CONS[int(rng.integers(len(_CONS)))] + _VOWELS[int(rng.integers(len(_VOWELS)))]
                    for _ in range(n_syl))
        if int(rng.integers(4)) == 0:
            s += _CONS[int(rng.integers(len(_CONS)))]
        if int(rng.integers(6)) == 0:
            s = s[:1].upper() + s[1:]
        if MIN_PIECE <= len(s) <= MAX_PIECE and s not in words:
            words.add(s)
            chosen.append(s)
    order = rng.permutation(len(chosen))
    return [chosen[i].encode("ascii") for i in order]


def vocab_arrays(pieces: list[bytes]) -> tuple[np.ndarray, np.ndarray]:
    """Pack the word strings into (bytes uint8[...], offsets uint32[n+1])."""
    offs = np.zeros(len(pieces) + 1, dtype=np.uint32)
    offs[1:] = np.cumsum([len(p) for p in pieces], dtype=np.uint64).astype(np.uint32)
    data = np.frombuffer(b"".join(pieces), dtype=np.uint8).copy()
    return data, offs
