"""Byte tokenizer (oracle).

The paper runs a transformer NER model over record text (§2 stage (2)) and
says nothing about its tokenizer; this project's reading is a byte-level
subword tokenizer:

* Pre-tokens are maximal runs of ASCII letters and digits ``[0-9A-Za-z]``;
  every other byte (punctuation, whitespace, any byte >= 0x80) is a token by
  itself.
* Inside a run, repeatedly take the longest vocabulary string (2..12 bytes)
  that is a prefix of what is left of the run; if none is, take one byte.
* Ids: 0 is padding, byte b is id b + 1, vocabulary string k is id 257 + k.

Because runs end at every non-alphanumeric byte, each pattern-recognizer
entity boundary is also a token boundary.
"""
from __future__ import annotations

MAX_PIECE = 12
FIRST_WORD_ID = 257


def is_alnum(b: int) -> bool:
    return 0x30 <= b <= 0x39 or 0x41 <= b <= 0x5A or 0x61 <= b <= 0x7A


def build_vocab_index(words: list[bytes]) -> dict[bytes, int]:
    """Map each vocabulary string to its id (257 + position)."""
    return {w: FIRST_WORD_ID + i for i, w in enumerate(words)}


def tokenize(data: bytes, vocab: dict[bytes, int]) -> tuple[list[int], list[int], list[int]]:
    """Return (ids, byte offsets, byte lengths) of the tokens of one record."""
    ids: list[int] = []
    offs: list[int] = []
    lens: list[int] = []
    n = len(data)
    i = 0
    while i < n:
        b = data[i]
        if not is_alnum(b):
            ids.append(b + 1)
            offs.append(i)
            lens.append(1)
            i += 1
            continue
        end = i
        while end < n and is_alnum(data[end]):
            end += 1
        pos = i
        while pos < end:
            take = 0
            tid = 0
            for L in range(min(MAX_PIECE, end - pos), 1, -1):
                t = vocab.get(data[pos:pos + L])
                if t is not None:
                    take, tid = L, t
                    break
            if take == 0:
                take, tid = 1, data[pos] + 1
            ids.append(tid)
            offs.append(pos)
            lens.append(take)
            pos += take
        i = end
    return ids, offs, lens
