"""Pins for the oracle tokenizer: brute force and invariants.

The independent formulation uses Python's ``re``: pre-tokens from one
alternation (alphanumeric run | any other byte), and inside a run an ordered
alternation of the vocabulary sorted longest-first, which ``re`` tries in
order, so it returns the longest vocabulary prefix.
"""
import itertools
import re

import pytest

from oracle.tokenizer import FIRST_WORD_ID, build_vocab_index, tokenize

TINY_VOCAB = [b"ab", b"ba", b"aab", b"a1", b"1b", b"abab", b"b1a", b"11", b"bab1ab"]


def re_tokenize(data: bytes, vocab_words: list[bytes]):
    idx = {w: FIRST_WORD_ID + i for i, w in enumerate(vocab_words)}
    alts = sorted(vocab_words, key=len, reverse=True)
    piece = re.compile(b"|".join(re.escape(w) for w in alts) + b"|.", re.S) if alts else re.compile(b".", re.S)
    out = []
    for m in re.finditer(rb"[0-9A-Za-z]+|[^0-9A-Za-z]", data):
        run = m.group(0)
        if not re.fullmatch(rb"[0-9A-Za-z]+", run):
            out.append((run[0] + 1, m.start(), 1))
            continue
        p = 0
        while p < len(run):
            mm = piece.match(run, p)
            tok = mm.group(0)
            tid = idx.get(tok, tok[0] + 1) if len(tok) > 1 else tok[0] + 1
            out.append((tid, m.start() + p, len(tok)))
            p += len(tok)
    return out


def test_brute_force_all_short_strings():
    alphabet = [b"a", b"b", b"1", b".", b" ", b"\xc3"]
    vi = build_vocab_index(TINY_VOCAB)
    n_checked = 0
    for n in range(0, 7):
        for combo in itertools.product(alphabet, repeat=n):
            s = b"".join(combo)
            ids, offs, lens = tokenize(s, vi)
            assert list(zip(ids, offs, lens)) == re_tokenize(s, TINY_VOCAB), s
            n_checked += 1
    assert n_checked == sum(6 ** n for n in range(7))


def _check_invariants(data: bytes, vi: dict, max_piece=12):
    ids, offs, lens = tokenize(data, vi)
    # concatenation of token bytes is the input
    assert b"".join(data[o:o + n] for o, n in zip(offs, lens)) == data
    assert all(offs[i] + lens[i] == offs[i + 1] for i in range(len(offs) - 1))
    inv = {v: k for k, v in vi.items()}
    for tid, o, n in zip(ids, offs, lens):
        if n > 1:
            assert inv[tid] == data[o:o + n]            # multi-byte tokens are vocabulary strings
        else:
            assert tid == data[o] + 1
        # greedy: no longer vocabulary prefix inside the same alphanumeric run
        end = o + n
        while end < len(data) and data[end:end + 1].isalnum() and data[end] < 128 and end - o < max_piece:
            end += 1
            assert data[o:end] not in vi
    return ids


def test_invariants_on_synthetic_records(c1_records, vocab_index):
    total = 0
    for i in range(0, c1_records.n, 4):
        total += len(_check_invariants(c1_records.record(i), vocab_index))
    assert total > 10000


def test_ids_in_range(c1_records, vocab_index):
    ids, _, _ = tokenize(c1_records.record(0), vocab_index)
    assert all(1 <= t < 8192 for t in ids)


@pytest.mark.parametrize("s", [b"", b" ", b"\xff\x00", b"Host: 10.0.0.1", b"A" * 40, b"x" * 13])
def test_edge_strings(s, vocab_index):
    _check_invariants(s, vocab_index)
