"""Pins for oracle/spans.py: token spans to byte spans, the overlap rule and the
preserve list.

The paper leaves all three open (§2 stage (2) names pattern recognizers beside
the NER model; Appendix D shows the truncation artefacts of replacing
overlapping detections one after the other; §2 names the preserve list). The
readings are: a token span covers the bytes of its tokens with ASCII white
space (0x09..0x0D, 0x20) trimmed from both ends, empty spans dropped;
recognizer spans win over any NER span that shares a byte with one; preserved
types are dropped afterwards.

The oracle computes these with offset arithmetic and interval tests. The
formulation here works on byte masks instead: a byte belongs to a token span
when the token that holds it lies in [first, last]; trimming keeps the
covered bytes that are not white space and takes their hull; a NER span
survives when none of its bytes is set in the mask of recognizer bytes. Both
are compared over exhaustive small spaces:

* every string of 1..8 bytes over {a, ' ', '\\t', '.'} with every byte its
  own token, i.e. every byte range [s, e);
* every string of 1..5 bytes over the same alphabet under every partition
  into tokens, with every token span [first, last];
* every set of disjoint recognizer spans over 9 bytes against every single
  NER span (4,181 sets x 45 spans), and random sets of several NER spans of
  three types against recognizer spans of two;
* every preserve mask over three types (and random ones in the random sets).

Mutants of the oracle (a one-sided trim, an end one byte short, a keep rule
that drops touching spans, a merge that drops every NER span, a preserve
filter applied before the overlap rule) must each fail the same check, so the
check has teeth.
"""
from __future__ import annotations

import itertools
import random

import pytest

from oracle import spans as S

ALPHABET = b"a \t."
WS = frozenset(b"\t\n\x0b\x0c\r ")


# ---------------------------------------------------------------- independent formulation

def mask_token_span_to_bytes(data: bytes, token_of_byte: list[int], first: int, last: int):
    covered = [b for b in range(len(data)) if first <= token_of_byte[b] <= last]
    solid = [b for b in covered if data[b] not in WS]
    if not solid:
        return None
    return min(solid), max(solid) + 1


def mask_merge(regex, ner, preserve_mask, n_bytes):
    taken = [False] * n_bytes
    for s, n, _ in regex:
        for b in range(s, s + n):
            taken[b] = True
    kept = [(s, n, t) for s, n, t in ner if not any(taken[b] for b in range(s, s + n))]
    out = sorted(regex + kept)
    return [sp for sp in out if not (preserve_mask >> sp[2]) & 1]


# ---------------------------------------------------------------- enumerations

def partitions(n: int):
    """Every split of n bytes into consecutive tokens, as (offs, lens)."""
    for cuts in itertools.product((0, 1), repeat=n - 1):
        offs = [0] + [i + 1 for i, c in enumerate(cuts) if c]
        ends = offs[1:] + [n]
        yield offs, [e - o for o, e in zip(offs, ends)]


def disjoint_span_sets(n: int, types=(1,)):
    """Every set of disjoint (start, length, type) spans over n bytes."""
    def rec(pos):
        if pos >= n:
            yield []
            return
        yield from rec(pos + 1)               # byte pos uncovered
        for e in range(pos + 1, n + 1):       # a span [pos, e)
            for t in types:
                for rest in rec(e):
                    yield [(pos, e - pos, t)] + rest
    yield from rec(0)


# ---------------------------------------------------------------- checks (return the first mismatch)

def _call(fn, *args):
    try:
        return fn(*args)
    except Exception as e:        # a mutant may index past the record: that is a failure too
        return ("raised", type(e).__name__)


def check_trim(fn) -> tuple | None:
    for n in range(1, 9):
        for tup in itertools.product(ALPHABET, repeat=n):
            data = bytes(tup)
            tob = list(range(n))
            offs, lens = list(range(n)), [1] * n
            for first in range(n):
                for last in range(first, n):
                    got = _call(fn, data, offs, lens, first, last)
                    want = mask_token_span_to_bytes(data, tob, first, last)
                    if got != want:
                        return data, offs, lens, first, last, got, want
    for n in range(1, 6):
        for tup in itertools.product(ALPHABET, repeat=n):
            data = bytes(tup)
            for offs, lens in partitions(n):
                tob = [i for i, ln in enumerate(lens) for _ in range(ln)]
                for first in range(len(offs)):
                    for last in range(first, len(offs)):
                        got = _call(fn, data, offs, lens, first, last)
                        want = mask_token_span_to_bytes(data, tob, first, last)
                        if got != want:
                            return data, offs, lens, first, last, got, want
    return None


def check_keep(fn, n: int = 9) -> tuple | None:
    singles = [(s, e - s, 3) for s in range(n) for e in range(s + 1, n + 1)]
    for regex in disjoint_span_sets(n):
        for sp in singles:
            got = fn(regex, [sp], 0)
            want = mask_merge(regex, [sp], 0, n)
            if got != want:
                return regex, [sp], got, want
    return None


def check_multi(fn, n: int = 12, trials: int = 4000) -> tuple | None:
    rng = random.Random(1234)
    for _ in range(trials):
        regex = _random_disjoint(rng, n, (1, 2))
        ner = _random_disjoint(rng, n, (1, 2, 3))
        mask = rng.randrange(16)
        got = fn(regex, ner, mask)
        want = mask_merge(regex, ner, mask, n)
        if got != want:
            return regex, ner, mask, got, want
    return None


def _random_disjoint(rng, n, types):
    out, pos = [], 0
    while pos < n:
        if rng.random() < 0.45:
            e = rng.randint(pos + 1, min(n, pos + 4))
            out.append((pos, e - pos, rng.choice(types)))
            pos = e
        else:
            pos += 1
    return out


# ---------------------------------------------------------------- the oracle passes

def test_trim_matches_mask_formulation():
    assert check_trim(S.token_span_to_bytes) is None


def test_ner_byte_spans_maps_and_drops():
    # every token span of every partition of every string over the alphabet up to 5 bytes,
    # handed over in one list per partition: same spans, same order, empty ones dropped
    for n in range(1, 6):
        for tup in itertools.product(ALPHABET, repeat=n):
            data = bytes(tup)
            for offs, lens in partitions(n):
                tob = [i for i, ln in enumerate(lens) for _ in range(ln)]
                k = len(offs)
                tspans = [(f, l, 1 + (f + l) % 4) for f in range(k) for l in range(f, k)]
                got = S.ner_byte_spans(data, offs, lens, tspans)
                want = []
                for f, l, t in tspans:
                    r = mask_token_span_to_bytes(data, tob, f, l)
                    if r is not None:
                        want.append((r[0], r[1] - r[0], t))
                assert got == want


def test_keep_rule_matches_mask_formulation():
    assert check_keep(S.merge) is None


def test_merge_many_spans_and_preserve():
    assert check_multi(S.merge) is None


def test_merge_both_directions():
    """Nothing that shares a byte with a recognizer span survives, and every NER span that
    shares none does, on every recognizer set over 9 bytes against every single NER span."""
    n = 9
    singles = [(s, e - s, 3) for s in range(n) for e in range(s + 1, n + 1)]
    for regex in disjoint_span_sets(n):
        taken = set(b for s, ln, _ in regex for b in range(s, s + ln))
        for sp in singles:
            out = S.merge(regex, [sp], 0)
            hits = any(b in taken for b in range(sp[0], sp[0] + sp[1]))
            assert (sp in out) == (not hits)
            assert all(r in out for r in regex)
            assert all(a[0] + a[1] <= b[0] for a, b in zip(out, out[1:]))


def test_preserve_every_mask():
    regex = [(0, 2, 1), (4, 1, 2)]
    ner = [(2, 2, 3), (5, 3, 1), (9, 1, 2), (3, 2, 1)]   # (3, 2) overlaps (4, 1): dropped
    for mask in range(16):
        got = S.merge(regex, ner, mask)
        want = mask_merge(regex, ner, mask, 10)
        assert got == want
        assert all(not (mask >> t) & 1 for _, _, t in got)
    # a preserved recognizer span still blocks the NER span under it
    assert S.merge([(0, 4, 2)], [(1, 2, 1)], preserve_mask=1 << 2) == []


def test_whitespace_set_is_the_ascii_one():
    for b in range(256):
        data = bytes([b]) + b"x" + bytes([b])
        got = S.token_span_to_bytes(data, [0, 1, 2], [1, 1, 1], 0, 2)
        want = (1, 2) if b in WS else (0, 3)
        assert got == want, b


# ---------------------------------------------------------------- mutants must fail

def _trim_left_only(data, offs, lens, first, last):
    s, e = offs[first], offs[last] + lens[last]
    while s < e and data[s] in WS:
        s += 1
    return (s, e) if e > s else None


def _end_one_short(data, offs, lens, first, last):
    s, e = offs[first], offs[last] + lens[last] - 1
    while s < e and data[s] in WS:
        s += 1
    while e > s and data[e - 1] in WS:
        e -= 1
    return (s, e) if e > s else None


def _len_of_first(data, offs, lens, first, last):
    s, e = offs[first], offs[last] + lens[first]
    while s < e and data[s] in WS:
        s += 1
    while e > s and data[e - 1] in WS:
        e -= 1
    return (s, e) if e > s else None


def _spaces_only(data, offs, lens, first, last):
    s, e = offs[first], offs[last] + lens[last]
    while s < e and data[s] == 0x20:
        s += 1
    while e > s and data[e - 1] == 0x20:
        e -= 1
    return (s, e) if e > s else None


def _keeps_empty(data, offs, lens, first, last):
    s, e = offs[first], offs[last] + lens[last]
    while s < e and data[s] in WS:
        s += 1
    while e > s and data[e - 1] in WS:
        e -= 1
    return s, e


@pytest.mark.parametrize("mutant", [_trim_left_only, _end_one_short, _len_of_first, _spaces_only, _keeps_empty])
def test_trim_mutants_fail(mutant):
    assert check_trim(mutant) is not None


def _drops_touching(regex, ner, mask):
    kept = [(s, n, t) for s, n, t in ner if not any(s <= rs + rn and rs <= s + n for rs, rn, _ in regex)]
    return [sp for sp in sorted(regex + kept) if not (mask >> sp[2]) & 1]


def _drops_all_ner(regex, ner, mask):
    return [sp for sp in sorted(regex) if not (mask >> sp[2]) & 1]


def _start_inside_only(regex, ner, mask):
    kept = [(s, n, t) for s, n, t in ner if not any(rs <= s < rs + rn for rs, rn, _ in regex)]
    return [sp for sp in sorted(regex + kept) if not (mask >> sp[2]) & 1]


def _preserve_first(regex, ner, mask):
    regex = [sp for sp in regex if not (mask >> sp[2]) & 1]
    ner = [sp for sp in ner if not (mask >> sp[2]) & 1]
    kept = [(s, n, t) for s, n, t in ner if not any(s < rs + rn and rs < s + n for rs, rn, _ in regex)]
    return sorted(regex + kept)


@pytest.mark.parametrize("mutant", [_drops_touching, _drops_all_ner, _start_inside_only])
def test_keep_mutants_fail(mutant):
    assert check_keep(mutant) is not None


def test_preserve_order_mutant_fails():
    assert check_multi(_preserve_first) is not None
