"""Pins of the per-field oracle (oracle/fields.py), no GPU.

- One detected field covering a whole record reduces to the whole-record
  pipeline (itself pinned elsewhere).
- An excluded field and the bytes outside fields pass through unchanged, even
  when they hold entities the recognizers would find.
- A forced field becomes exactly "[TYPE_slug]" with slug = first hex digits of
  HMAC-SHA256(key, trimmed value), computed here with Python's hmac/hashlib.
- Detected fields are independent: the result equals the whole-record
  pipeline run on each field as a record of its own, spliced back.
"""
import hashlib
import hmac

import pytest

import synth
from oracle import fields as F
from oracle import pipeline as P
from oracle.encoder import Encoder

DIMS = synth.C1.dims
SCHEMA = P.Schema(synth.TYPE_NAMES_4)
KEY = b"field-policy-key"


@pytest.fixture(scope="module")
def enc():
    return Encoder(DIMS, synth.make_weights(DIMS, seed=31, random_affine=True))


def _slug(ent: bytes, n=10) -> bytes:
    return hmac.new(KEY, ent, hashlib.sha256).hexdigest()[:n].encode()


def test_single_detect_field_is_whole_record(enc, vocab_index, c1_records):
    recs = c1_records.records()[:6]
    whole = P.anonymize(recs, SCHEMA, KEY, enc, vocab_index)
    got = F.anonymize_fields(recs, [[(0, len(r), 3)] for r in recs], F.FieldPolicy(), SCHEMA, KEY, enc, vocab_index)
    assert got.outputs == whole.outputs
    assert [(e.type, e.original, e.first_seen, e.count) for e in got.map] == \
        [(e.type, e.original, e.first_seen, e.count) for e in whole.map]


def test_exclude_and_structure_pass_through(enc, vocab_index):
    parts = [b"10.0.0.1", b"host srv01.example.com CVE-2021-44228", b"aa:bb:cc:dd:ee:ff"]
    rec = b"|".join(parts)
    fields, pos = [], 0
    for i, p in enumerate(parts):
        fields.append((pos, len(p), i))
        pos += len(p) + 1
    pol = F.FieldPolicy({0: (F.EXCLUDE, 0), 1: (F.EXCLUDE, 0), 2: (F.EXCLUDE, 0)})
    got = F.anonymize_fields([rec], [fields], pol, SCHEMA, KEY, enc, vocab_index)
    assert got.outputs == [rec] and got.map == []
    # no fields at all: everything is structure
    got = F.anonymize_fields([rec], [[]], F.FieldPolicy(), SCHEMA, KEY, enc, vocab_index)
    assert got.outputs == [rec] and got.map == []


def test_forced_field_closed_form(enc, vocab_index):
    rec = b"ip=  10.9.8.7 \t;name=db-primary;note=  \n"
    a0, a1, a2 = rec.index(b"  10.9"), rec.index(b"db-"), rec.index(b"note=") + 5
    fields = [(a0, 12, 0), (a1, 10, 1), (a2, len(rec) - a2, 2)]   # the last value is only whitespace
    assert rec[a0:a0 + 12] == b"  10.9.8.7 \t" and rec[a1:a1 + 10] == b"db-primary" and rec[a2:] == b"  \n"
    pol = F.FieldPolicy({0: (F.FORCE, 1), 1: (F.FORCE, 2), 2: (F.FORCE, 3)})
    sch = P.Schema(synth.TYPE_NAMES_4, preserve_mask=(1 << 1) | (1 << 2))  # preserve ignored for forced fields
    got = F.anonymize_fields([rec], [fields], pol, sch, KEY, enc, vocab_index)
    want = (b"ip=  [IP_ADDRESS_" + _slug(b"10.9.8.7") + b"] \t;name=[HOSTNAME_" + _slug(b"db-primary") +
            b"];note=  \n")
    assert got.outputs == [want]
    assert sorted((e.type, e.original) for e in got.map) == [(1, b"10.9.8.7"), (2, b"db-primary")]


def test_detected_fields_independent(enc, vocab_index, c1_records):
    recs = c1_records.records()[10:14]
    lines = []
    for r in recs:
        parts = r.split(b"\n")
        lines.append(parts)
    # a record = its lines joined by b"||" (structure); line i is field i; even fields detected, odd excluded
    records, fields = [], []
    for parts in lines:
        rec, fl, pos = b"", [], 0
        for i, p in enumerate(parts):
            if i:
                rec += b"||"
                pos += 2
            fl.append((pos, len(p), i))
            rec += p
            pos += len(p)
        records.append(rec)
        fields.append(fl)
    pol = F.FieldPolicy(default=F.EXCLUDE)
    pol.actions = {i: (F.DETECT, 0) for i in range(0, 64, 2)}
    got = F.anonymize_fields(records, fields, pol, SCHEMA, KEY, enc, vocab_index)
    for r, parts in enumerate(lines):
        rebuilt = []
        for i, p in enumerate(parts):
            rebuilt.append(P.anonymize([p], SCHEMA, KEY, enc, vocab_index).outputs[0] if i % 2 == 0 else p)
        assert got.outputs[r] == b"||".join(rebuilt)


def test_fields_checked(enc, vocab_index):
    with pytest.raises(ValueError):
        F.anonymize_fields([b"abcdef"], [[(2, 3, 0), (4, 1, 1)]], F.FieldPolicy(), SCHEMA, KEY, enc, vocab_index)
    with pytest.raises(ValueError):
        F.anonymize_fields([b"abc"], [[(2, 5, 0)]], F.FieldPolicy(), SCHEMA, KEY, enc, vocab_index)
