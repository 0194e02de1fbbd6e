"""Pins for the oracle's re-identification.

Independent of its matching loop: anonymizing records with the oracle's own
(separately pinned) substitution and map and re-identifying them must give
the records back; the number of pseudonyms left ambiguous must equal the
number of replaced spans whose (type, slug) several distinct originals
share, counted from the forward spans; a wrong key or an altered row leaves
every affected pseudonym as it is; pseudonym-shaped text that names no
entry stays unchanged.
"""
from collections import defaultdict

import numpy as np
import pytest

import synth
from oracle import pipeline as P
from oracle import reidentify as RI
from oracle.hmac_sha256 import hmac_sha256

NAMES = list(synth.TYPE_NAMES_4)
KEY = synth.make_key()


def _labels(rng, n_tok: int) -> list[int]:
    """A seeded label stream with occasional B/I runs (stand-in for the encoder)."""
    out, t = [], 0
    while t < n_tok:
        if rng.random() < 0.03:
            ty = int(rng.integers(1, 5))
            run = int(rng.integers(1, 4))
            out += [2 * ty - 1] + [2 * ty] * (run - 1)
            t += run
        else:
            out.append(0)
            t += 1
    return out[:n_tok]


def _anonymized(records, vocab_index, slug_len):
    from oracle import tokenizer
    rng = np.random.default_rng(9)
    labels = [_labels(rng, len(tokenizer.tokenize(r, vocab_index)[0])) for r in records]
    schema = P.Schema(tuple(NAMES), slug_hex_len=slug_len)
    return P.anonymize_from_labels(records, labels, schema, KEY, vocab_index)


@pytest.fixture(scope="module")
def recs(c1_records):
    return c1_records.records()[:120]


def test_round_trip(recs, vocab_index):
    res = _anonymized(recs, vocab_index, 10)
    st = RI.ReidStats()
    back = RI.reidentify(res.outputs, res.map, NAMES, 10, KEY, st)
    assert back == recs
    n_final = sum(len(t.final) for t in res.traces)
    assert st.pseudonyms == st.resolved == n_final > 500
    assert st.ambiguous == st.unverified == 0


def test_short_slugs_leave_exactly_the_shared_ones(recs, vocab_index):
    """With L = 2 many entities of one type share a slug: those stay, all others resolve."""
    res = _anonymized(recs, vocab_index, 2)
    originals = defaultdict(set)
    for e in res.map:
        originals[(e.type, e.full_hash[:2])].add(e.original)
    shared = sum(1 for tr, data in zip(res.traces, recs) for s, n, t in tr.final
                 if len(originals[(t, hmac_sha256(KEY, data[s:s + n]).hex()[:2])]) > 1)
    st = RI.ReidStats()
    back = RI.reidentify(res.outputs, res.map, NAMES, 2, KEY, st)
    assert st.ambiguous == shared > 0
    assert st.resolved + st.ambiguous == st.pseudonyms == sum(len(t.final) for t in res.traces)
    # records without a shared slug come back whole
    whole = 0
    for tr, data, b in zip(res.traces, recs, back):
        if all(len(originals[(t, hmac_sha256(KEY, data[s:s + n]).hex()[:2])]) == 1 for s, n, t in tr.final):
            assert b == data
            whole += 1
    assert whole > 0


def test_wrong_key_and_altered_row(recs, vocab_index):
    res = _anonymized(recs[:40], vocab_index, 10)
    st = RI.ReidStats()
    assert RI.reidentify(res.outputs, res.map, NAMES, 10, KEY + b"x", st) == res.outputs
    assert st.unverified == st.pseudonyms > 0 and st.resolved == 0
    bad = list(res.map)
    victim = bad[0]
    bad[0] = type(victim)(victim.type, victim.original + b"!", victim.full_hash, victim.slug, victim.first_seen,
                          victim.last_seen, victim.count)
    st = RI.ReidStats()
    back = RI.reidentify(res.outputs, bad, NAMES, 10, KEY, st)
    assert st.unverified == victim.count and st.resolved == st.pseudonyms - victim.count
    assert victim.original + b"!" not in b"".join(back)


def test_pseudonym_shaped_text():
    from oracle.pseudonym import MapEntry
    h = hmac_sha256(KEY, b"db01.corp.example").hex()
    entries = [MapEntry(2, b"db01.corp.example", h, h[:10], 0, 0, 1)]
    slug = h[:10].encode()
    recs = [b"a [HOSTNAME_" + slug + b"] b",
            b"[HOSTNAME_" + slug.upper() + b"]",            # upper-case hex: not a pseudonym
            b"[HOSTNAMES_" + slug + b"] [CVE_ID_" + slug + b"]",  # unknown name; known name, no entry
            b"[HOSTNAME_" + slug,                            # cut by the record end
            b"[[HOSTNAME_" + slug + b"]]",
            b""]
    st = RI.ReidStats()
    out = RI.reidentify(recs, entries, NAMES, 10, KEY, st)
    assert out == [b"a db01.corp.example b", recs[1], recs[2], recs[3], b"[db01.corp.example]", b""]
    assert (st.pseudonyms, st.resolved, st.ambiguous, st.unverified) == (3, 2, 0, 0)


def test_rejected_schemas():
    with pytest.raises(ValueError):
        RI.reidentify([b""], [], NAMES, 0, KEY)
    with pytest.raises(ValueError):
        RI.reidentify([b""], [], ["A[B"], 10, KEY)
