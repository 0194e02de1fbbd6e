"""Pins for substitution and the entity map (oracle).

* The paper's worked example (§2 stage (3), ``tests/golden/paper_example.txt``):
  format only, since the key is not published.
* Reconstruction: putting each entity's original bytes back where its
  replacement stands restores the input exactly (only sensitive values are
  replaced, §2 stage (5)).
* Referential integrity: the same entity under the same key always gets the
  same pseudonym, across records and calls (Fig. 1 caption).
* No detected entity survives: re-running the recognizers on the output finds
  no mapped entity of the same type (Appendix D: leaking one occurrence of k
  is as bad as leaking all).
* The map: first/last sighting and counts equal a direct count over spans;
  merging shard maps equals the map of the whole run.
"""
import os
import re

import numpy as np
import pytest

import synth
from oracle import pipeline as P
from oracle import recognizers as R
from oracle.encoder import Encoder
from oracle.hmac_sha256 import hmac_sha256
from oracle.pseudonym import merge_maps, replacement

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_example.txt")


def _golden():
    vals = {}
    for line in open(GOLDEN, encoding="utf-8"):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.rstrip("\n").split("\t")
        vals[k] = v
    return vals


def test_paper_example_format():
    g = _golden()
    data = g["input"].encode()
    spans = R.recognize(data)
    assert spans == [(0, len(data), R.IP_ADDRESS)]
    assert synth.TYPE_NAMES_4[R.IP_ADDRESS - 1] == g["type"]
    L = int(g["slug_hex_len"])
    pattern = re.compile(r"\[" + g["type"] + r"_[0-9a-f]{%d}\]" % L)
    assert pattern.fullmatch(g["output"])
    for key in (b"k", b"another key", bytes(range(64))):
        rep, slug = replacement(g["type"], hmac_sha256(key, data), L)
        assert pattern.fullmatch(rep.decode())
        assert slug == hmac_sha256(key, data).hex()[:L]


@pytest.mark.parametrize("L", [0, 1, 7, 10, 64])
def test_slug_lengths(L):
    rep, slug = replacement("HOSTNAME", bytes(range(32)), L)
    assert len(slug) == L
    assert rep == (b"[HOSTNAME]" if L == 0 else b"[HOSTNAME_" + slug.encode() + b"]")


@pytest.fixture(scope="module")
def c1_run(c1_records, vocab_index):
    w = synth.make_weights(synth.C1.dims)
    enc = Encoder(synth.C1.dims, w)
    sch = P.Schema(synth.TYPE_NAMES_4)
    recs = c1_records.records()[:96]
    return recs, P.anonymize(recs, sch, synth.make_key(), enc, vocab_index), sch


def test_reconstruction_and_pass_through(c1_run):
    recs, res, sch = c1_run
    n_spans = 0
    for data, tr in zip(recs, res.traces):
        out = tr.output
        rebuilt = bytearray()
        pos_in, pos_out = 0, 0
        for s, n, t in tr.final:
            gap = s - pos_in
            assert out[pos_out:pos_out + gap] == data[pos_in:s]          # pass-through bytes unchanged
            rebuilt += out[pos_out:pos_out + gap]
            pos_out += gap
            rep, _ = replacement(sch.type_names[t - 1], hmac_sha256(synth.make_key(), data[s:s + n]), 10)
            assert out[pos_out:pos_out + len(rep)] == rep
            rebuilt += data[s:s + n]
            pos_out += len(rep)
            pos_in = s + n
            n_spans += 1
        rebuilt += out[pos_out:]
        assert bytes(rebuilt) == data
    assert n_spans > 500


def test_referential_integrity_and_map_counts(c1_run):
    recs, res, sch = c1_run
    seen = {}
    counts = {}
    first, last = {}, {}
    for ri, (data, tr) in enumerate(zip(recs, res.traces)):
        for s, n, t in tr.final:
            k = (t, data[s:s + n])
            rep = replacement(sch.type_names[t - 1], hmac_sha256(synth.make_key(), k[1]), 10)[0]
            assert seen.setdefault(k, rep) == rep
            counts[k] = counts.get(k, 0) + 1
            first.setdefault(k, ri)
            last[k] = ri
    assert [(e.type, e.original) for e in res.map] == sorted(counts)
    for e in res.map:
        k = (e.type, e.original)
        assert (e.count, e.first_seen, e.last_seen) == (counts[k], first[k], last[k])
        assert e.full_hash == hmac_sha256(synth.make_key(), e.original).hex()
        assert e.slug == e.full_hash[:10]


def test_no_detected_entity_survives(c1_run):
    recs, res, sch = c1_run
    mapped = {(e.type, e.original) for e in res.map}
    for tr in res.traces:
        for s, n, t in R.recognize(tr.output):
            assert (t, tr.output[s:s + n]) not in mapped


def test_overlap_rule_and_preserve(c1_run, vocab_index):
    recs, res, sch = c1_run
    for tr in res.traces:
        for s, n, t in tr.final:
            if (s, n, t) not in tr.regex:
                assert all(s + n <= rs or rs + rn <= s for rs, rn, _ in tr.regex)
        assert all(a[0] + a[1] <= b[0] for a, b in zip(tr.final, tr.final[1:]))
    # preserving HOSTNAME (bit 2) drops exactly the HOSTNAME spans
    w = synth.make_weights(synth.C1.dims)
    sch2 = P.Schema(synth.TYPE_NAMES_4, preserve_mask=1 << R.HOSTNAME)
    labels = [tr.labels for tr in res.traces[:20]]
    r2 = P.anonymize_from_labels(recs[:20], labels, sch2, synth.make_key(), vocab_index)
    for a, b in zip(res.traces[:20], r2.traces):
        assert b.final == [sp for sp in a.final if sp[2] != R.HOSTNAME]


def test_empty_and_entity_free_records(vocab_index):
    w = synth.make_weights(synth.C1.dims)
    enc = Encoder(synth.C1.dims, w)
    sch = P.Schema(synth.TYPE_NAMES_4)
    res = P.anonymize([b"", b"   ", b"no entities here"], sch, b"key", enc, vocab_index)
    assert res.outputs[0] == b""
    assert res.traces[1].output == b"   " or res.traces[1].final


def test_shard_maps_merge_to_whole(c1_run, vocab_index):
    recs, res, sch = c1_run
    labels = [tr.labels for tr in res.traces]
    key = synth.make_key()
    half = len(recs) // 2
    a = P.anonymize_from_labels(recs[:half], labels[:half], sch, key, vocab_index, record_base=0)
    b = P.anonymize_from_labels(recs[half:], labels[half:], sch, key, vocab_index, record_base=half)
    merged = merge_maps([a.map, b.map])
    assert [(e.type, e.original, e.full_hash, e.first_seen, e.last_seen, e.count) for e in merged] == \
           [(e.type, e.original, e.full_hash, e.first_seen, e.last_seen, e.count) for e in res.map]
