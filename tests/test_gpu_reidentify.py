"""Controlled re-identification on the GPU vs the oracle, through the C ABI.

The GPU's own anonymized output, re-identified with its map and key, gives
the input back (10-hex slugs); with 2-hex slugs, where many entities share a
slug, the output and the counts equal the oracle's. A map imported under
another key, or with an altered row, leaves the affected pseudonyms; text
that only looks like a pseudonym, cut by a record end, or naming no entry
stays unchanged. Host and device inputs give the same bytes.
"""
import numpy as np
import pytest

import synth
import paper_2606_15650_b300.api as api
from oracle import reidentify as RI
from oracle.hmac_sha256 import hmac_sha256

pytestmark = pytest.mark.gpu

DIMS = synth.C1.dims
NAMES = list(synth.TYPE_NAMES_4)
KEY = synth.make_key()


@pytest.fixture(scope="module")
def blob():
    return synth.pack_blob(DIMS, synth.make_weights(DIMS, seed=2002, random_affine=True))


def _oracle(out_recs, entries, slug_len, key):
    st = RI.ReidStats()
    back = RI.reidentify(out_recs, entries, NAMES, slug_len, key, st)
    return back, (st.pseudonyms, st.resolved, st.ambiguous, st.unverified)


def _counts(o):
    s = o.stats()
    return s["n_pseudonyms"], s["n_reidentified"], s["n_ambiguous"], s["n_unverified"]


@pytest.mark.parametrize("slug_len", [10, 2])
def test_round_trip_and_oracle(blob, vocab_words, c1_records, slug_len):
    ctx = api.Context(DIMS, blob, vocab_words, precision="bf16")
    schema = api.Schema(synth.TYPE_NAMES_4, slug_hex_len=slug_len)
    recs = c1_records.records()
    fwd = ctx.anonymize(c1_records.data, c1_records.offsets, schema, KEY)
    pseud = fwd.records()
    n_final = fwd.stats()["n_final_spans"]
    ps = synth.records_from_list(pseud)
    back = ctx.reidentify(ps.data, ps.offsets, schema, KEY)
    got = back.records()
    want, counts = _oracle(pseud, ctx.map_export(), slug_len, KEY)
    assert got == want
    assert _counts(back) == counts
    assert counts[0] == n_final
    if slug_len == 10:
        assert got == recs and counts[1] == n_final
    else:
        assert counts[2] > 0 and counts[1] > 0
    # device in, device out: same bytes
    import torch
    d = torch.from_numpy(ps.data).cuda()
    off = torch.from_numpy(ps.offsets.astype(np.int64)).cuda()
    dev = ctx.reidentify(d, off, schema, KEY)
    assert dev.copy_to_host() == got
    for o in (fwd, back, dev):
        o.free()
    ctx.close()


def test_wrong_key_and_altered_row(blob, vocab_words, c1_records):
    ctx = api.Context(DIMS, blob, vocab_words, precision="bf16")
    schema = api.Schema(synth.TYPE_NAMES_4)
    sub = synth.records_from_list(c1_records.records()[:64])
    pseud = ctx.anonymize(sub.data, sub.offsets, schema, KEY).records()
    entries = ctx.map_export()
    ps = synth.records_from_list(pseud)
    other = b"not the key"
    # the map imported under another key: nothing verifies
    ctx2 = api.Context(DIMS, blob, vocab_words, precision="bf16")
    ctx2.map_import(other, entries)
    o = ctx2.reidentify(ps.data, ps.offsets, schema, other)
    want, counts = _oracle(pseud, entries, 10, other)
    assert o.records() == want == pseud
    assert _counts(o) == counts and counts[3] == counts[0] > 0
    # one altered row: its pseudonyms stay, the rest resolve
    victim = max(entries, key=lambda e: e.count)
    bad = [api.Entity(e.type, e.original + b"!" if e is victim else e.original, e.full_hash, e.slug, e.first_seen,
                      e.last_seen, e.count) for e in entries]
    ctx3 = api.Context(DIMS, blob, vocab_words, precision="bf16")
    ctx3.map_import(KEY, bad)
    o3 = ctx3.reidentify(ps.data, ps.offsets, schema, KEY)
    want3, counts3 = _oracle(pseud, bad, 10, KEY)
    assert o3.records() == want3
    assert _counts(o3) == counts3 and counts3[3] == victim.count
    # a key that differs from the non-empty map's key is refused
    with pytest.raises(api.AnonShieldError, match="AS_ERR_STATE"):
        ctx.reidentify(ps.data, ps.offsets, schema, other)
    for c in (ctx, ctx2, ctx3):
        c.close()


def test_pseudonym_shaped_text(blob, vocab_words):
    ctx = api.Context(DIMS, blob, vocab_words, precision="bf16")
    schema = api.Schema(synth.TYPE_NAMES_4)
    orig = b"db01.corp.example"
    h = hmac_sha256(KEY, orig).hex()
    ctx.map_import(KEY, [api.Entity(2, orig, h, h[:10], 0, 0, 1)])
    slug = h[:10].encode()
    recs = [b"a [HOSTNAME_" + slug + b"] b",
            b"[HOSTNAME_" + slug.upper() + b"]",
            b"[HOSTNAMES_" + slug + b"] [CVE_ID_" + slug + b"]",
            b"[HOSTNAME_" + slug,                           # cut by the record end ...
            b"] [HOSTNAME_" + slug[:5],                     # ... and the next record holds the rest
            slug[5:] + b"]",
            b"[[HOSTNAME_" + slug + b"]][HOSTNAME_" + slug + b"]",
            b"",
            b"[HOSTNAME_" + slug + b"]"]
    rs = synth.records_from_list(recs)
    o = ctx.reidentify(rs.data, rs.offsets, schema, KEY)
    want, counts = _oracle(recs, ctx.map_export(), 10, KEY)
    assert o.records() == want
    assert _counts(o) == counts == (5, 4, 0, 0)
    ctx.close()


def test_rejected_arguments(blob, vocab_words):
    ctx = api.Context(DIMS, blob, vocab_words, precision="bf16")
    rs = synth.records_from_list([b"x"])
    with pytest.raises(api.AnonShieldError, match="slug_hex_len 0"):
        ctx.reidentify(rs.data, rs.offsets, api.Schema(synth.TYPE_NAMES_4, slug_hex_len=0), KEY)
    with pytest.raises(api.AnonShieldError, match="brackets"):
        ctx.reidentify(rs.data, rs.offsets, api.Schema(("IP", "HOST[", "CVE", "MAC")), KEY)
    empty = ctx.reidentify(np.zeros(0, np.uint8), np.zeros(1, np.uint64), api.Schema(synth.TYPE_NAMES_4), KEY)
    assert empty.records() == [] and _counts(empty) == (0, 0, 0, 0)
    ctx.close()
