"""Dataset-scale parity: 70,951 records, 12-layer d=768 encoder, BF16, packed.

This is the launch configuration the benchmark times. The oracle is too
slow for the whole batch, so it checks seeded samples record by record
(tokens, recognizer spans, output bytes from the GPU's labels; FP64 logits
on sampled records), and properties that hold at any size are checked on the
whole batch: tokens tile every record's bytes; every byte outside the
final spans is copied to its shifted position; every span is replaced by
"[TYPE_slug]" at its shifted position with the HMAC slug; record offsets
follow; the map holds one entry per distinct (type, bytes) with its counts.
"""
import hashlib
import hmac

import numpy as np
import pytest

import synth
import paper_2606_15650_b300.api as api
from oracle import pipeline as P
from oracle.encoder import Encoder
from oracle.tokenizer import tokenize

import parity_util as U

pytestmark = pytest.mark.gpu

DIMS = synth.C2.dims
SCHEMA = api.Schema(synth.TYPE_NAMES_4)


@pytest.fixture(scope="module")
def c2(vocab_words):
    recs = synth.make_records(synth.C2.records, vocab_words)
    w = synth.make_weights(DIMS)
    key = synth.make_key()
    ctx = api.Context(DIMS, synth.pack_blob(DIMS, w), vocab_words, precision="bf16", keep_trace=True)
    out = ctx.anonymize(recs.data, recs.offsets, SCHEMA, key)
    data, offs = out.arrays()
    return recs, w, key, ctx, out, ctx.trace(), data, offs


def test_sampled_records_exact(c2, vocab_index):
    recs, w, key, ctx, out, tr, odata, ooffs = c2
    rng = np.random.default_rng(123)
    idx = sorted(rng.choice(recs.n, size=300, replace=False).tolist())
    sub = [recs.record(i) for i in idx]
    ref = P.anonymize_from_labels(sub, [U.gpu_labels_per_record(tr, recs.n)[i] for i in idx],
                                  U.oracle_schema(SCHEMA), key, vocab_index)
    # tokens and recognizer spans: bit-exact
    tok_traces = {i: t for i, t in zip(idx, ref.traces)}
    U.check_tokens(tr, None, recs.offsets, tok_traces, idx=idx)
    U.check_regex(tr, recs.offsets, tok_traces, idx=idx)
    for j, i in enumerate(idx):
        got = odata[int(ooffs[i]):int(ooffs[i + 1])].tobytes()
        assert got == ref.outputs[j], f"record {i}"


def test_sampled_logits_fp64(c2, vocab_index):
    """FP64 logits of sampled records of the whole-dataset batch (the benchmark's launch
    configuration), from the oracle's own tokens; 64 more records are compared in
    test_gpu_precision.py."""
    recs, w, key, ctx, out, tr, _, _ = c2
    rng = np.random.default_rng(7)
    idx = sorted(rng.choice(recs.n, size=12, replace=False).tolist())
    enc = Encoder(DIMS, w)
    traces = {}
    for i in idx:
        ids = tokenize(recs.record(i), vocab_index)[0]

        class T:  # minimal trace with the oracle's logits and labels
            pass
        t = T()
        t.logits = enc.logits(ids)
        traces[i] = t
    err, agree, flips = U.check_logits(tr, traces, "bf16", idx=idx)
    print(f"c2 sampled: max|dlogit| {err:.3e}, agreement {agree:.5f}, flips {flips}")


def test_whole_batch_tokens_tile_bytes(c2):
    recs, _, _, _, _, tr, _, _ = c2
    off, ln, rt = tr["tok_off"].astype(np.int64), tr["tok_len"].astype(np.int64), tr["rec_tok"].astype(np.int64)
    N = int(recs.offsets[-1])
    assert off[0] == 0 and np.all(off[1:] == off[:-1] + ln[:-1]) and off[-1] + ln[-1] == N
    nonempty = rt[1:] > rt[:-1]
    assert np.array_equal(off[rt[:-1][nonempty]], recs.offsets[:-1].astype(np.int64)[nonempty])
    assert np.all(ln >= 1) and np.all(ln <= 12)
    assert int((rt[1:] - rt[:-1]).max()) <= 512


def test_whole_batch_substitution(c2):
    recs, _, key, ctx, out, tr, odata, ooffs = c2
    data = recs.data
    N = len(data)
    s, l, t = (tr["final_start"].astype(np.int64), tr["final_len"].astype(np.int64),
               tr["final_type"].astype(np.int64))
    assert np.all(s[1:] >= s[:-1] + l[:-1]), "final spans sorted and disjoint"
    names = [b""] + [n.encode() for n in synth.TYPE_NAMES_4]
    name_len = np.array([len(n) for n in names])
    rep = 2 + name_len[t] + 1 + SCHEMA.slug_hex_len
    delta = rep - l
    excl = np.concatenate([[0], np.cumsum(delta)])
    assert len(odata) == N + excl[-1]
    cover = np.zeros(N + 1, np.int64)
    np.add.at(cover, s, 1)
    np.add.at(cover, s + l, -1)
    in_span = np.cumsum(cover)[:N] > 0
    b = np.nonzero(~in_span)[0]
    j = np.searchsorted(s, b, side="right")
    assert np.array_equal(odata[b + excl[j]], data[b]), "pass-through bytes"
    p = s + excl[:-1]
    assert np.all(odata[p] == ord("[")) and np.all(odata[p + rep - 1] == ord("]"))
    rng = np.random.default_rng(5)
    for k in rng.choice(len(s), size=min(2000, len(s)), replace=False):
        ent = data[s[k]:s[k] + l[k]].tobytes()
        slug = hmac.new(key, ent, hashlib.sha256).hexdigest()[:SCHEMA.slug_hex_len].encode()
        assert odata[p[k]:p[k] + rep[k]].tobytes() == b"[" + names[t[k]] + b"_" + slug + b"]"
    jr = np.searchsorted(s, recs.offsets.astype(np.int64), side="left")
    assert np.array_equal(ooffs.astype(np.int64), recs.offsets.astype(np.int64) + excl[jr])


def test_whole_batch_map(c2):
    recs, _, key, ctx, out, tr, _, _ = c2
    data = recs.data
    s, l, t = tr["final_start"], tr["final_len"], tr["final_type"]
    rec = np.searchsorted(recs.offsets.astype(np.int64), s.astype(np.int64), side="right") - 1
    agg = {}
    for a, b, c, r in zip(s.tolist(), l.tolist(), t.tolist(), rec.tolist()):
        k = (c, data[a:a + b].tobytes())
        e = agg.get(k)
        agg[k] = (r, r, 1) if e is None else (min(e[0], r), max(e[1], r), e[2] + 1)
    m = ctx.map_export()
    assert len(m) == len(agg)
    assert [(e.type, e.original) for e in m] == sorted(agg)
    for e in m[::max(1, len(m) // 5000)]:
        f, la, c = agg[(e.type, e.original)]
        assert (e.first_seen, e.last_seen, e.count) == (f, la, c)
        assert e.full_hash == hmac.new(key, e.original, hashlib.sha256).hexdigest()
