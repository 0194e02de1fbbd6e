"""Edge cases of the C ABI on the GPU, each compared with the oracle.

Empty batches and records, whitespace-only and single-byte records, a
record of exactly max_pos tokens, one over max_pos (AS_ERR_TOO_LONG without
windows, sliding windows with it), slug lengths 0 / 7 / 64, the preserve
list, keys of length 0 and 131 (hashed first), a key change on a non-empty
map (AS_ERR_STATE), two calls sharing one map (record indices continue),
device-resident inputs, map export/import round trip, invalid arguments.
"""
import numpy as np
import pytest
import torch

import synth
import paper_2606_15650_b300.api as api
from oracle import pipeline as P
from oracle.encoder import Encoder

import parity_util as U

pytestmark = pytest.mark.gpu

DIMS = synth.C1.dims
SCHEMA = api.Schema(synth.TYPE_NAMES_4)


@pytest.fixture(scope="module")
def model():
    w = synth.make_weights(DIMS, seed=31, random_affine=True)
    return w, synth.pack_blob(DIMS, w), Encoder(DIMS, w)


def _arrays(recs: list[bytes]):
    rs = synth.records_from_list(recs)
    return rs.data, rs.offsets


def _ctx(model, words, prec="fp32", **kw):
    return api.Context(DIMS, model[1], words, precision=prec, keep_trace=True, **kw)


@pytest.mark.parametrize("attention", ["mma_sync", "tcgen05"])
def test_windows_both_attention_engines(model, vocab_words, vocab_index, c1_records, attention):
    recs = c1_records.records()[40:70]
    ctx = _ctx(model, vocab_words, prec="bf16", attention=attention)
    win = api.Schema(synth.TYPE_NAMES_4, window=128, stride=96)
    _check_full(ctx, recs, win, synth.make_key(), model, vocab_index)


def _check_full(ctx, recs, schema, key, model, vocab_index, record_base=0, emap=None):
    data, offs = _arrays(recs)
    out = ctx.anonymize(data, offs, schema, key)
    tr = ctx.trace()
    ref = P.anonymize(recs, U.oracle_schema(schema), key, model[2], vocab_index, record_base=record_base, emap=emap)
    U.check_tokens(tr, recs, offs, ref.traces)
    U.check_regex(tr, offs, ref.traces)
    if any(len(t.ids) for t in ref.traces):
        U.check_logits(tr, ref.traces, ctx.precision)
    got = out.records()
    U.check_stage_isolated(got, tr, recs, schema, key, vocab_index, record_base=record_base)
    return out, got, ref


def test_empty_batch(model, vocab_words):
    ctx = _ctx(model, vocab_words)
    out = ctx.anonymize(np.zeros(0, np.uint8), np.zeros(1, np.uint64), SCHEMA, b"k")
    assert out.records() == []
    assert out.stats()["n_records"] == 0


def test_degenerate_records(model, vocab_words, vocab_index):
    recs = [b"", b"   \t\n", b"x", b"", b"10.0.0.1", b"a " * 256, b"\xff\xfe", b"CVE-2024-0001."]
    ctx = _ctx(model, vocab_words)
    out, got, ref = _check_full(ctx, recs, SCHEMA, b"key", model, vocab_index)
    assert got[0] == b"" and got[3] == b""
    assert got[4].startswith(b"[IP_ADDRESS_") and len(ref.traces[5].ids) == 512


def test_too_long_without_windows_and_windows(model, vocab_words, vocab_index):
    long = b"ab " * 300 + b"host 192.168.1.1 done"   # > 512 tokens
    ctx = _ctx(model, vocab_words)
    data, offs = _arrays([long])
    with pytest.raises(api.AnonShieldError) as e:
        ctx.anonymize(data, offs, SCHEMA, b"k")
    assert e.value.status == -4
    win = api.Schema(synth.TYPE_NAMES_4, window=128, stride=96)
    out, got, ref = _check_full(ctx, [long, b"short one", long[:700]], win, b"k", model, vocab_index)
    assert out.stats()["n_encoded_tokens"] > out.stats()["n_tokens"]


def test_windows_on_c1_records(model, vocab_words, vocab_index, c1_records):
    recs = c1_records.records()[:40]
    ctx = _ctx(model, vocab_words, prec="bf16")
    win = api.Schema(synth.TYPE_NAMES_4, window=64, stride=48)
    _check_full(ctx, recs, win, synth.make_key(), model, vocab_index)


@pytest.mark.parametrize("slug", [0, 7, 64])
def test_slug_lengths_and_preserve(model, vocab_words, vocab_index, c1_records, slug):
    recs = c1_records.records()[:30]
    sch = api.Schema(synth.TYPE_NAMES_4, preserve_mask=(1 << 3) | (1 << 4), slug_hex_len=slug)
    ctx = _ctx(model, vocab_words)
    out, got, ref = _check_full(ctx, recs, sch, b"slug-key", model, vocab_index)
    assert all(b"[CVE_ID" not in g and b"[MAC_ADDRESS" not in g for g in got)


@pytest.mark.parametrize("key", [b"", bytes(range(131)), bytes(64), b"\x00"])
def test_keys(model, vocab_words, vocab_index, c1_records, key):
    recs = c1_records.records()[:10]
    ctx = _ctx(model, vocab_words)
    _check_full(ctx, recs, SCHEMA, key, model, vocab_index)


def test_key_change_and_map_across_calls(model, vocab_words, vocab_index, c1_records):
    recs = c1_records.records()[:60]
    ctx = _ctx(model, vocab_words)
    emap = {}
    out1, _, _ = _check_full(ctx, recs[:25], SCHEMA, b"K1", model, vocab_index, record_base=0, emap=emap)
    tr1 = ctx.trace()
    out2, _, ref2 = _check_full(ctx, recs[25:], SCHEMA, b"K1", model, vocab_index, record_base=25, emap=emap)
    # the whole map equals the oracle's map over both calls, fed the GPU labels
    lab1 = U.gpu_labels_per_record(tr1, 25)
    lab2 = U.gpu_labels_per_record(ctx.trace(), len(recs) - 25)
    em = {}
    P.anonymize_from_labels(recs[:25], lab1, U.oracle_schema(SCHEMA), b"K1", vocab_index, 0, em)
    whole = P.anonymize_from_labels(recs[25:], lab2, U.oracle_schema(SCHEMA), b"K1", vocab_index, 25, em)
    assert U.map_tuples(ctx.map_export()) == U.map_tuples(whole.map)
    touched = out2.map()
    assert {(e.type, e.original) for e in touched} == {(t, o) for (t, o) in
                                                        {(s[2], r[s[0]:s[0] + s[1]]) for tr, r in
                                                         zip(whole.traces, recs[25:]) for s in tr.final}}
    assert all(e.slug == e.full_hash[:10] for e in touched)
    data, offs = _arrays(recs[:3])
    with pytest.raises(api.AnonShieldError) as e:
        ctx.anonymize(data, offs, SCHEMA, b"K2")
    assert e.value.status == -6
    ctx.map_clear()
    ctx.anonymize(data, offs, SCHEMA, b"K2").free()


def test_device_inputs_match_host(model, vocab_words, c1_records):
    recs = c1_records.records()[:50]
    data, offs = _arrays(recs)
    ctx_h = _ctx(model, vocab_words, prec="bf16")
    host = ctx_h.anonymize(data, offs, SCHEMA, b"dev").records()
    ctx_d = _ctx(model, vocab_words, prec="bf16")
    dd = torch.from_numpy(data).cuda()
    do = torch.from_numpy(offs.astype(np.int64)).cuda()
    out = ctx_d.anonymize(dd, do, SCHEMA, b"dev")
    assert out.device_pointers()[2] == len(recs)
    assert out.copy_to_host() == host


def test_map_export_import_roundtrip(model, vocab_words, c1_records):
    recs = c1_records.records()[:20]
    data, offs = _arrays(recs)
    a = _ctx(model, vocab_words)
    a.anonymize(data, offs, SCHEMA, b"RT").free()
    exported = a.map_export()
    assert exported
    b = _ctx(model, vocab_words)
    b.map_import(b"RT", exported)
    assert U.map_tuples(b.map_export()) == U.map_tuples(exported)
    b.map_import(b"RT", exported)   # importing again sums counts, keeps min/max sightings
    again = b.map_export()
    assert [e.count for e in again] == [2 * e.count for e in exported]
    with pytest.raises(api.AnonShieldError) as e:
        b.map_import(b"other", exported)
    assert e.value.status == -6


def test_invalid_arguments(model, vocab_words):
    ctx = _ctx(model, vocab_words)
    with pytest.raises(api.AnonShieldError) as e:
        ctx.anonymize(np.frombuffer(b"abcdef", np.uint8), np.array([0, 4, 2, 6], np.uint64), SCHEMA, b"k")
    assert e.value.status == -1
    with pytest.raises(api.AnonShieldError):
        ctx.anonymize(np.frombuffer(b"abc", np.uint8), np.array([0, 3], np.uint64),
                      api.Schema(synth.TYPE_NAMES_8), b"k")
    with pytest.raises(api.AnonShieldError):
        ctx.anonymize(np.frombuffer(b"abc", np.uint8), np.array([0, 3], np.uint64),
                      api.Schema(synth.TYPE_NAMES_4, slug_hex_len=65), b"k")
    with pytest.raises(api.AnonShieldError):
        api.Context(DIMS, model[1][:-1], vocab_words)
