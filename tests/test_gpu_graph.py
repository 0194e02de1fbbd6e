"""Encoder batches replayed as CUDA graphs.

Batches are padded to a shape bucket (a power of two up to AS_GRAPH_MAX_ROWS
rows, above that a multiple of 1/16 of the next power of two) and run as one
graph launch after the lane's first batch; the work items of each batch are
copied into one fixed buffer, so every batch of a bucket replays one graph,
within a call and across calls. The results must be bit-identical to
kernel-by-kernel launches (a context with graphs off): the padded rows belong
to no record and padded attention work items to an empty sequence. Covers
BF16 and FP8, sliding windows, a change of tile choices (a new graph is
captured), calls of several large batches, and the FP64 oracle on a replayed
call.
"""
import numpy as np
import pytest

import synth
import paper_2606_15650_b300.api as api
from oracle import pipeline as P
from oracle.encoder import Encoder

import parity_util as U

pytestmark = pytest.mark.gpu

DIMS = synth.C1.dims
KEY = synth.make_key()


@pytest.fixture(scope="module")
def blob():
    return synth.pack_blob(DIMS, synth.make_weights(DIMS, seed=31, random_affine=True))


def _calls(recs):
    """One-record calls, then batches of 3, 8 and 20 records (several row buckets)."""
    out = [[r] for r in recs[:12]]
    out += [recs[12:15], recs[15:23], recs[23:43], recs[43:46]]
    return out


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("window", [0, 96])
def test_graph_replay_bit_identical(blob, vocab_words, c1_records, prec, window):
    schema = api.Schema(synth.TYPE_NAMES_4, window=window, stride=window * 3 // 4)
    recs = c1_records.records()[:60]
    ctxs = [api.Context(DIMS, blob, vocab_words, precision=prec, keep_trace=True, graphs=g) for g in (True, False)]
    if prec == "fp8":
        cal = synth.make_records(synth.scaled(synth.C1, 16).records, vocab_words, seed=synth.SEED_CALIB)
        ctxs[0].calibrate(cal.data, cal.offsets, schema)
        ctxs[1].set_scales(ctxs[0].scales())
    replays = [0, 0]
    for k, batch in enumerate(_calls(recs)):
        if k == 8:  # new tile choices: a new graph must be captured
            for c in ctxs:
                c.set_tiles([2, 2, 3, 3])
        rs = synth.records_from_list(batch)
        res = []
        for j, c in enumerate(ctxs):
            o = c.anonymize(rs.data, rs.offsets, schema, KEY)
            replays[j] += o.stats()["graph_replays"]
            res.append((o.records(), c.trace()))
            o.free()
        assert res[0][0] == res[1][0], f"call {k}"
        assert np.array_equal(res[0][1]["logits"], res[1][1]["logits"]), f"call {k}"
        assert np.array_equal(res[0][1]["labels"], res[1][1]["labels"])
    assert replays[1] == 0
    assert replays[0] >= len(_calls(recs)) - 4   # every call after the first ran its encoder as one graph
    assert sorted((e.type, e.original, e.count) for e in ctxs[0].map_export()) == \
        sorted((e.type, e.original, e.count) for e in ctxs[1].map_export())
    for c in ctxs:
        c.close()


def test_graph_counts_launches(blob, vocab_words, c1_records):
    """A replayed graph counts its kernels in the library's launch counter."""
    ctx = api.Context(DIMS, blob, vocab_words, precision="bf16")
    schema = api.Schema(synth.TYPE_NAMES_4)
    rs = synth.records_from_list(c1_records.records()[:2])
    a = ctx.anonymize(rs.data, rs.offsets, schema, KEY).stats()     # kernel by kernel
    b = ctx.anonymize(rs.data, rs.offsets, schema, KEY).stats()     # captured and launched
    c = ctx.anonymize(rs.data, rs.offsets, schema, KEY).stats()     # replayed
    assert a["graph_replays"] == 0 and b["graph_replays"] == 1 and c["graph_replays"] == 1
    assert a["kernel_launches"] <= b["kernel_launches"] == c["kernel_launches"]
    ctx.close()


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_large_batches_replay_one_graph(blob, vocab_words, c1_records, prec):
    """A call of several encoder batches above AS_GRAPH_MAX_ROWS rows (20,000-row cap): from the
    second call on every batch is a replay, and results equal kernel-by-kernel launches bit for bit."""
    schema = api.Schema(synth.TYPE_NAMES_4)
    rs = c1_records
    ctxs = [api.Context(DIMS, blob, vocab_words, precision=prec, keep_trace=True, graphs=g, max_chunk_tokens=20000)
            for g in (True, False)]
    if prec == "fp8":
        cal = synth.make_records(synth.scaled(synth.C1, 16).records, vocab_words, seed=synth.SEED_CALIB)
        ctxs[0].calibrate(cal.data, cal.offsets, schema)
        ctxs[1].set_scales(ctxs[0].scales())
    for call in range(2):
        res, st = [], []
        for c in ctxs:
            c.map_clear()
            o = c.anonymize(rs.data, rs.offsets, schema, KEY)
            st.append(o.stats())
            res.append((o.records(), c.trace()))
            o.free()
        n_batches = -(-st[0]["n_encoded_tokens"] // 20000)
        assert n_batches >= 3
        assert res[0][0] == res[1][0]
        assert np.array_equal(res[0][1]["logits"], res[1][1]["logits"])
        assert st[1]["graph_replays"] == 0
        if call == 1:
            assert st[0]["graph_replays"] >= n_batches - 1 and st[0]["graph_replays"] >= 3
    for c in ctxs:
        c.close()


def test_replayed_call_matches_oracle(blob, vocab_words, vocab_index, c1_records):
    """The FP64 oracle against a call whose encoder ran as graph replays (BF16, 2e-2)."""
    schema = api.Schema(synth.TYPE_NAMES_4)
    recs = c1_records.records()[:96]
    rs = synth.records_from_list(recs)
    w = synth.make_weights(DIMS, seed=31, random_affine=True)
    ref = P.anonymize(recs, U.oracle_schema(schema), KEY, Encoder(DIMS, w), vocab_index)
    ctx = api.Context(DIMS, blob, vocab_words, precision="bf16", keep_trace=True, max_chunk_tokens=4096)
    ctx.anonymize(rs.data, rs.offsets, schema, KEY).free()      # captures
    ctx.map_clear()
    out = ctx.anonymize(rs.data, rs.offsets, schema, KEY)
    assert out.stats()["graph_replays"] >= 3
    tr = ctx.trace()
    U.check_tokens(tr, recs, rs.offsets, ref.traces)
    err, agree, flips = U.check_logits(tr, ref.traces, "bf16")
    # record indices continue across calls: the second call's records are 96..191
    iso = U.check_stage_isolated(out.records(), tr, recs, schema, KEY, vocab_index, record_base=len(recs))
    assert U.map_tuples(ctx.map_export()) == U.map_tuples(iso.map)
    print(f"replayed call: max|dlogit| {err:.2e}, agreement {agree:.5f}")
    ctx.close()
