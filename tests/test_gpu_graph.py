"""Small encoder batches replayed as CUDA graphs.

Batches of at most AS_GRAPH_MAX_ROWS rows are padded to power-of-two shapes
and run as one graph launch after the lane's first batch. The results must be
bit-identical to kernel-by-kernel launches (a context with graphs off): the
padded rows belong to no record and padded attention work items to an empty
sequence. Covers BF16 and FP8, sliding windows, and a change of tile choices
(a new graph is captured).
"""
import numpy as np
import pytest

import synth
import paper_2606_15650_b300.api as api

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
