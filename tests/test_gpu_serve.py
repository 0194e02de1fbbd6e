"""Serving loop (continuous batching) through the C ABI on the GPU.

A served request's result must not depend on the batch it joined: each
record's output is compared with the same records run as one as_anonymize
call (and a sample with each record run alone), under several admission
budgets and lane counts, with requests submitted from several threads. With
one submitter the request ids are the record indices, so the served entity
map (first_seen / last_seen / count) must equal the map of the single call.
"""
import threading
import time

import numpy as np
import pytest

import synth
import paper_2606_15650_b300.api as api

import parity_util as U

pytestmark = pytest.mark.gpu

DIMS = synth.C1.dims
SCHEMA = api.Schema(synth.TYPE_NAMES_4)
KEY = synth.make_key()


@pytest.fixture(scope="module")
def blob():
    return synth.pack_blob(DIMS, synth.make_weights(DIMS, seed=31, random_affine=True))


@pytest.fixture(scope="module")
def batch_ref(blob, vocab_words, c1_records):
    recs = c1_records.records()[:240]
    ctx = api.Context(DIMS, blob, vocab_words, precision="bf16")
    rs = synth.records_from_list(recs)
    got = ctx.anonymize(rs.data, rs.offsets, SCHEMA, KEY).records()
    emap = sorted(U.map_tuples(ctx.map_export()))
    ctx.close()
    return recs, got, emap


def _ctx(blob, words, **kw):
    return api.Context(DIMS, blob, words, precision="bf16", **kw)


def test_batch_independence_alone(blob, vocab_words, batch_ref):
    recs, got, _ = batch_ref
    ctx = _ctx(blob, vocab_words)
    for i in range(0, len(recs), 16):
        rs = synth.records_from_list([recs[i]])
        assert ctx.anonymize(rs.data, rs.offsets, SCHEMA, KEY).records()[0] == got[i], i


@pytest.mark.parametrize("lanes,batch_bytes,chunk", [(1, 1, 0), (2, 0, 8192), (3, 3000, 0), (4, 20000, 16384)])
def test_served_equals_batch(blob, vocab_words, batch_ref, lanes, batch_bytes, chunk):
    recs, got, emap = batch_ref
    ctx = _ctx(blob, vocab_words, max_chunk_tokens=chunk)
    ctx.serve_start(SCHEMA, KEY, lanes=lanes, max_batch_bytes=batch_bytes)
    ids = [ctx.submit(r) for r in recs]
    assert ids == list(range(len(recs)))
    out = [ctx.poll(i, timeout_s=60) for i in ids]
    st = ctx.serve_stats()
    assert st["completed"] == len(recs) and st["failed"] == 0 and st["pending"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    if batch_bytes == 1:
        assert st["batches"] == len(recs)
    for i in range(len(recs)):
        assert out[i] == got[i], i
    assert sorted(U.map_tuples(ctx.map_export())) == emap
    with pytest.raises(api.AnonShieldError):
        one = synth.records_from_list(recs[:1])
        ctx.anonymize(one.data, one.offsets, SCHEMA, KEY)
    ctx.serve_stop()
    ctx.close()


def test_served_multithreaded_mix(blob, vocab_words, batch_ref):
    recs, got, _ = batch_ref
    ctx = _ctx(blob, vocab_words)
    ctx.serve_start(SCHEMA, KEY, lanes=3, max_batch_bytes=4096)
    res, errs = {}, []

    def client(t):
        try:
            mine = [(i, ctx.submit(recs[i])) for i in range(t, len(recs), 4)]
            for i, rid in mine:
                res[i] = ctx.poll(rid, timeout_s=60)
        except Exception as e:  # reported below
            errs.append(e)

    th = [threading.Thread(target=client, args=(t,)) for t in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join(120)
    assert not errs, errs
    assert all(res[i] == got[i] for i in range(len(recs)))
    ctx.serve_stop()
    ctx.close()


def test_admission_bound_and_discard(blob, vocab_words, batch_ref):
    recs = batch_ref[0]
    ctx = _ctx(blob, vocab_words)
    ctx.serve_start(SCHEMA, KEY, lanes=2, max_pending=2)
    accepted = sum(ctx.submit(recs[i % len(recs)], discard=True) is not None for i in range(400))
    t0 = time.time()
    while time.time() - t0 < 60:
        st = ctx.serve_stats()
        if st["pending"] == 0 and st["completed"] + st["failed"] == accepted:
            break
        time.sleep(0.01)
    assert st["completed"] == accepted and st["rejected"] == 400 - accepted and st["failed"] == 0
    rid = ctx.submit(recs[0], discard=True)
    with pytest.raises(api.AnonShieldError):
        ctx.poll(rid, timeout_s=1)
    with pytest.raises(api.AnonShieldError):
        ctx.poll(10 ** 9, timeout_s=0)
    ctx.serve_stop()


def test_stop_drains_and_batch_api_resumes(blob, vocab_words, batch_ref):
    recs, got, _ = batch_ref
    ctx = _ctx(blob, vocab_words)
    ctx.serve_start(SCHEMA, KEY)
    for r in recs[:50]:
        ctx.submit(r, discard=True)
    ctx.serve_stop()
    n_before = {e.original: e.count for e in ctx.map_export()}
    assert sum(n_before.values()) > 0
    rs = synth.records_from_list(recs[50:60])
    out = ctx.anonymize(rs.data, rs.offsets, SCHEMA, KEY).records()
    assert out == got[50:60]
    # record indices continue after the served requests
    assert max(e.last_seen for e in ctx.map_export()) >= 50


def test_replica_maps_merge_to_single_run(blob, vocab_words, batch_ref):
    """Two contexts (replicas) on disjoint halves, merged on the host == one context over all."""
    from paper_2606_15650_b300 import replicas
    recs, got, emap = batch_ref
    ranges = replicas.shard_ranges(np.array([len(r) for r in recs]), 2)
    shards, outs = [], []
    for a, b in ranges:
        ctx = _ctx(blob, vocab_words)
        rs = synth.records_from_list(recs[a:b])
        outs += ctx.anonymize(rs.data, rs.offsets, SCHEMA, KEY).records()
        shards.append(ctx.map_export())
        ctx.close()
    assert outs == got
    merged = api.map_merge(shards, [a for a, _ in ranges])
    assert sorted(U.map_tuples(merged)) == emap


# ---------------------------------------------------------------- against the oracle, serving-shaped records

@pytest.fixture(scope="module")
def c4_oracle(vocab_words, vocab_index):
    """Serving-shaped records (lognormal(300, 0.6) clipped 32..4096 tokens, windows 512/384) through
    the FP64 oracle end to end, with each record's smallest FP64 top-2 logit margin."""
    from oracle import pipeline as P
    from oracle.encoder import Encoder
    recs = synth.make_records(synth.scaled(synth.C4, 48).records, vocab_words, seed=synth.SEED_RECORDS + 4)
    recs = recs.records()
    w = synth.make_weights(DIMS, seed=31, random_affine=True)
    sch = P.Schema(synth.TYPE_NAMES_4, window=512, stride=384)
    ref = P.anonymize(recs, sch, KEY, Encoder(DIMS, w), vocab_index)
    margin = []
    for t in ref.traces:
        if t.logits is None or len(t.logits) == 0:
            margin.append(np.inf)
            continue
        s = np.sort(t.logits, axis=1)
        margin.append(float((s[:, -1] - s[:, -2]).min()))
    assert max(len(t.ids) for t in ref.traces) > 512      # some records run as several windows
    return recs, ref, np.array(margin)


def _check_vs_oracle(got, recs, ref, margin, tol=1e-4):
    """Records whose FP64 labels cannot flip under an FP32 error of tol equal the oracle's output."""
    safe = margin > 2 * tol
    assert safe.mean() > 0.9
    for i in np.nonzero(safe)[0]:
        assert got[i] == ref.outputs[i], f"record {i}"
    return int(safe.sum())


def test_served_fp32_windows_equal_oracle(blob, vocab_words, c4_oracle):
    """FP32 serving with 512/384 windows and records up to 4,096 tokens: every served record equals
    the oracle's end-to-end output (records with a near-tie FP64 label excepted), and the served
    entity map equals the oracle's over those records when all qualify."""
    recs, ref, margin = c4_oracle
    ctx = api.Context(DIMS, blob, vocab_words, precision="fp32")
    ctx.serve_start(api.Schema(synth.TYPE_NAMES_4, window=512, stride=384), KEY, lanes=2)
    ids = [ctx.submit(r) for r in recs]
    got = [ctx.poll(i, timeout_s=120) for i in ids]
    n = _check_vs_oracle(got, recs, ref, margin)
    if n == len(recs):
        assert sorted(U.map_tuples(ctx.map_export())) == sorted(U.map_tuples(ref.map))
    ctx.serve_stop()
    ctx.close()


def test_admission_by_activation_budget(blob, vocab_words, c4_oracle):
    """A small activation budget: the lanes' encoder activations never exceed it, batches stay
    within the row cap (records longer than the cap run as several encoder batches), and the
    results equal the oracle's, as with the default budget."""
    recs, ref, margin = c4_oracle
    ctx = api.Context(DIMS, blob, vocab_words, precision="fp32")
    # FP32 activation buffers per row (row indices, X, Y, QKV, attention out, FFN), each allocated
    # with 1/8 slack: a budget of 1,152 rows' worth per lane is a 1,024-row cap
    per_row = 4 + 4 + 1 + 4 * DIMS.d_model * 2 + 4 * 3 * DIMS.d_model + 4 * DIMS.d_model + 4 * DIMS.d_ffn
    budget = 2 * 1152 * per_row          # 1-2 records per batch
    ctx.serve_start(api.Schema(synth.TYPE_NAMES_4, window=512, stride=384), KEY, lanes=2,
                    activation_budget=budget)
    st0 = ctx.serve_stats()
    assert st0["activation_budget"] == budget and st0["row_cap"] == 1024
    ids = [ctx.submit(r) for r in recs]
    got = [ctx.poll(i, timeout_s=120) for i in ids]
    st = ctx.serve_stats()
    assert st["completed"] == len(recs) and st["failed"] == 0
    assert 0 < st["activation_peak"] <= budget, st
    assert st["batches"] > len(recs) // 4
    _check_vs_oracle(got, recs, ref, margin)
    ctx.serve_stop()
    with pytest.raises(api.AnonShieldError):       # a budget below one full sequence per lane
        ctx.serve_start(SCHEMA, KEY, lanes=2, activation_budget=2 * 288 * per_row)
    ctx.close()
