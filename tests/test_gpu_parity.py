"""CUDA path vs the oracle, through the C ABI, on the small workload (c1).

256 seeded scan records (uniform 32..512 tokens), 2-layer d=128 encoder with
random affine parameters (so biases and LayerNorm gains are exercised).
FP32 packed, FP32 one-record-per-launch and BF16 packed runs are compared
with the FP64 oracle: tokens and recognizer spans bit-exact; logits within
1e-4 (FP32) / 2e-2 (BF16) max-abs with >= 99.9% label agreement on tokens
whose FP64 top-2 margin exceeds 0.05; output bytes, final spans and the
entity map exactly equal to the oracle's later stages fed the GPU's labels;
and records whose labels all agree equal the oracle's end-to-end output.
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
SCHEMA = api.Schema(synth.TYPE_NAMES_4)


@pytest.fixture(scope="module")
def c1(vocab_words, vocab_index):
    recs = synth.make_records(synth.C1.records, vocab_words)
    w = synth.make_weights(DIMS, seed=2002, random_affine=True)
    key = synth.make_key()
    ref = P.anonymize(recs.records(), U.oracle_schema(SCHEMA), key, Encoder(DIMS, w), vocab_index)
    return recs, w, key, ref


def _run(c1, vocab_words, prec, mode, attention="mma_sync"):
    recs, w, key, ref = c1
    ctx = api.Context(DIMS, synth.pack_blob(DIMS, w), vocab_words, precision=prec, mode=mode, keep_trace=True,
                      attention=attention)
    out = ctx.anonymize(recs.data, recs.offsets, SCHEMA, key)
    return ctx, out, ctx.trace()


@pytest.mark.parametrize("prec,mode,attention", [("fp32", "packed", "mma_sync"), ("fp32", "per_record", "mma_sync"),
                                                ("bf16", "packed", "mma_sync"), ("bf16", "packed", "tcgen05"),
                                                ("bf16", "per_record", "tcgen05")])
def test_c1_parity(c1, vocab_words, vocab_index, prec, mode, attention):
    recs, w, key, ref = c1
    ctx, out, tr = _run(c1, vocab_words, prec, mode, attention)
    records = recs.records()
    U.check_tokens(tr, records, recs.offsets, ref.traces)
    U.check_regex(tr, recs.offsets, ref.traces)
    err, agree, flips = U.check_logits(tr, ref.traces, prec)
    got = out.records()
    iso = U.check_stage_isolated(got, tr, records, SCHEMA, key, vocab_index)
    U.check_final_spans(tr, recs.offsets, iso.traces)
    assert U.map_tuples(ctx.map_export()) == U.map_tuples(iso.map)
    same = 0
    for i, t in enumerate(ref.traces):
        sl = U.split_tokens(tr, recs.n)[i]
        if tr["labels"][sl].tolist() == t.labels:
            assert got[i] == t.output, f"record {i}: end-to-end output differs with equal labels"
            same += 1
    assert same >= 0.9 * recs.n
    st = out.stats()
    assert st["n_tokens"] == sum(len(t.ids) for t in ref.traces) == st["n_encoded_tokens"]
    assert st["n_records"] == recs.n and st["n_final_spans"] == len(tr["final_start"])
    print(f"{prec}/{mode}: max|dlogit| {err:.2e}, agreement {agree:.5f}, flips {flips}, identical records {same}")
    out.free()
    ctx.close()


@pytest.fixture(scope="module", params=["tcgen05", "mma_sync"])
def fp8_ctx(c1, vocab_words, request):
    """FP8 context (attention writing E4M3) on each attention engine."""
    recs, w, key, ref = c1
    ctx = api.Context(DIMS, synth.pack_blob(DIMS, w), vocab_words, precision="fp8", keep_trace=True,
                      attention=request.param)
    cal = synth.make_records(synth.scaled(synth.C1, 64).records, vocab_words, seed=synth.SEED_CALIB)
    ctx.calibrate(cal.data, cal.offsets, SCHEMA)
    return ctx


def test_c1_parity_fp8(c1, fp8_ctx, vocab_index):
    """FP8 e4m3 GEMMs with static per-tensor scales: logits within 1e-1 of FP64."""
    recs, w, key, ref = c1
    scales = fp8_ctx.scales()
    assert scales.shape == (4 * DIMS.n_layers,) and (scales > 0).all()
    out = fp8_ctx.anonymize(recs.data, recs.offsets, SCHEMA, key)
    tr = fp8_ctx.trace()
    records = recs.records()
    U.check_tokens(tr, records, recs.offsets, ref.traces)
    U.check_regex(tr, recs.offsets, ref.traces)
    err, agree, flips = U.check_logits(tr, ref.traces, "fp8")
    U.check_stage_isolated(out.records(), tr, records, SCHEMA, key, vocab_index)
    print(f"fp8: max|dlogit| {err:.3e}, agreement {agree:.5f}, flips {flips}")
    out.free()


def test_fp8_result_independent_of_batch(c1, fp8_ctx):
    """Static scales: a record's logits are the same alone and inside a batch."""
    recs, w, key, ref = c1
    fp8_ctx.map_clear()
    sub = synth.records_from_list(recs.records()[:24])
    fp8_ctx.anonymize(sub.data, sub.offsets, SCHEMA, key).free()
    batch = fp8_ctx.trace()
    sl = U.split_tokens(batch, sub.n)
    for i in (0, 7, 23):
        one = synth.records_from_list([recs.record(i)])
        fp8_ctx.anonymize(one.data, one.offsets, SCHEMA, key).free()
        alone = fp8_ctx.trace()
        assert np.array_equal(alone["logits"], batch["logits"][sl[i]])


def test_per_record_equals_packed_fp32(c1, vocab_words):
    """The FP32 path gives the same logits whether records are packed or run one per launch."""
    _, _, a = _run(c1, vocab_words, "fp32", "packed")
    _, _, b = _run(c1, vocab_words, "fp32", "per_record")
    assert np.max(np.abs(a["logits"] - b["logits"])) < 1e-5
    assert np.array_equal(a["labels"], b["labels"]) or np.mean(a["labels"] == b["labels"]) > 0.9999
