"""Tile autotuner (as_autotune / as_set_tiles) on the GPU.

Every tile configuration must give bit-identical logits: the configuration
only changes which CTA computes an output tile and in which order tiles
are visited, never the accumulation order inside an output. The tuner must
report a timing for every valid configuration and keep the fastest. The
2-SM configuration is also checked against the FP64 oracle directly.
"""
import numpy as np
import pytest

import synth
import paper_2606_15650_b300.api as api
from oracle import pipeline as P
from oracle.encoder import Encoder
from synth.workloads import ModelDims

import parity_util as U

pytestmark = pytest.mark.gpu

SCHEMA = api.Schema(synth.TYPE_NAMES_4)
# d = 256 makes every projection width a multiple of 256 (all eight configurations valid)
DIMS = ModelDims(vocab=8192, d_model=256, n_heads=4, d_ffn=1024, n_layers=2, n_labels=9)


@pytest.fixture(scope="module")
def setup(vocab_words, c1_records):
    blob = synth.pack_blob(DIMS, synth.make_weights(DIMS, seed=7, random_affine=True))
    rs = synth.records_from_list(c1_records.records()[:64])
    return blob, rs


@pytest.mark.parametrize("prec,fused_ln", [("bf16", True), ("bf16", False), ("fp8", False)])
def test_all_tile_configurations_identical(setup, vocab_words, prec, fused_ln):
    """Every configuration, 2-SM pairs included (each CTA of a pair loads half of the
    weight tile; the residual projections run on them only when the LayerNorm is not
    fused)."""
    blob, rs = setup
    ctx = api.Context(DIMS, blob, vocab_words, precision=prec, keep_trace=True, fused_ln=fused_ln)
    if prec == "fp8":
        ctx.calibrate(rs.data, rs.offsets, SCHEMA)
    key = synth.make_key()
    ref = None
    for cfg in (-1, 0, 1, 2, 3, 4, 5, 6, 7):
        ctx.set_tiles([cfg] * 4)
        assert ctx.tiles() == [cfg] * 4
        ctx.map_clear()
        out = ctx.anonymize(rs.data, rs.offsets, SCHEMA, key).records()
        tr = ctx.trace()
        if ref is None:
            ref = (out, tr["logits"])
        else:
            assert out == ref[0]
            assert np.array_equal(tr["logits"], ref[1]), f"configuration {cfg}"
    ctx.close()


def test_autotune_reports_and_keeps_fastest(setup, vocab_words):
    blob, rs = setup
    ctx = api.Context(DIMS, blob, vocab_words, precision="bf16", keep_trace=True)
    ent = ctx.autotune(rows=8192)
    assert [e["role"] for e in ent] == list(api.TUNE_ROLES)
    for e in ent:
        assert e["m"] == 8192 and e["k"] in (256, 1024)
        valid = [x for x in e["ms"] if x >= 0]
        # the fused post-LN blocks: single-CTA tiles (0) or 2-SM pairs (4), each with
        # the long or the short main-loop ring (| 2)
        fused = e["role"] in ("attn_out", "ffn2")
        assert len(valid) == (4 if fused else 8) and all(x > 0 for x in valid)
        if fused:
            assert all(e["ms"][k] > 0 for k in (0, 2, 4, 6))
        assert e["ms"][e["chosen"]] == min(valid)
    assert ctx.tiles() == [e["chosen"] for e in ent]
    ctx.close()


def test_tile_choices_checked(vocab_words):
    dims = synth.C1.dims  # d = 128: 256-column tiles are not valid for the N = 128 / 384 projections
    blob = synth.pack_blob(dims, synth.make_weights(dims, seed=7))
    ctx = api.Context(dims, blob, vocab_words, precision="bf16")
    with pytest.raises(api.AnonShieldError):
        ctx.set_tiles([0, 2, 2, 2])
    ent = ctx.autotune(rows=1024)
    assert ent[0]["ms"][0] < 0 and ent[0]["ms"][2] > 0   # QKV N = 384: only 128-column tiles
    ctx.close()
    f32 = api.Context(dims, blob, vocab_words, precision="fp32")
    with pytest.raises(api.AnonShieldError):
        f32.autotune()
    f32.close()


def test_pair_tiles_match_oracle(setup, vocab_words, vocab_index):
    """2-SM tiles on every projection (BF16, fused LayerNorm blocks): logits within the BF16
    tolerance of the FP64 oracle and output bytes equal to the oracle's later stages fed the
    device labels."""
    blob, rs = setup
    recs = rs.records()
    key = synth.make_key()
    w = synth.make_weights(DIMS, seed=7, random_affine=True)
    ref = P.anonymize(recs, U.oracle_schema(SCHEMA), key, Encoder(DIMS, w), vocab_index)
    ctx = api.Context(DIMS, blob, vocab_words, precision="bf16", keep_trace=True)
    ctx.set_tiles([4, 4, 4, 4])
    out = ctx.anonymize(rs.data, rs.offsets, SCHEMA, key)
    tr = ctx.trace()
    U.check_tokens(tr, recs, rs.offsets, ref.traces)
    err, agree, flips = U.check_logits(tr, ref.traces, "bf16")
    U.check_stage_isolated(out.records(), tr, recs, SCHEMA, key, vocab_index)
    print(f"2-SM tiles: max|dlogit| {err:.2e}, agreement {agree:.5f}")
    ctx.close()
