"""Opt-in launch and stage timing (as_profile / as_profile_read) on the GPU.

One profiled call must time each of its four integer stages once, every
encoder GEMM and attention launch once, with the timed parts adding up to no
more than the whole call measured by CUDA events on the ctx's stream; the
profiled call's output must be the unprofiled call's, byte for byte; turning
profiling off clears the totals.
"""
import pytest
import torch

import synth
import paper_2606_15650_b300.api as api

pytestmark = pytest.mark.gpu


def test_profile_counts_and_totals(vocab_words, c1_records):
    dims = synth.C1.dims
    blob = synth.pack_blob(dims, synth.make_weights(dims, seed=5))
    ctx = api.Context(dims, blob, vocab_words, precision="bf16", graphs=False)
    schema = api.Schema(synth.TYPE_NAMES_4)
    key = synth.make_key()
    # host inputs: the output comes back to the host, where it is compared
    data, offs = c1_records.data, c1_records.offsets
    plain = ctx.anonymize(data, offs, schema, key)
    want = plain.records()
    plain.free()

    stream = torch.cuda.ExternalStream(ctx.stream())
    ctx.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = ctx.anonymize(data, offs, schema, key)
    e1.record(stream)
    e1.synchronize()
    call_ms = e0.elapsed_time(e1)
    st = out.stats()
    assert out.records() == want
    out.free()
    prof = ctx.profile_read()

    assert prof["stage_calls"] == 1
    assert set(prof["stage_ms"]) == set(api.PROFILE_STAGES)
    for name, ms in prof["stage_ms"].items():
        assert ms > 0.0, name
    # one encoder batch here: 4 projections per layer, one attention per layer
    assert st["n_encoded_tokens"] <= 524288
    assert prof["gemm_launches"] == 4 * dims.n_layers
    assert prof["attn_launches"] == dims.n_layers
    timed = prof["gemm_ms"] + prof["attn_ms"] + sum(prof["stage_ms"].values())
    assert timed <= call_ms * 1.001 + 0.05, (timed, call_ms)

    ctx.profile(False)
    cleared = ctx.profile_read()
    assert cleared["stage_calls"] == 0 and cleared["gemm_launches"] == 0
    assert all(v == 0.0 for v in cleared["stage_ms"].values())
    ctx.close()
