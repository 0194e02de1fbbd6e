"""The device entity map under Zipf(1.1) entity reuse over 50,000 distinct
entities (the packed-batch workload's entity draw), against the oracle.

3,000 records of that workload's shape (lognormal lengths around 600 tokens,
16..4,096, windows 512/384) go in two calls of 1,500. The 2-layer d=128
encoder in BF16 supplies the NER labels, which the oracle takes as given
(stage isolation: its tokenizer, recognizers, BIO decode, overlap rule, HMAC,
map and substitution run on the GPU's labels). Checked after each call:

* every output record, byte for byte;
* the whole exported map equal to the oracle's, entry by entry (type, bytes,
  HMAC, first and last record, count), the second call's record indices
  continuing from the first's and its counts adding to them;
* that the draw really reuses: more than 10,000 distinct entities, over a
  thousand of them seen in both calls.
"""
import pytest

import synth
import paper_2606_15650_b300.api as api
from oracle import pipeline as P

import parity_util as U

pytestmark = pytest.mark.gpu

N_CALL = 1500


@pytest.fixture(scope="module")
def zipf_case(vocab_words):
    w = synth.scaled(synth.C3, 2 * N_CALL)
    assert w.records.zipf_distinct == 50000
    recs = synth.make_records(w.records, vocab_words)
    dims = synth.C1.dims
    blob = synth.pack_blob(dims, synth.make_weights(dims, seed=2003, random_affine=True))
    ctx = api.Context(dims, blob, vocab_words, precision="bf16", keep_trace=True)
    schema = api.Schema(synth.TYPE_NAMES_4, window=w.window, stride=w.stride)
    yield recs.records(), ctx, schema, synth.make_key()
    ctx.close()


def test_zipf_entity_map_two_calls(zipf_case, vocab_index):
    records, ctx, schema, key = zipf_case
    emap = {}          # the oracle's map, carried across the two calls like the device's
    maps = []
    for c in range(2):
        part = records[c * N_CALL:(c + 1) * N_CALL]
        sub = synth.records_from_list(part)
        out = ctx.anonymize(sub.data, sub.offsets, schema, key)
        got = out.records()
        out.free()
        labels = U.gpu_labels_per_record(ctx.trace(), len(part))
        ref = P.anonymize_from_labels(part, labels, U.oracle_schema(schema), key, vocab_index,
                                      record_base=c * N_CALL, emap=emap)
        for i, (a, b) in enumerate(zip(got, ref.outputs)):
            assert a == b, f"call {c}, record {i}: output bytes differ"
        device_map = sorted(U.map_tuples(ctx.map_export()))
        oracle_map = sorted(U.map_tuples(ref.map))
        assert len(device_map) == len(oracle_map), (c, len(device_map), len(oracle_map))
        assert device_map == oracle_map, f"call {c}: entity map differs"
        maps.append(oracle_map)
    final = maps[1]
    print(f"distinct entities: {len(maps[0])} after one call, {len(final)} after two")
    assert len(final) > 10000
    # (type, original, hash, first_seen, last_seen, count): seen in both calls
    assert sum(1 for e in final if e[3] < N_CALL <= e[4]) > 1000
