"""The seeded record generator keeps every record within its token target.

The generator sizes records with an upper-bound token estimate; every record
of the sampled workloads, tokenized by the oracle, must have at most its
target count of tokens, hence at most the workload's length cap (records over
max_pos without windows are refused by the library). The 20,000-record sample
of the 70,951-record workload once produced a 513-token record (a field label
added past the room left), which this file keeps covered.
"""
import pytest

import synth
from oracle.tokenizer import build_vocab_index, tokenize


@pytest.fixture(scope="module")
def vi(vocab_words):
    return build_vocab_index(vocab_words)


@pytest.mark.parametrize("shape,n", [(synth.C1, None), (synth.C2, 3000), (synth.C3, 600), (synth.C4, 2000),
                                     (synth.C5, 200), (synth.C1X, None)])
def test_records_within_target(vocab_words, vi, shape, n):
    w = synth.scaled(shape, n) if n else shape
    recs = synth.make_records(w.records, vocab_words, seed=synth.SEED_RECORDS)
    for i in range(recs.n):
        t = len(tokenize(recs.record(i), vi)[0])
        assert t <= int(recs.target_tokens[i]) <= w.records.hi, (i, t, int(recs.target_tokens[i]))


def test_dataset_sample_that_once_overflowed(vocab_words, vi):
    w = synth.scaled(synth.C2, 20000)
    recs = synth.make_records(w.records, vocab_words, seed=synth.SEED_RECORDS)
    long = [i for i in range(recs.n) if recs.target_tokens[i] >= 500]
    assert 7498 in long
    for i in long:
        assert len(tokenize(recs.record(i), vi)[0]) <= 512, i
