"""The tokenizer entry point that allocates nothing (as_tokenize_static).

It exists for callers that cannot call cudaMalloc (hosts that own all device
memory through their own allocator, loops where an allocation would
synchronize the device and stall queued work). Its scratch is a
fixed array inside the library, shared by every call. This test calls it
through the C ABI twice in a row, the second time on a smaller batch so that
stale contents left in the shared array by the first call would show, and
compares every output with the tokens the allocating entry point
(as_anonymize) produces for the same records: token ids, offsets, lengths,
record token ranges and the token count, exactly; and, record by record,
with the oracle's tokenizer (ids, offsets within the record, lengths). It
also checks that a batch over the size limit is refused. This file is collected last on
purpose, so that a failure here does not hide any other test.
"""
import numpy as np
import pytest
import torch

import synth
import paper_2606_15650_b300.api as api
from oracle.tokenizer import tokenize

pytestmark = pytest.mark.gpu


def test_static_tokenizer_matches_allocating_path(vocab_words, vocab_index):
    dims = synth.C1.dims
    blob = synth.pack_blob(dims, synth.make_weights(dims, seed=3))
    ctx = api.Context(dims, blob, vocab_words, precision="fp32", keep_trace=True)
    schema = api.Schema(synth.TYPE_NAMES_4)
    for n, seed in ((160, 41), (37, 42)):
        recs = synth.make_records(synth.scaled(synth.C1, n).records, vocab_words, seed=seed)
        assert len(recs.data) <= api.STATIC_MAX_BYTES
        ctx.anonymize(recs.data, recs.offsets, schema, b"k").free()
        ref = ctx.trace()
        d_data = torch.from_numpy(recs.data).cuda()
        d_offs = torch.from_numpy(recs.offsets.astype(np.int64)).cuda()
        got = api.tokenize_static(ctx, d_data, d_offs)
        torch.cuda.synchronize()
        T = int(got["n_tokens"].item())
        assert T == len(ref["tok_ids"])
        assert np.array_equal(got["tok_ids"][:T].cpu().numpy(), ref["tok_ids"])
        assert np.array_equal(got["tok_off"][:T].cpu().numpy().astype(np.uint32), ref["tok_off"])
        assert np.array_equal(got["tok_len"][:T].cpu().numpy().astype(np.uint32), ref["tok_len"])
        assert np.array_equal(got["rec_tok"].cpu().numpy().astype(np.uint64), ref["rec_tok"])
        # and the oracle's tokenizer, record by record
        rt = got["rec_tok"].cpu().numpy().astype(np.int64)
        ids = got["tok_ids"][:T].cpu().numpy().astype(np.int64)
        off = got["tok_off"][:T].cpu().numpy().astype(np.int64)
        ln = got["tok_len"][:T].cpu().numpy().astype(np.int64)
        for r in range(recs.n):
            a, b = int(rt[r]), int(rt[r + 1])
            o_ids, o_off, o_len = tokenize(recs.record(r), vocab_index)
            base = int(recs.offsets[r])
            assert ids[a:b].tolist() == o_ids, f"record {r}: ids"
            assert (off[a:b] - base).tolist() == o_off, f"record {r}: offsets"
            assert ln[a:b].tolist() == o_len, f"record {r}: lengths"


def test_static_tokenizer_rejects_oversize(vocab_words):
    dims = synth.C1.dims
    ctx = api.Context(dims, synth.pack_blob(dims, synth.make_weights(dims, seed=3)), vocab_words)
    big = torch.zeros(api.STATIC_MAX_BYTES + 1, dtype=torch.uint8, device="cuda")
    offs = torch.tensor([0, big.numel()], dtype=torch.int64, device="cuda")
    with pytest.raises(api.AnonShieldError) as e:
        api.tokenize_static(ctx, big, offs)
    assert e.value.status == -1 and "static limit" in str(e.value)


def test_static_tokenizer_refuses_unusable_tensors(vocab_words):
    """Tensors the kernels cannot read in place are refused before the call: int32
    offsets (the kernels read 64-bit offsets), a strided view of the bytes, host offsets."""
    dims = synth.C1.dims
    ctx = api.Context(dims, synth.pack_blob(dims, synth.make_weights(dims, seed=3)), vocab_words)
    data = torch.zeros(64, dtype=torch.uint8, device="cuda")
    offs = torch.tensor([0, 32], dtype=torch.int64, device="cuda")
    for d, o, msg in ((data[:32], offs.int(), "dtype"), (data[::2], offs, "contiguous"),
                      (data[:32], offs.cpu(), "cuda:0")):
        with pytest.raises(api.AnonShieldError) as e:
            api.tokenize_static(ctx, d, o)
        assert e.value.status == -1 and msg in str(e.value)
