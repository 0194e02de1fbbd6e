"""Per-field policy (as_anonymize_fields) on the GPU.

- One detected field covering each record gives exactly as_anonymize.
- Fielded scan records under mixed policies (forced, excluded, detected
  columns; forced types under a preserve list) against the oracle, stage-
  isolated: the oracle gets the GPU's own labels for every detected field
  (from the debug trace, one sub-record per field) and everything else must
  match byte for byte, map included (record indices of the records).
- Device-resident records, empty and whitespace-only forced values, and the
  argument checks.
"""
import numpy as np
import pytest
import torch

import synth
import paper_2606_15650_b300.api as api
from oracle import fields as F
from oracle import pipeline as P

import parity_util as U

pytestmark = pytest.mark.gpu

DIMS = synth.C1.dims
KEY = synth.make_key()


@pytest.fixture(scope="module")
def blob():
    return synth.pack_blob(DIMS, synth.make_weights(DIMS, seed=31, random_affine=True))


@pytest.fixture(scope="module")
def fielded(vocab_words):
    return synth.make_fielded_records(synth.scaled(synth.C1, 40).records, vocab_words, seed=77)


def _abs_fields(fr):
    return fr.start, fr.length, fr.field_id


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
def test_single_field_is_whole_record(blob, vocab_words, c1_records, prec):
    recs = c1_records.records()[:30]
    rs = synth.records_from_list(recs)
    schema = api.Schema(synth.TYPE_NAMES_4)
    a = api.Context(DIMS, blob, vocab_words, precision=prec)
    b = api.Context(DIMS, blob, vocab_words, precision=prec)
    ref = a.anonymize(rs.data, rs.offsets, schema, KEY).records()
    start = rs.offsets[:-1].astype(np.uint64)
    length = np.diff(rs.offsets).astype(np.uint32)
    got = b.anonymize_fields(rs.data, rs.offsets, start, length, np.zeros(len(recs), np.uint32), {}, schema, KEY)
    assert got.records() == ref
    assert U.map_tuples(b.map_export()) == U.map_tuples(a.map_export())
    assert got.stats()["n_records"] == len(recs)


POLICY = {0: ("force", 1), 1: ("force", 2), 2: "exclude", 3: "exclude", 4: "exclude", 5: "exclude",
          6: "detect", 7: "exclude", 8: "detect"}


def _oracle_policy(pol):
    out = F.FieldPolicy(default=F.DETECT)
    for fid, a in pol.items():
        if isinstance(a, tuple):
            out.actions[fid] = (F.FORCE, a[1])
        else:
            out.actions[fid] = ({"detect": F.DETECT, "exclude": F.EXCLUDE}[a], 0)
    return out


@pytest.mark.parametrize("preserve", [0, 1 << 2])
@pytest.mark.parametrize("device", [False, True])
def test_fielded_against_oracle(blob, vocab_words, vocab_index, fielded, preserve, device):
    fr = fielded
    schema = api.Schema(synth.TYPE_NAMES_4, preserve_mask=preserve)
    ctx = api.Context(DIMS, blob, vocab_words, precision="bf16", keep_trace=True)
    data, offs = fr.records.data, fr.records.offsets
    if device:
        data = torch.from_numpy(data).cuda()
        offs = torch.from_numpy(offs.astype(np.int64)).cuda()
    out = ctx.anonymize_fields(data, offs, fr.start, fr.length, fr.field_id, POLICY, schema, KEY)
    got = out.copy_to_host() if device else out.records()
    tr = ctx.trace()
    # labels of every sub-record (one per field, in field order); detected fields only
    rt, lab = tr["rec_tok"], tr["labels"]
    assert len(rt) == len(fr.start) + 1
    pol = _oracle_policy(POLICY)
    recs = fr.records.records()
    labels, k = [], 0
    for r in range(len(recs)):
        per = []
        for s, n, fid in fr.fields_of(r):
            if pol.of(fid)[0] == F.DETECT:
                per.append(lab[rt[k]:rt[k + 1]].tolist())
            else:
                assert rt[k + 1] == rt[k]   # no tokens for fields that are not detected
            k += 1
        labels.append(per)
    ref = F.anonymize_fields(recs, [fr.fields_of(r) for r in range(len(recs))], pol,
                             U.oracle_schema(schema), KEY, None, vocab_index, labels=labels)
    assert got == ref.outputs
    assert U.map_tuples(ctx.map_export()) == U.map_tuples(ref.map)
    # the forced columns were replaced whatever the preserve list says
    for r, o in enumerate(got):
        assert o.startswith(b"[IP_ADDRESS_") and b" | [HOSTNAME_" in o
    ctx.close()


def test_forced_edge_values_and_checks(blob, vocab_words):
    ctx = api.Context(DIMS, blob, vocab_words, precision="bf16")
    schema = api.Schema(synth.TYPE_NAMES_4)
    recs = [b"a=  \t;b=x;c=", b"", b"q=10.0.0.1"]
    rs = synth.records_from_list(recs)
    o = rs.offsets
    start = np.array([o[0] + 2, o[0] + 8, o[0] + 12, o[2] + 2], np.uint64)
    length = np.array([3, 1, 0, 8], np.uint32)
    fid = np.array([0, 0, 0, 1], np.uint32)
    got = ctx.anonymize_fields(rs.data, rs.offsets, start, length, fid, {0: ("force", 2), 1: "exclude"},
                               schema, KEY).records()
    assert got[0].startswith(b"a=  \t;b=[HOSTNAME_") and got[0].endswith(b"];c=")
    assert got[1] == b"" and got[2] == b"q=10.0.0.1"   # excluded: the IP stays
    bad = [
        (np.array([5, 2], np.uint64), np.array([1, 1], np.uint32)),          # not sorted
        (np.array([0, 1], np.uint64), np.array([3, 1], np.uint32)),          # overlapping
        (np.array([o[0] + 10], np.uint64), np.array([5], np.uint32)),         # crosses into the next record
    ]
    for s, l in bad:
        with pytest.raises(api.AnonShieldError):
            ctx.anonymize_fields(rs.data, rs.offsets, s, l, np.zeros(len(s), np.uint32), {}, schema, KEY)
    with pytest.raises(api.AnonShieldError):
        ctx.anonymize_fields(rs.data, rs.offsets, start, length, fid, {0: ("force", 9)}, schema, KEY)
    ctx.close()
