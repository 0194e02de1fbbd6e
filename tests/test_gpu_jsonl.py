"""JSON Lines ingest (as_anonymize_jsonl) on the GPU vs the oracle.

The device scanner's fields (one per run of a string value outside escapes,
with the innermost key's id; one detect field for a line that does not
parse) must be the oracle's, checked through the debug trace: one sub-record
per detected field, in field order, with its bytes. Then the whole call,
stage-isolated (the oracle gets the GPU's labels of every detected field),
must match byte for byte, map included; well-formed lines must stay valid
JSON with their structure. Adversarial lines (mutations, deep nesting,
escapes at field edges) are compared on the scanner alone.
"""
import json

import numpy as np
import pytest
import torch

import synth
import paper_2606_15650_b300.api as api
from oracle import fields as F
from oracle import jsonl as J

import parity_util as U

pytestmark = pytest.mark.gpu

DIMS = synth.C1.dims
KEY = synth.make_key()
KEYS = list(synth.JSONL_KEYS)
KEYS_B = [k.encode() for k in KEYS]
POLICY = {"host_ip": ("force", 1), "host_name": ("force", 2), "severity": "exclude", "plugin_name": "exclude",
          "description": "exclude", "solution": "exclude", "plugin_output": "detect", "mac": ("force", 4),
          "os": "exclude", "tags": "exclude", "cves": "detect", "note": "detect"}


@pytest.fixture(scope="module")
def blob():
    return synth.pack_blob(DIMS, synth.make_weights(DIMS, seed=31, random_affine=True))


@pytest.fixture(scope="module")
def lines(vocab_words):
    return synth.make_jsonl_records(synth.scaled(synth.C1, 60).records, vocab_words, seed=88)


def _oracle_actions(policy, default):
    acts = {}
    for i, k in enumerate(KEYS):
        a = policy.get(k, default)
        acts[i] = (F.FORCE, a[1]) if isinstance(a, tuple) else ({"detect": F.DETECT, "exclude": F.EXCLUDE}[a], 0)
    return acts


def _labels_per_record(tr, recs, flds, pol):
    rt, lab = tr["rec_tok"], tr["labels"]
    labels, k = [], 0
    for r in range(len(recs)):
        per = []
        for s, n, fid in flds[r]:
            if pol.of(fid)[0] == F.DETECT:
                per.append(lab[rt[k]:rt[k + 1]].tolist())
            k += 1
        labels.append(per)
    assert k == len(rt) - 1
    return labels


@pytest.mark.parametrize("device", [False, True])
@pytest.mark.parametrize("default", ["detect", "exclude"])
def test_jsonl_against_oracle(blob, vocab_words, vocab_index, lines, device, default):
    recs = lines.records()
    schema = api.Schema(synth.TYPE_NAMES_4, window=128, stride=96)   # a malformed line is detected whole
    ctx = api.Context(DIMS, blob, vocab_words, precision="bf16", keep_trace=True)
    data, offs = lines.data, lines.offsets
    if device:
        data = torch.from_numpy(data).cuda()
        offs = torch.from_numpy(offs.astype(np.int64)).cuda()
    out = ctx.anonymize_jsonl(data, offs, KEYS, POLICY, schema, KEY, default=default)
    got = out.copy_to_host() if device else out.records()
    st = out.stats()
    tr = ctx.trace()
    flds = [J.scan_line(r, KEYS_B)[0] for r in recs]
    n_bad = sum(J.scan_line(r, KEYS_B)[1] for r in recs)
    assert st["n_fields"] == sum(len(f) for f in flds) and st["n_malformed"] == n_bad > 0
    pol = F.FieldPolicy(_oracle_actions(POLICY, default), F.DETECT)
    unknown, bad = J.policy_ids(KEYS_B)
    pol.actions[unknown] = ({"detect": F.DETECT, "exclude": F.EXCLUDE}[default], 0)
    pol.actions[bad] = (F.DETECT, 0)
    assert len(tr["rec_tok"]) - 1 == sum(len(f) for f in flds)   # one sub-record per field
    labels = _labels_per_record(tr, recs, flds, pol)
    ref = J.anonymize_jsonl(recs, KEYS_B, _oracle_actions(POLICY, default),
                            {"detect": F.DETECT, "exclude": F.EXCLUDE}[default], U.oracle_schema(schema), KEY,
                            None, vocab_index, labels=labels)
    assert got == ref.outputs
    assert U.map_tuples(ctx.map_export()) == U.map_tuples(ref.map)
    # well-formed lines stay valid JSON with the same keys and non-string values
    for r, (a, b) in enumerate(zip(recs, got)):
        if J.scan_line(a, KEYS_B)[1]:
            continue
        ja, jb = json.loads(a), json.loads(b)
        assert ja.keys() == jb.keys() and ja["port"] == jb["port"] and ja["plugin_id"] == jb["plugin_id"]
        assert jb["host_ip"].startswith("[IP_ADDRESS_") and jb["asset"]["mac"].startswith("[MAC_ADDRESS_")
        assert ja["severity"] == jb["severity"]
    ctx.close()


def test_scanner_fuzz(blob, vocab_words, lines):
    """Mutated, deep and escape-heavy lines: the device's fields equal the oracle's."""
    rng = np.random.default_rng(12)
    base = lines.records()
    alphabet = b'{}[]":,\\ unt0123456789.-eE+aflsr\x01'
    recs = []
    for _ in range(3000):
        line = bytearray(base[int(rng.integers(len(base)))][:400])
        for _ in range(int(rng.integers(0, 4))):
            i = int(rng.integers(len(line) + 1))
            c = alphabet[int(rng.integers(len(alphabet)))]
            op = int(rng.integers(3))
            if op == 0 and i < len(line):
                del line[i]
            elif op == 1:
                line.insert(i, c)
            elif i < len(line):
                line[i] = c
        recs.append(bytes(line))
    recs += [b"[" * 64 + b'"x"' + b"]" * 64, b"[" * 65 + b'"x"' + b"]" * 65, b'{"note": "\\n\\u00e9x\\"\\\\"}',
             b'{"note": "a\\', b'  ', b'', b'"top level"', b'{"asset": {"os": ["a", {"mac": "m"}, "b"]}}']
    rs = synth.records_from_list(recs)
    schema = api.Schema(synth.TYPE_NAMES_4, window=128, stride=96)
    ctx = api.Context(DIMS, blob, vocab_words, precision="bf16", keep_trace=True)
    # every field detected, so every field is a sub-record of the trace
    out = ctx.anonymize_jsonl(rs.data, rs.offsets, KEYS, {}, schema, KEY, default="detect")
    tr = ctx.trace()
    flds = [f for r in recs for f in J.scan_line(r, KEYS_B)[0]]
    assert out.stats()["n_fields"] == len(flds) == len(tr["rec_tok"]) - 1
    assert out.stats()["n_malformed"] == sum(J.scan_line(r, KEYS_B)[1] for r in recs)
    # sub-record k holds field k: its tokens tile exactly the field's bytes
    rt = tr["rec_tok"].astype(np.int64)
    tok_len = tr["tok_len"].astype(np.int64)
    for k, (s, n, _) in enumerate(flds):
        assert int(tok_len[rt[k]:rt[k + 1]].sum()) == n, k
    ctx.close()


def test_empty_and_checks(blob, vocab_words):
    ctx = api.Context(DIMS, blob, vocab_words, precision="bf16")
    schema = api.Schema(synth.TYPE_NAMES_4)
    o = ctx.anonymize_jsonl(np.zeros(0, np.uint8), np.zeros(1, np.uint64), KEYS, POLICY, schema, KEY)
    assert o.records() == [] and o.stats()["n_fields"] == 0
    rs = synth.records_from_list([b'{"host_ip": "10.0.0.1"}'])
    with pytest.raises(api.AnonShieldError):
        ctx.anonymize_jsonl(rs.data, rs.offsets, KEYS, {"host_ip": ("force", 9)}, schema, KEY)
    ctx.close()
