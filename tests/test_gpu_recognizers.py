"""The twelve pattern recognizers on the GPU vs the oracle, through the C ABI.

Records with every recognizer kind planted (c1x: URLs, hashes, CPE names,
UUIDs, OIDs, certificate fingerprints and PEM blocks besides the address and
CVE kinds) run through a 23-label encoder: tokens and recognizer spans are
bit-exact, and the output bytes, final spans and entity map equal the
oracle's later stages fed the GPU's labels. Adversarial records (edges of
each rule, multi-word spans covering other candidates, candidates cut by the
record end, multi-word spans longer than the resolve pass's 512-byte step)
are compared span by span under several recognizer tables. The serving and
streaming paths carry the table as well.
"""
import numpy as np
import pytest

import synth
import paper_2606_15650_b300.api as api
from oracle import pipeline as P
from oracle import recognizers as R
from oracle.encoder import Encoder

import parity_util as U
from rx_fuzz import fuzz_record

pytestmark = pytest.mark.gpu

DIMS = synth.C1X.dims
KEY = synth.make_key()
ALL = api.recognizer_table({"mac": 4, "ipv6": 1, "ipv4": 1, "cve": 3, "hostname": 2, "url": 5, "hash": 6,
                            "uuid": 9, "cpe": 7, "oid": 10, "cert_fp": 11, "pem": 11})
assert ALL == synth.RECOGNIZERS_11
SCHEMA = api.Schema(synth.TYPE_NAMES_11, recognizers=ALL)
TABLES = {
    "all": ALL,
    "multiword_only": api.recognizer_table({"url": 5, "cpe": 7, "pem": 11}),
    "words_only": api.recognizer_table({"mac": 4, "ipv6": 1, "ipv4": 1, "cve": 3, "hostname": 2, "hash": 6,
                                        "uuid": 9, "oid": 10, "cert_fp": 11}),
    "default": None,
}


@pytest.fixture(scope="module")
def weights():
    return synth.make_weights(DIMS, seed=2002, random_affine=True)


@pytest.fixture(scope="module")
def c1x(vocab_words):
    return synth.make_records(synth.C1X.records, vocab_words)


def test_table_matches_oracle_kinds():
    """The binding's kind order is the oracle's."""
    assert api.RX_KINDS == R.N_KINDS
    assert [api.RX_KIND[k] for k in R.KIND_NAMES] == list(range(R.N_KINDS))
    assert tuple(api.recognizer_table({"mac": 4, "ipv6": 1, "ipv4": 1, "cve": 3, "hostname": 2})) == R.DEFAULT_TYPES


@pytest.fixture(scope="module")
def c1x_ref(c1x, weights, vocab_index):
    return P.anonymize(c1x.records(), U.oracle_schema(SCHEMA), KEY, Encoder(DIMS, weights), vocab_index)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_c1x_parity(c1x, c1x_ref, weights, vocab_words, vocab_index, prec):
    ctx = api.Context(DIMS, synth.pack_blob(DIMS, weights), vocab_words, precision=prec, keep_trace=True)
    out = ctx.anonymize(c1x.data, c1x.offsets, SCHEMA, KEY)
    tr = ctx.trace()
    records = c1x.records()
    ref = c1x_ref
    U.check_tokens(tr, records, c1x.offsets, ref.traces)
    U.check_regex(tr, c1x.offsets, ref.traces)
    got_types = set(tr["regex_type"].tolist())
    assert got_types == {1, 2, 3, 4, 5, 6, 7, 9, 10, 11}
    err, agree, _ = U.check_logits(tr, ref.traces, prec)
    got = out.records()
    iso = U.check_stage_isolated(got, tr, records, SCHEMA, KEY, vocab_index)
    U.check_final_spans(tr, c1x.offsets, iso.traces)
    assert U.map_tuples(ctx.map_export()) == U.map_tuples(iso.map)
    same = 0
    for i, t in enumerate(ref.traces):
        if tr["labels"][U.split_tokens(tr, c1x.n)[i]].tolist() == t.labels:
            assert got[i] == t.output, f"record {i}: end-to-end output differs with equal labels"
            same += 1
    assert same >= 0.9 * c1x.n
    print(f"c1x {prec}: {len(tr['regex_start'])} recognizer spans, max|dlogit| {err:.2e}, agreement {agree:.5f}")
    out.free()
    ctx.close()


def _edge_records() -> list[bytes]:
    h32 = b"d41d8cd98f00b204e9800998ecf8427e"
    long_url = b"see https://a.example.com/" + b"/".join([b"seg%d" % k for k in range(150)]) + b"?x=" + h32 + b". end"
    pem_body = b"\n".join([b"QUJD" * 16] * 40 + [h32 + b"+" + b"MIIB" * 4])
    pem = b"-----BEGIN CERTIFICATE-----\n" + pem_body + b"\n-----END CERTIFICATE-----"
    return [
        long_url,                                   # > 512 bytes: resolve spans several steps
        b"x\n" + pem + b"\n10.0.0.1 after",         # PEM of ~2.7 KB with hash-like words inside
        pem,                                        # PEM at the record start
        b"cut http://",                             # scheme at the record end
        b"-----BEGIN CERTIFICATE-----\nAAAA",       # PEM without END: the next record's END does not count
        b"-----END CERTIFICATE----- 10.1.1.1",
        b"url http://host/?c=cpe:2.3:a:b:c:d:e:f:g:h:i:j:k done",
        b"cpe:2.3:a:b:c:d:e:f:g:h:i:j:k:extra.example.com",
        b"cpe:/a:apache:tomcat:9.0:.",
        b"",
        b"http://a.b",
        b"9" * 600 + b" 2001:db8::1",
    ]


@pytest.fixture(scope="module")
def fuzz_recs():
    rng = np.random.default_rng(2024)
    recs = [fuzz_record(rng, extended=True) for _ in range(6000)]
    recs += [fuzz_record(rng, extended=False) for _ in range(1000)]
    edges = _edge_records()
    # edge records interleaved so that neighbours share 16-byte words of the resolve pass
    out = []
    for i, r in enumerate(recs):
        out.append(r)
        if i % 500 == 0:
            out.extend(edges)
    return out


@pytest.mark.parametrize("table", list(TABLES))
def test_recognizer_fuzz(fuzz_recs, weights, vocab_words, table):
    rx = TABLES[table]
    ctx = api.Context(DIMS, synth.pack_blob(DIMS, weights), vocab_words, precision="fp32", keep_trace=True)
    rs = synth.records_from_list(fuzz_recs)
    schema = api.Schema(synth.TYPE_NAMES_11, recognizers=rx, window=512, stride=384)  # edge records exceed 512 tokens
    out = ctx.anonymize(rs.data, rs.offsets, schema, KEY)
    tr = ctx.trace()
    per = U.spans_by_record(tr["regex_start"], tr["regex_len"], tr["regex_type"], rs.offsets)
    n = 0
    for i, rec in enumerate(fuzz_recs):
        assert per[i] == R.recognize(rec, rx), f"record {i}: {rec[:120]!r}"
        n += len(per[i])
    assert n > 1000
    out.free()
    ctx.close()


def test_recognizer_table_validation(weights, vocab_words):
    ctx = api.Context(DIMS, synth.pack_blob(DIMS, weights), vocab_words, precision="fp32")
    rs = synth.records_from_list([b"10.0.0.1"])
    bad = api.recognizer_table({"url": 12})
    with pytest.raises(api.AnonShieldError, match="exceeds n_types"):
        ctx.anonymize(rs.data, rs.offsets, api.Schema(synth.TYPE_NAMES_11, recognizers=bad), KEY)
    with pytest.raises(ValueError):
        ctx.anonymize(rs.data, rs.offsets, api.Schema(synth.TYPE_NAMES_11, recognizers=(1, 2)), KEY)
    ctx.close()


def test_serving_and_streaming_carry_the_table(c1x, weights, vocab_words):
    """Served requests and the streamed batches use the schema's recognizer table."""
    ctx = api.Context(DIMS, synth.pack_blob(DIMS, weights), vocab_words, precision="bf16")
    recs = c1x.records()[:96]
    rs = synth.records_from_list(recs)
    want = ctx.anonymize(rs.data, rs.offsets, SCHEMA, KEY).records()
    assert any(b"[URL_" in w for w in want) and any(b"[CERTIFICATE_" in w for w in want)
    streamed = ctx.anonymize_stream(rs.data, rs.offsets, SCHEMA, KEY, batch_bytes=8192, lanes=2).records()
    assert streamed == want
    ctx.map_clear()
    ctx.serve_start(SCHEMA, KEY, lanes=2)
    try:
        ids = [ctx.submit(r) for r in recs]
        served = [ctx.poll(i, timeout_s=30.0) for i in ids]
    finally:
        ctx.serve_stop()
    assert served == want
    ctx.close()
