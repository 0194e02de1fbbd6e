"""Helpers for the GPU-vs-oracle parity tests (imported by test modules)."""
from __future__ import annotations

import numpy as np

from oracle import pipeline as P

TOL = {"fp32": 1e-4, "bf16": 2e-2, "fp8": 1e-1}
MARGIN = 0.05


def oracle_schema(s) -> P.Schema:
    rx = None if s.recognizers is None else tuple(s.recognizers)
    return P.Schema(tuple(s.type_names), s.preserve_mask, s.slug_hex_len, s.window, s.stride, rx)


def split_tokens(tr: dict, n: int) -> list[slice]:
    rt = tr["rec_tok"].astype(np.int64)
    return [slice(int(rt[i]), int(rt[i + 1])) for i in range(n)]


def check_tokens(tr: dict, recs: list[bytes], offsets: np.ndarray, ref_traces, idx=None):
    """Token ids, byte offsets and lengths equal the oracle's, record by record (bit-exact)."""
    sl = split_tokens(tr, len(offsets) - 1)
    idx = range(len(recs)) if idx is None else idx
    for i in idx:
        rt = ref_traces[i]
        s = sl[i]
        assert tr["tok_ids"][s].tolist() == rt.ids, f"record {i}: token ids"
        assert (tr["tok_off"][s].astype(np.int64) - int(offsets[i])).tolist() == rt.offs, f"record {i}: offsets"
        assert tr["tok_len"][s].tolist() == rt.lens, f"record {i}: lengths"


def spans_by_record(starts, lens, types, offsets: np.ndarray) -> list[list[tuple[int, int, int]]]:
    n = len(offsets) - 1
    out = [[] for _ in range(n)]
    rec = np.searchsorted(offsets.astype(np.int64), starts.astype(np.int64), side="right") - 1
    for s, l, t, r in zip(starts.tolist(), lens.tolist(), types.tolist(), rec.tolist()):
        out[r].append((s - int(offsets[r]), l, t))
    return out


def check_regex(tr: dict, offsets: np.ndarray, ref_traces, idx=None):
    per = spans_by_record(tr["regex_start"], tr["regex_len"], tr["regex_type"], offsets)
    idx = range(len(ref_traces)) if idx is None else idx
    for i in idx:
        assert per[i] == ref_traces[i].regex, f"record {i}: recognizer spans"


def check_logits(tr: dict, ref_traces, prec: str, idx=None):
    """Max-abs logit error within the stated tolerance; label agreement on confident tokens."""
    sl = split_tokens(tr, len(tr["rec_tok"]) - 1)
    idx = range(len(ref_traces)) if idx is None else idx
    errs, agree, conf, flips = [], 0, 0, []
    for i in idx:
        ref = ref_traces[i].logits
        if ref is None or len(ref) == 0:
            continue
        got = tr["logits"][sl[i]].astype(np.float64)
        errs.append(np.max(np.abs(got - ref)))
        srt = np.sort(ref, axis=1)
        margin = srt[:, -1] - srt[:, -2]
        lab = tr["labels"][sl[i]].astype(np.int64)
        ref_lab = np.argmax(ref, axis=1)
        # the label is the argmax of the kernel's own logits, lowest label on ties
        assert np.array_equal(lab, np.argmax(tr["logits"][sl[i]], axis=1)), f"record {i}: label != argmax"
        c = margin > MARGIN
        conf += int(c.sum())
        agree += int((lab[c] == ref_lab[c]).sum())
        for t in np.nonzero(lab != ref_lab)[0]:
            flips.append(float(margin[t]))
    err = max(errs) if errs else 0.0
    assert err <= TOL[prec], f"{prec} logits max abs error {err} > {TOL[prec]}"
    assert conf == 0 or agree / conf >= 0.999, f"label agreement {agree / conf:.5f} < 99.9%"
    # a label can only flip where the two top logits are within twice the error
    assert all(m <= 2 * err + 1e-12 for m in flips), f"label flip at margin {max(flips)} > 2 x {err}"
    return err, (agree / conf if conf else 1.0), len(flips)


def gpu_labels_per_record(tr: dict, n: int) -> list[list[int]]:
    return [tr["labels"][s].tolist() for s in split_tokens(tr, n)]


def check_stage_isolated(out_records: list[bytes], tr: dict, recs: list[bytes], schema, key: bytes, vocab_index,
                         record_base: int = 0, idx=None):
    """The oracle's decode/merge/HMAC/substitute fed the GPU's labels gives the GPU's bytes."""
    labels = gpu_labels_per_record(tr, len(recs))
    if idx is not None:
        sub = list(idx)
        res = P.anonymize_from_labels([recs[i] for i in sub], [labels[i] for i in sub], oracle_schema(schema), key,
                                      vocab_index, record_base=record_base)
        for j, i in enumerate(sub):
            assert out_records[i] == res.outputs[j], f"record {i}: output bytes differ"
        return res
    res = P.anonymize_from_labels(recs, labels, oracle_schema(schema), key, vocab_index, record_base=record_base)
    for i, (a, b) in enumerate(zip(out_records, res.outputs)):
        assert a == b, f"record {i}: output bytes differ\nGPU:    {a[:200]!r}\noracle: {b[:200]!r}"
    return res


def check_final_spans(tr: dict, offsets: np.ndarray, iso_traces, idx=None):
    per = spans_by_record(tr["final_start"], tr["final_len"], tr["final_type"], offsets)
    idx = range(len(iso_traces)) if idx is None else idx
    for j, i in enumerate(idx):
        assert per[i] == iso_traces[j].final, f"record {i}: final spans"


def map_tuples(entries) -> list[tuple]:
    return [(e.type, e.original, e.full_hash, e.first_seen, e.last_seen, e.count) for e in entries]


def oracle_logits(enc, records: list[bytes], vocab_index, window: int = 0, stride: int = 0) -> list[np.ndarray]:
    """Per-record logits of the oracle's encoder on the oracle's own tokens."""
    from oracle.encoder import record_logits
    from oracle.tokenizer import tokenize
    return [record_logits(enc, tokenize(r, vocab_index)[0], window, stride) for r in records]


def logit_stats(tr: dict, n: int, ref: list[np.ndarray], idx=None) -> dict:
    """Max / rms |logit error| of the GPU trace against reference logits per record, and
    the label agreement over tokens whose reference top-2 margin exceeds MARGIN."""
    sl = split_tokens(tr, n)
    idx = range(len(ref)) if idx is None else idx
    errs, conf, agree, flips = [], 0, 0, []
    for j, i in enumerate(idx):
        r = ref[j]
        if len(r) == 0:
            continue
        g = tr["logits"][sl[i]].astype(np.float64)
        assert g.shape == r.shape, f"record {i}: {g.shape} logits vs {r.shape}"
        errs.append(np.abs(g - r).ravel())
        srt = np.sort(r, axis=1)
        margin = srt[:, -1] - srt[:, -2]
        lab, rl = tr["labels"][sl[i]].astype(np.int64), np.argmax(r, axis=1)
        c = margin > MARGIN
        conf += int(c.sum())
        agree += int((lab[c] == rl[c]).sum())
        flips += [float(m) for m in margin[lab != rl]]
    e = np.concatenate(errs) if errs else np.zeros(1)
    return {"max": float(e.max()), "rms": float(np.sqrt(np.mean(e ** 2))), "tokens": int(e.size // ref[0].shape[1]),
            "agreement": agree / conf if conf else 1.0, "confident": conf, "flips": flips}


def logit_stats_ref(a: list[np.ndarray], b: list[np.ndarray]) -> dict:
    """Max / rms |a - b| and label agreement of a against b (b's top-2 margin > MARGIN), oracle vs oracle."""
    e = np.concatenate([np.abs(x - y).ravel() for x, y in zip(a, b) if len(y)])
    conf = agree = 0
    for x, y in zip(a, b):
        if not len(y):
            continue
        srt = np.sort(y, axis=1)
        c = (srt[:, -1] - srt[:, -2]) > MARGIN
        conf += int(c.sum())
        agree += int((np.argmax(x, axis=1)[c] == np.argmax(y, axis=1)[c]).sum())
    return {"max": float(e.max()), "rms": float(np.sqrt(np.mean(e ** 2))), "agreement": agree / conf if conf else 1.0}
