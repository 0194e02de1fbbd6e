"""The whole call, record by record (oracle).

anonymize(records, schema, key) -> pseudonymised records + entity map, the
problem statement of §2 (stages (2)-(5)): tokenize, run the pattern
recognizers, tag tokens with the encoder, decode BIO labels, resolve
overlaps, drop preserved types, then replace each entity with its keyed
pseudonym and record it in the map. Records are independent except for the
map; record index = ``record_base`` + position in the call.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import bio, recognizers, spans as spans_mod, tokenizer
from .encoder import Encoder, argmax_first, encoded_tokens, record_logits
from .pseudonym import MapEntry, export, substitute


@dataclass
class Schema:
    type_names: tuple[str, ...]
    preserve_mask: int = 0
    slug_hex_len: int = 10
    window: int = 0
    stride: int = 0
    recognizers: tuple[int, ...] | None = None   # kind -> entity type (None: the default five)


@dataclass
class RecordTrace:
    ids: list[int]
    offs: list[int]
    lens: list[int]
    regex: list[tuple[int, int, int]]
    logits: np.ndarray | None
    labels: list[int]
    ner_token_spans: list[tuple[int, int, int]]
    ner_spans: list[tuple[int, int, int]]
    final: list[tuple[int, int, int]]
    output: bytes


@dataclass
class Result:
    outputs: list[bytes]
    map: list[MapEntry]
    traces: list[RecordTrace] = field(default_factory=list)
    encoded_tokens: int = 0


def _finish(data: bytes, ids, offs, lens, regex, logits, labels, schema: Schema, key: bytes,
            record_index: int, emap) -> RecordTrace:
    tspans = bio.decode(list(labels))
    nspans = spans_mod.ner_byte_spans(data, offs, lens, tspans)
    final = spans_mod.merge(regex, nspans, schema.preserve_mask)
    out = substitute(data, final, key, list(schema.type_names), schema.slug_hex_len, record_index, emap)
    return RecordTrace(ids, offs, lens, regex, logits, list(labels), tspans, nspans, final, out)


def anonymize(records: list[bytes], schema: Schema, key: bytes, encoder: Encoder,
              vocab: dict[bytes, int], record_base: int = 0,
              emap: dict | None = None, keep_traces: bool = True) -> Result:
    emap = {} if emap is None else emap
    outs, traces = [], []
    n_enc = 0
    for i, data in enumerate(records):
        ids, offs, lens = tokenizer.tokenize(data, vocab)
        regex = recognizers.recognize(data, schema.recognizers)
        logits = record_logits(encoder, ids, schema.window, schema.stride)
        labels = argmax_first(logits).tolist() if len(ids) else []
        n_enc += encoded_tokens(len(ids), schema.window, schema.stride)
        tr = _finish(data, ids, offs, lens, regex, logits, labels, schema, key, record_base + i, emap)
        outs.append(tr.output)
        if keep_traces:
            traces.append(tr)
    return Result(outs, export(emap), traces, n_enc)


def anonymize_from_labels(records: list[bytes], labels: list[list[int]], schema: Schema, key: bytes,
                          vocab: dict[bytes, int], record_base: int = 0,
                          emap: dict | None = None) -> Result:
    """Every step after the encoder, fed a given label stream (one list per record)."""
    emap = {} if emap is None else emap
    outs, traces = [], []
    for i, data in enumerate(records):
        ids, offs, lens = tokenizer.tokenize(data, vocab)
        if len(labels[i]) != len(ids):
            raise ValueError(f"record {i}: {len(labels[i])} labels for {len(ids)} tokens")
        regex = recognizers.recognize(data, schema.recognizers)
        tr = _finish(data, ids, offs, lens, regex, None, labels[i], schema, key, record_base + i, emap)
        outs.append(tr.output)
        traces.append(tr)
    return Result(outs, export(emap), traces, 0)
