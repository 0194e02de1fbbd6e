"""Per-field policy (oracle); test infrastructure, not part of the product path.

The schema-aware configuration of AnonShield §2 (``anonymization_config``:
``force_anonymize``, ``fields_to_anonymize``, ``fields_to_exclude``): a record
is a byte string with fields, (start, length, field id) spans inside it,
sorted and disjoint. Each field id has an action:

- DETECT: the field's bytes are a record of their own for every detection
  step (tokenizer, recognizers, encoder with windows, BIO decode, overlap
  rule, preserve list); the spans found are shifted by the field start.
- EXCLUDE: the field passes through unchanged and is never scanned.
- FORCE t: the field's value with ASCII whitespace (space, \\t \\n \\v \\f \\r)
  trimmed at both ends is one entity of type t, replaced whatever the
  preserve list says (force_anonymize); nothing when empty after trimming.

Bytes outside every field (separators, keys) pass through unchanged. The
record index of a map sighting is the record's index, as for whole records.
"""
from __future__ import annotations

from dataclasses import dataclass, field

from . import bio, recognizers, spans as spans_mod, tokenizer
from .encoder import Encoder, argmax_first, record_logits
from .pipeline import Result, Schema
from .pseudonym import export, substitute

DETECT, EXCLUDE, FORCE = 0, 1, 2
WS = b" \t\n\v\f\r"


@dataclass
class FieldPolicy:
    actions: dict[int, tuple[int, int]] = field(default_factory=dict)  # field id -> (action, force type)
    default: int = DETECT

    def of(self, fid: int) -> tuple[int, int]:
        return self.actions.get(fid, (self.default, 0))


def check_fields(data: bytes, fields: list[tuple[int, int, int]]) -> None:
    prev = 0
    for s, n, _ in fields:
        if s < prev or s + n > len(data):
            raise ValueError("fields must be sorted, disjoint and inside the record")
        prev = s + n


def detect_spans(sub: bytes, schema: Schema, encoder: Encoder, vocab: dict[bytes, int],
                 labels: list[int] | None = None) -> list[tuple[int, int, int]]:
    """Final spans of one detected field (its own record), relative to the field."""
    ids, offs, lens = tokenizer.tokenize(sub, vocab)
    regex = recognizers.recognize(sub, schema.recognizers)
    if labels is None:
        logits = record_logits(encoder, ids, schema.window, schema.stride)
        labels = argmax_first(logits).tolist() if len(ids) else []
    token_spans = bio.decode(list(labels))
    ner = spans_mod.ner_byte_spans(sub, offs, lens, token_spans)
    return spans_mod.merge(regex, ner, schema.preserve_mask)


def forced_span(sub: bytes, ftype: int) -> tuple[int, int, int] | None:
    a, b = 0, len(sub)
    while a < b and sub[a] in WS:
        a += 1
    while b > a and sub[b - 1] in WS:
        b -= 1
    return (a, b - a, ftype) if b > a else None


def record_spans(data: bytes, fields: list[tuple[int, int, int]], policy: FieldPolicy, schema: Schema,
                 encoder: Encoder | None, vocab: dict[bytes, int],
                 labels: list[list[int]] | None = None) -> list[tuple[int, int, int]]:
    """All spans of one record, sorted; ``labels`` (one list per detected field, in
    field order) replaces the encoder when given."""
    check_fields(data, fields)
    out = []
    k = 0
    for s, n, fid in fields:
        action, ftype = policy.of(fid)
        sub = data[s:s + n]
        if action == EXCLUDE:
            continue
        if action == FORCE:
            sp = forced_span(sub, ftype)
            if sp is not None:
                out.append((s + sp[0], sp[1], sp[2]))
            continue
        lab = None if labels is None else labels[k]
        k += 1
        out += [(s + a, m, t) for a, m, t in detect_spans(sub, schema, encoder, vocab, lab)]
    return sorted(out)


def anonymize_fields(records: list[bytes], fields: list[list[tuple[int, int, int]]], policy: FieldPolicy,
                     schema: Schema, key: bytes, encoder: Encoder | None, vocab: dict[bytes, int],
                     record_base: int = 0, emap: dict | None = None,
                     labels: list[list[list[int]]] | None = None) -> Result:
    """Pseudonymised records and map; ``labels[r]`` = per-detected-field label lists of record r."""
    emap = {} if emap is None else emap
    outs = []
    for r, data in enumerate(records):
        sp = record_spans(data, fields[r], policy, schema, encoder, vocab, None if labels is None else labels[r])
        outs.append(substitute(data, sp, key, list(schema.type_names), schema.slug_hex_len, record_base + r, emap))
    return Result(outs, export(emap), [], 0)
