"""BIO label decoding (oracle).

The NER model tags tokens (§2 stage (2)); the paper does not say how tags
become entities. Reading used here, label ids first:

* label 0 is O; for entity type t = 1..K, label 2t-1 is B-t and label 2t is
  I-t (nine labels for four types, seventeen for eight);
* decoding is lenient: a span starts at B-t, or at I-t whose predecessor is
  neither B-t nor I-t; it goes on while the next label is I-t; B-t always
  starts a new span and O ends one.
"""
from __future__ import annotations


def label_type(label: int) -> tuple[int, bool]:
    """(type, is_begin) of a label; type 0 for O."""
    if label == 0:
        return 0, False
    return (label + 1) // 2, (label % 2) == 1


def decode(labels: list[int]) -> list[tuple[int, int, int]]:
    """Token spans (first, last, type) of one sequence of labels, in order."""
    spans: list[tuple[int, int, int]] = []
    cur_t = 0
    cur_first = 0
    for i, lab in enumerate(labels):
        t, begin = label_type(lab)
        if t == 0:
            if cur_t:
                spans.append((cur_first, i - 1, cur_t))
            cur_t = 0
            continue
        if begin or t != cur_t:
            if cur_t:
                spans.append((cur_first, i - 1, cur_t))
            cur_t, cur_first = t, i
        # else: I-t continuing a span of type t
    if cur_t:
        spans.append((cur_first, len(labels) - 1, cur_t))
    return spans
