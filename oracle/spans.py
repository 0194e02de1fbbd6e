"""From token spans to the final entity spans of a record (oracle).

Readings (the paper leaves all three open):

* A token span [first, last] covers bytes [off(first), off(last) + len(last)).
  ASCII whitespace (0x09..0x0D, 0x20) is trimmed from both ends; a span left
  empty is dropped.
* Overlaps: pattern-recognizer spans win. Every NER span sharing at least one
  byte with a recognizer span is dropped. The paper's fast ``standalone``
  strategy has no overlap resolution and can truncate entities, e.g. leaving
  ``[IP_ADDRESS_...].1.72`` behind (Appendix D); this rule removes that.
* Preserve list: a span whose type bit (bit t of ``preserve_mask``) is set is
  dropped after the overlap rule, so its bytes pass through (the paper's
  ``--entities-to-preserve``, §2).
"""
from __future__ import annotations

_WS = {0x09, 0x0A, 0x0B, 0x0C, 0x0D, 0x20}


def token_span_to_bytes(data: bytes, offs: list[int], lens: list[int],
                        first: int, last: int) -> tuple[int, int] | None:
    s = offs[first]
    e = offs[last] + lens[last]
    while s < e and data[s] in _WS:
        s += 1
    while e > s and data[e - 1] in _WS:
        e -= 1
    if e <= s:
        return None
    return s, e


def ner_byte_spans(data: bytes, offs: list[int], lens: list[int],
                   token_spans: list[tuple[int, int, int]]) -> list[tuple[int, int, int]]:
    out = []
    for first, last, t in token_spans:
        r = token_span_to_bytes(data, offs, lens, first, last)
        if r is not None:
            out.append((r[0], r[1] - r[0], t))
    return out


def merge(regex_spans: list[tuple[int, int, int]], ner_spans: list[tuple[int, int, int]],
          preserve_mask: int = 0) -> list[tuple[int, int, int]]:
    """Final disjoint spans (start, length, type) sorted by start."""
    kept = []
    for s, n, t in ner_spans:
        e = s + n
        if any(s < rs + rn and rs < e for rs, rn, _ in regex_spans):
            continue
        kept.append((s, n, t))
    allspans = sorted(list(regex_spans) + kept)
    return [sp for sp in allspans if not (preserve_mask >> sp[2]) & 1]
