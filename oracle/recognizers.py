"""Pattern recognizers (oracle).

The paper combines its NER model with 21 custom patterns covering, among
others, IPv4/IPv6 addresses, host names and CVE identifiers (§2 stage (2)),
and does not print them. This project implements five, as plain character
checks (no regular-expression engine), under the following reading:

* A word is a maximal run of bytes in ``[A-Za-z0-9.:-]``. Trailing ``.`` and
  ``-`` are stripped, and so is a trailing ``:`` unless it is the second
  colon of a final ``::`` (so ``fe80::`` stays an IPv6 address).
* Each word yields at most one entity; the checks run in this order and the
  first that accepts the whole word wins (no matching inside a word):
  MAC, IPv6, IPv4 (optionally ``:port``), CVE, host name (optionally ``:port``).
  A port is ``:`` and 1..5 digits and is left out of the entity span.
* MAC: six groups of two hex digits joined by one separator used throughout,
  ``:`` or ``-``.
* IPv6: groups of 1..4 hex digits separated by ``:``; either exactly eight
  groups and no ``::``, or exactly one ``::`` and at most seven groups. No
  embedded IPv4, no zone id.
* IPv4: four decimal octets 0..255, no leading zeros (``0`` alone is fine).
* CVE: ``CVE-`` (upper case), four digits, ``-``, four or more digits.
* Host name: two or more labels of 1..63 bytes from ``[A-Za-z0-9-]`` that
  neither start nor end with ``-``, the last label all letters and at least
  two long, at most 253 bytes in all.

Entity type ids: 1 IP_ADDRESS (both IP families; the paper's example prefix,
§2 stage (3)), 2 HOSTNAME, 3 CVE_ID, 4 MAC_ADDRESS.
"""
from __future__ import annotations

IP_ADDRESS, HOSTNAME, CVE_ID, MAC_ADDRESS = 1, 2, 3, 4

_HEX = set(b"0123456789abcdefABCDEF")
_DIG = set(b"0123456789")
_ALPHA = set(b"ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz")
_WORD = _HEX | _DIG | _ALPHA | set(b".:-")
_LABEL = _DIG | _ALPHA | {ord("-")}


def words(data: bytes) -> list[tuple[int, int]]:
    """(start, end) of each word after stripping its trailing punctuation."""
    out = []
    n = len(data)
    i = 0
    while i < n:
        if data[i] not in _WORD:
            i += 1
            continue
        j = i
        while j < n and data[j] in _WORD:
            j += 1
        end = j
        while end > i:
            c = data[end - 1]
            if c == ord(".") or c == ord("-"):
                end -= 1
            elif c == ord(":") and not (end - 2 >= i and data[end - 2] == ord(":")):
                end -= 1
            else:
                break
        if end > i:
            out.append((i, end))
        i = j
    return out


def is_mac(w: bytes) -> bool:
    if len(w) != 17:
        return False
    sep = w[2]
    if sep not in (ord(":"), ord("-")):
        return False
    for g in range(6):
        if w[3 * g] not in _HEX or w[3 * g + 1] not in _HEX:
            return False
        if g < 5 and w[3 * g + 2] != sep:
            return False
    return True


def _hex_groups(part: bytes) -> int:
    """Number of groups in a ':'-separated run of 1..4-hex-digit groups, -1 if invalid.

    An empty part has zero groups."""
    if len(part) == 0:
        return 0
    groups = part.split(b":")
    for g in groups:
        if not (1 <= len(g) <= 4) or any(c not in _HEX for c in g):
            return -1
    return len(groups)


def is_ipv6(w: bytes) -> bool:
    if ord(":") not in w:
        return False
    k = w.count(b"::")
    if k == 0:
        return _hex_groups(w) == 8
    if k != 1 or b":::" in w:
        return False
    left, right = w.split(b"::")
    nl, nr = _hex_groups(left), _hex_groups(right)
    if nl < 0 or nr < 0:
        return False
    return nl + nr <= 7


def _is_octet(s: bytes) -> bool:
    if not (1 <= len(s) <= 3) or any(c not in _DIG for c in s):
        return False
    if len(s) > 1 and s[0] == ord("0"):
        return False
    return int(s) <= 255


def _port_len(w: bytes, at: int) -> int:
    """Length of a ':' + 1..5 digits suffix that starts at ``at`` and ends the word, else -1."""
    rest = w[at:]
    if len(rest) == 0:
        return 0
    if rest[0] != ord(":") or not (2 <= len(rest) <= 6) or any(c not in _DIG for c in rest[1:]):
        return -1
    return len(rest)


def ipv4_len(w: bytes) -> int:
    """Span length of an IPv4 address (port excluded) filling the word, else 0."""
    c = w.find(b":")
    core = w if c < 0 else w[:c]
    parts = core.split(b".")
    if len(parts) != 4 or not all(_is_octet(p) for p in parts):
        return 0
    return len(core) if _port_len(w, len(core)) >= 0 else 0


def is_cve(w: bytes) -> bool:
    if len(w) < 13 or w[:4] != b"CVE-":
        return False
    if any(c not in _DIG for c in w[4:8]) or w[8] != ord("-"):
        return False
    tail = w[9:]
    return len(tail) >= 4 and all(c in _DIG for c in tail)


def hostname_len(w: bytes) -> int:
    """Span length of a host name (port excluded) filling the word, else 0."""
    c = w.find(b":")
    core = w if c < 0 else w[:c]
    if _port_len(w, len(core)) < 0:
        return 0
    if len(core) > 253:
        return 0
    labels = core.split(b".")
    if len(labels) < 2:
        return 0
    for lab in labels:
        if not (1 <= len(lab) <= 63) or any(ch not in _LABEL for ch in lab):
            return 0
        if lab[0] == ord("-") or lab[-1] == ord("-"):
            return 0
    last = labels[-1]
    if len(last) < 2 or any(ch not in _ALPHA for ch in last):
        return 0
    return len(core)


def recognize(data: bytes) -> list[tuple[int, int, int]]:
    """Entity spans (start, length, type) of one record, in order of start."""
    spans = []
    for s, e in words(data):
        w = data[s:e]
        if is_mac(w):
            spans.append((s, e - s, MAC_ADDRESS))
        elif is_ipv6(w):
            spans.append((s, e - s, IP_ADDRESS))
        elif (n := ipv4_len(w)) > 0:
            spans.append((s, n, IP_ADDRESS))
        elif is_cve(w):
            spans.append((s, e - s, CVE_ID))
        elif (n := hostname_len(w)) > 0:
            spans.append((s, n, HOSTNAME))
    return spans
