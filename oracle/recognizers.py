"""Pattern recognizers (oracle).

The paper combines its NER model with 21 custom patterns covering, among
others, IPv4/IPv6 addresses, URLs, host names, hashes, certificates and
CVE/CPE identifiers, and lists UUIDs and OIDs among its entity types
(§2 stages (2) and (5)); it does not print the patterns. This project
implements twelve recognizers, as plain character checks (no
regular-expression engine), under the following reading.

Words and word recognizers
* A word is a maximal run of bytes in ``[A-Za-z0-9.:-]``. Trailing ``.`` and
  ``-`` are stripped, and so is a trailing ``:`` unless it is the second
  colon of a final ``::`` (so ``fe80::`` stays an IPv6 address).
* A word yields at most one entity; the checks run in this order and the
  first that accepts the whole word wins (no matching inside a word):
  MAC, IPv6, IPv4 (optionally ``:port``), CVE, host name (optionally
  ``:port``), hash, UUID, certificate fingerprint, OID.
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
* Hash: 32, 40, 64 or 128 hex digits (MD5, SHA-1, SHA-256, SHA-512).
* UUID: hex groups of 8, 4, 4, 4 and 12 digits joined by ``-``.
* Certificate fingerprint: 16, 20 or 32 groups of two hex digits joined by
  ``:`` (MD5, SHA-1, SHA-256 fingerprints).
* OID: five or more decimal arcs joined by ``.``, no leading zeros, the first
  arc 0, 1 or 2, and the second at most 39 when the first is 0 or 1. (Four
  arcs would collide with IPv4 and three with version numbers.)

Recognizers that span several words. They are tried first, at the start of
a word run; the first that matches there wins:
* PEM certificate, only at the start of a line (record start or after
  ``\\n``): ``-----BEGIN CERTIFICATE-----``, then only base64 bytes
  ``[A-Za-z0-9+/=]`` and ASCII white space, then
  ``-----END CERTIFICATE-----``, which ends the span.
* URL: a scheme of 2..16 letters and digits beginning with a letter,
  ``://``, then the longest run of URL bytes (letters, digits and
  ``-._~:/?#[]@!$&*+,;=%``); trailing ``.,:;!?`` are stripped and at least
  one byte must remain after ``://``.
* CPE, formatted-string form: ``cpe:2.3:`` and eleven non-empty components
  of ``[A-Za-z0-9._~%!*?-]`` joined by ``:``; the first (part) is ``a``,
  ``o``, ``h``, ``*`` or ``-``; the span ends with the eleventh component,
  less trailing ``.``. URI form: ``cpe:/``, a part letter ``a``, ``o`` or
  ``h``, then up to six ``:``-prefixed components of ``[A-Za-z0-9._~%-]``
  (possibly empty); trailing ``.`` and ``:`` are stripped.

Resolution. Candidates are taken left to right, as a scanning regex engine
does: a candidate whose start lies inside an already accepted span is
dropped. Only the multi-word recognizers can cover another candidate.

Recognizers map to entity types through a table of twelve entries indexed
by kind (``KIND_*``; 0 switches a recognizer off). The default maps the
five address/CVE recognizers to 1 IP_ADDRESS (both IP families; the
paper's example prefix, §2 stage (3)), 2 HOSTNAME, 3 CVE_ID, 4 MAC_ADDRESS
and switches the rest off.
"""
from __future__ import annotations

IP_ADDRESS, HOSTNAME, CVE_ID, MAC_ADDRESS = 1, 2, 3, 4

# recognizer kinds (index into the kind -> entity type table)
(KIND_MAC, KIND_IPV6, KIND_IPV4, KIND_CVE, KIND_HOSTNAME, KIND_URL, KIND_HASH, KIND_UUID,
 KIND_CPE, KIND_OID, KIND_CERT_FP, KIND_PEM) = range(12)
N_KINDS = 12
KIND_NAMES = ("mac", "ipv6", "ipv4", "cve", "hostname", "url", "hash", "uuid", "cpe", "oid",
              "cert_fp", "pem")
DEFAULT_TYPES = (MAC_ADDRESS, IP_ADDRESS, IP_ADDRESS, CVE_ID, HOSTNAME, 0, 0, 0, 0, 0, 0, 0)

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


def is_hash(w: bytes) -> bool:
    return len(w) in (32, 40, 64, 128) and all(c in _HEX for c in w)


def is_uuid(w: bytes) -> bool:
    groups = w.split(b"-")
    if [len(g) for g in groups] != [8, 4, 4, 4, 12]:
        return False
    return all(c in _HEX for g in groups for c in g)


def is_cert_fingerprint(w: bytes) -> bool:
    groups = w.split(b":")
    if len(groups) not in (16, 20, 32):
        return False
    return all(len(g) == 2 and g[0] in _HEX and g[1] in _HEX for g in groups)


def is_oid(w: bytes) -> bool:
    arcs = w.split(b".")
    if len(arcs) < 5:
        return False
    for a in arcs:
        if len(a) == 0 or any(c not in _DIG for c in a):
            return False
        if len(a) > 1 and a[0] == ord("0"):
            return False
    first = int(arcs[0])
    if first > 2:
        return False
    return first == 2 or int(arcs[1]) <= 39


_B64 = _DIG | _ALPHA | set(b"+/=")
_SPACE = set(b"\t\n\v\f\r ")
_PEM_BEGIN = b"-----BEGIN CERTIFICATE-----"
_PEM_END = b"-----END CERTIFICATE-----"
_URL = _DIG | _ALPHA | set(b"-._~:/?#[]@!$&*+,;=%")
_URL_TRAIL = set(b".,:;!?")
_CPE_FS = _DIG | _ALPHA | set(b"._~%!*?-")
_CPE_URI = _DIG | _ALPHA | set(b"._~%-")


def pem_end(data: bytes, i: int) -> int:
    """End of a PEM certificate block starting at ``i``, else -1."""
    if not (i == 0 or data[i - 1] == ord("\n")):
        return -1
    if data[i:i + len(_PEM_BEGIN)] != _PEM_BEGIN:
        return -1
    j = i + len(_PEM_BEGIN)
    while j < len(data) and (data[j] in _B64 or data[j] in _SPACE):
        j += 1
    if data[j:j + len(_PEM_END)] != _PEM_END:
        return -1
    return j + len(_PEM_END)


def url_end(data: bytes, i: int) -> int:
    """End of a URL starting at ``i``, else -1."""
    j = i
    while j < len(data) and (data[j] in _ALPHA or data[j] in _DIG):
        j += 1
    if not (2 <= j - i <= 16) or data[i] not in _ALPHA or data[j:j + 3] != b"://":
        return -1
    body = j + 3
    e = body
    while e < len(data) and data[e] in _URL:
        e += 1
    while e > body and data[e - 1] in _URL_TRAIL:
        e -= 1
    return e if e > body else -1


def _run(data: bytes, j: int, allowed: set) -> int:
    while j < len(data) and data[j] in allowed:
        j += 1
    return j


def cpe_end(data: bytes, i: int) -> int:
    """End of a CPE name (formatted string or URI form) starting at ``i``, else -1."""
    if data[i:i + 8] == b"cpe:2.3:":
        j = i + 8
        for comp in range(11):
            if comp > 0:
                if j >= len(data) or data[j] != ord(":"):
                    return -1
                j += 1
            e = _run(data, j, _CPE_FS)
            if e == j:
                return -1
            if comp == 0 and data[j:e] not in (b"a", b"o", b"h", b"*", b"-"):
                return -1
            start_last, j = j, e
        while j > start_last + 1 and data[j - 1] == ord("."):
            j -= 1
        return j if data[j - 1] != ord(".") else -1
    if data[i:i + 5] == b"cpe:/" and i + 5 < len(data) and data[i + 5] in b"aoh":
        j = i + 6
        for _ in range(6):
            if j < len(data) and data[j] == ord(":"):
                j = _run(data, j + 1, _CPE_URI)
            else:
                break
        while data[j - 1] in b".:":
            j -= 1
        return j
    return -1


def _word_runs(data: bytes) -> list[tuple[int, int, int]]:
    """(run start, run end, stripped end) of each maximal run of word bytes."""
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
        out.append((i, j, end))
        i = j
    return out


def _word_match(w: bytes, types) -> tuple[int, int]:
    """(span length, type) of the first enabled word recognizer accepting ``w``, else (0, 0)."""
    checks = (
        (KIND_MAC, lambda: len(w) if is_mac(w) else 0),
        (KIND_IPV6, lambda: len(w) if is_ipv6(w) else 0),
        (KIND_IPV4, lambda: ipv4_len(w)),
        (KIND_CVE, lambda: len(w) if is_cve(w) else 0),
        (KIND_HOSTNAME, lambda: hostname_len(w)),
        (KIND_HASH, lambda: len(w) if is_hash(w) else 0),
        (KIND_UUID, lambda: len(w) if is_uuid(w) else 0),
        (KIND_CERT_FP, lambda: len(w) if is_cert_fingerprint(w) else 0),
        (KIND_OID, lambda: len(w) if is_oid(w) else 0),
    )
    for kind, check in checks:
        if types[kind]:
            n = check()
            if n > 0:
                return n, types[kind]
    return 0, 0


def candidates(data: bytes, types=None) -> list[tuple[int, int, int]]:
    """Every recognizer candidate (start, length, type), one per word run, before resolution."""
    types = DEFAULT_TYPES if types is None else tuple(types)
    assert len(types) == N_KINDS
    out = []
    for s, _, e in _word_runs(data):
        hit = None
        for kind, find in ((KIND_PEM, pem_end), (KIND_URL, url_end), (KIND_CPE, cpe_end)):
            if types[kind]:
                end = find(data, s)
                if end > s:
                    hit = (s, end - s, types[kind])
                    break
        if hit is None and e > s:
            n, t = _word_match(data[s:e], types)
            if n > 0:
                hit = (s, n, t)
        if hit is not None:
            out.append(hit)
    return out


def recognize(data: bytes, types=None) -> list[tuple[int, int, int]]:
    """Entity spans (start, length, type) of one record, in order of start.

    ``types`` is the kind -> entity type table (``N_KINDS`` entries, 0 = off);
    None selects ``DEFAULT_TYPES``."""
    spans = []
    kept_end = 0
    for s, n, t in candidates(data, types):
        if s < kept_end:
            continue
        spans.append((s, n, t))
        kept_end = s + n
    return spans
