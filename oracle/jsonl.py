"""JSON Lines ingest (oracle): the fields of one JSON line; test infrastructure.

AnonShield reads JSON and JSONL inputs as streams and keeps their structure,
replacing only sensitive values (§2 stages (1) and (5)), with per-field
control through the schema-aware ``anonymization_config`` (§2). This project
reads a JSONL record as one line of text and turns it into the fields of the
per-field policy (``oracle/fields.py``):

* The line is well formed when it is one JSON value (RFC 8259) with optional
  white space (space, tab, LF, CR) around it, nested at most MAX_DEPTH
  containers deep. Strings hold no raw byte below 0x20; escapes are
  ``\\" \\\\ \\/ \\b \\f \\n \\r \\t`` and ``\\u`` with four hex digits; other
  bytes, UTF-8 or not, are taken as they are. Numbers follow the RFC grammar;
  the literals are ``true``, ``false`` and ``null``.
* Every string VALUE (object keys are structure) gives fields: the maximal
  runs of its raw bytes between the quotes that lie outside escape sequences
  (so a replacement never cuts an escape and the output stays valid JSON).
  Their id is the index of the innermost enclosing member's key in
  ``key_names`` (keys compared as raw bytes), ``len(key_names)`` when that
  key is not listed or the value is in no member (top-level value or array).
* A line that is not well formed is one field covering the whole line with
  id ``len(key_names) + 1``, which the caller maps to DETECT: text that
  cannot be parsed is scanned as free text rather than passed through.
* An empty or all-white-space line has no fields.
"""
from __future__ import annotations

MAX_DEPTH = 64
_WS = b" \t\n\r"
_ESC = set(b'"\\/bfnrt')
_HEX = set(b"0123456789abcdefABCDEF")
_DIG = set(b"0123456789")


class Malformed(Exception):
    pass


class _Scanner:
    def __init__(self, line: bytes, key_names: list[bytes]):
        self.s = line
        self.keys = key_names
        self.fields: list[tuple[int, int, int]] = []
        self.strings: list[tuple[int, int, int]] = []   # (raw start, raw end, id) of each string value

    def ws(self, i: int) -> int:
        while i < len(self.s) and self.s[i] in _WS:
            i += 1
        return i

    def string(self, i: int) -> tuple[int, list[tuple[int, int]]]:
        """Position after the string starting with the quote at i, and its runs outside escapes."""
        s = self.s
        i += 1
        runs, run0 = [], i
        while True:
            if i >= len(s):
                raise Malformed("unterminated string")
            c = s[i]
            if c == ord('"'):
                if i > run0:
                    runs.append((run0, i))
                return i + 1, runs
            if c < 0x20:
                raise Malformed("control byte in a string")
            if c == ord("\\"):
                if i > run0:
                    runs.append((run0, i))
                if i + 1 >= len(s):
                    raise Malformed("escape at the end")
                e = s[i + 1]
                if e == ord("u"):
                    if len(s) < i + 6 or any(h not in _HEX for h in s[i + 2:i + 6]):
                        raise Malformed("bad \\u escape")
                    i += 6
                elif e in _ESC:
                    i += 2
                else:
                    raise Malformed("bad escape")
                run0 = i
                continue
            i += 1

    def number(self, i: int) -> int:
        s = self.s
        j = i
        if j < len(s) and s[j] == ord("-"):
            j += 1
        if j < len(s) and s[j] == ord("0"):
            j += 1
        elif j < len(s) and s[j] in _DIG:
            while j < len(s) and s[j] in _DIG:
                j += 1
        else:
            raise Malformed("bad number")
        if j < len(s) and s[j] == ord("."):
            j += 1
            if not (j < len(s) and s[j] in _DIG):
                raise Malformed("bad fraction")
            while j < len(s) and s[j] in _DIG:
                j += 1
        if j < len(s) and s[j] in b"eE":
            j += 1
            if j < len(s) and s[j] in b"+-":
                j += 1
            if not (j < len(s) and s[j] in _DIG):
                raise Malformed("bad exponent")
            while j < len(s) and s[j] in _DIG:
                j += 1
        return j

    def value(self, i: int, fid: int, depth: int) -> int:
        s = self.s
        if i >= len(s):
            raise Malformed("value expected")
        c = s[i]
        if c == ord('"'):
            j, runs = self.string(i)
            self.strings.append((i + 1, j - 1, fid))
            self.fields += [(a, b - a, fid) for a, b in runs]
            return j
        if c == ord("{"):
            if depth + 1 > MAX_DEPTH:
                raise Malformed("too deep")
            i = self.ws(i + 1)
            if i < len(s) and s[i] == ord("}"):
                return i + 1
            while True:
                if i >= len(s) or s[i] != ord('"'):
                    raise Malformed("key expected")
                j, _ = self.string(i)
                raw = s[i + 1:j - 1]
                kid = self.keys.index(raw) if raw in self.keys else len(self.keys)
                i = self.ws(j)
                if i >= len(s) or s[i] != ord(":"):
                    raise Malformed("':' expected")
                i = self.value(self.ws(i + 1), kid, depth + 1)
                i = self.ws(i)
                if i < len(s) and s[i] == ord(","):
                    i = self.ws(i + 1)
                    continue
                if i < len(s) and s[i] == ord("}"):
                    return i + 1
                raise Malformed("',' or '}' expected")
        if c == ord("["):
            if depth + 1 > MAX_DEPTH:
                raise Malformed("too deep")
            i = self.ws(i + 1)
            if i < len(s) and s[i] == ord("]"):
                return i + 1
            while True:
                i = self.ws(self.value(i, fid, depth + 1))
                if i < len(s) and s[i] == ord(","):
                    i = self.ws(i + 1)
                    continue
                if i < len(s) and s[i] == ord("]"):
                    return i + 1
                raise Malformed("',' or ']' expected")
        for lit in (b"true", b"false", b"null"):
            if s[i:i + len(lit)] == lit:
                return i + len(lit)
        return self.number(i)


def scan_line(line: bytes, key_names: list[bytes]) -> tuple[list[tuple[int, int, int]], bool]:
    """(fields (start, length, id) in order, malformed) of one JSON line."""
    sc = _Scanner(line, key_names)
    i = sc.ws(0)
    if i == len(line):
        return [], False
    try:
        i = sc.ws(sc.value(i, len(key_names), 0))
        if i != len(line):
            raise Malformed("text after the value")
    except Malformed:
        return [(0, len(line), len(key_names) + 1)], True
    return sc.fields, False


def string_values(line: bytes, key_names: list[bytes]) -> list[tuple[int, int, int]]:
    """(raw start, raw end, id) of every string value of a well-formed line (for tests)."""
    sc = _Scanner(line, key_names)
    sc.ws(sc.value(sc.ws(0), len(key_names), 0))
    return sc.strings


def policy_ids(key_names: list[bytes]) -> tuple[int, int]:
    """(id of values under unlisted keys, id of malformed lines)."""
    return len(key_names), len(key_names) + 1


def anonymize_jsonl(records: list[bytes], key_names: list[bytes], actions: dict[int, tuple[int, int]],
                    default: int, schema, key: bytes, encoder, vocab, labels=None):
    """The per-field pipeline over the fields of each JSON line (``actions``: key index ->
    (action, force type); unlisted keys take ``default``, malformed lines DETECT)."""
    from . import fields as F
    unknown, bad = policy_ids(key_names)
    acts = dict(actions)
    acts[unknown] = (default, 0)
    acts[bad] = (F.DETECT, 0)
    pol = F.FieldPolicy(acts, default)
    flds = [scan_line(r, key_names)[0] for r in records]
    return F.anonymize_fields(records, flds, pol, schema, key, encoder, vocab, labels=labels)
