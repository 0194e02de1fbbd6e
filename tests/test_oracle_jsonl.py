"""Pins for the oracle's JSON Lines scanner.

Independent of its hand-written parser: Python's ``json`` module decides
which lines are well formed and gives every string value with its innermost
member key, in document order; each string the scanner reports must decode
(with ``json``) to that value under that key's id, and its fields must be
exactly the raw bytes outside escape sequences, found here by an ``re``
pattern. Malformed lines are mutations of well-formed ones.
"""
import json
import re

import numpy as np
import pytest

import synth
from oracle import jsonl as J

KEYS = [k.encode() for k in synth.JSONL_KEYS]
ESC_RE = re.compile(rb'\\(?:u[0-9a-fA-F]{4}|["\\/bfnrt])')


def _no_constants(x):
    raise ValueError(x)


def json_ok(line: bytes) -> bool:
    try:
        json.loads(line.decode("utf-8"), parse_constant=_no_constants)
        return True
    except (ValueError, UnicodeDecodeError):
        return False


class _Obj(list):
    """An object's members as a list of pairs (duplicate keys kept)."""


def json_tree(line: bytes):
    return json.loads(line.decode("utf-8"), object_pairs_hook=_Obj, parse_constant=_no_constants)


def json_strings(node, key=None, out=None):
    """(innermost member key, decoded string) of every string value, in document order."""
    out = [] if out is None else out
    if isinstance(node, str):
        out.append((key, node))
    elif isinstance(node, _Obj):
        for k, v in node:
            json_strings(v, k, out)
    elif isinstance(node, list):
        for v in node:
            json_strings(v, key, out)
    return out


def check_line(line: bytes):
    fields, bad = J.scan_line(line, KEYS)
    if line.strip(b" \t\n\r") == b"":
        assert fields == [] and not bad
        return
    assert bad == (not json_ok(line)), line
    if bad:
        assert fields == [(0, len(line), len(KEYS) + 1)]
        return
    strings = J.string_values(line, KEYS)
    want = json_strings(json_tree(line))
    assert len(strings) == len(want)
    expect_fields = []
    for (a, b, fid), (k, v) in zip(strings, want):
        assert json.loads(b'"' + line[a:b] + b'"') == v
        kb = None if k is None else k.encode("utf-8")
        assert fid == (KEYS.index(kb) if kb in KEYS else len(KEYS))
        pos = a
        for m in ESC_RE.finditer(line, a, b):
            if m.start() > pos:
                expect_fields.append((pos, m.start() - pos, fid))
            pos = m.end()
        if b > pos:
            expect_fields.append((pos, b - pos, fid))
    assert fields == expect_fields


@pytest.fixture(scope="module")
def lines(vocab_words):
    rs = synth.make_jsonl_records(synth.scaled(synth.C1, 300).records, vocab_words)
    return rs.records()


def test_generated_lines(lines):
    bad = 0
    for line in lines:
        check_line(line)
        bad += J.scan_line(line, KEYS)[1]
    assert 0 < bad < len(lines) // 10


CASES = [b'{}', b'[]', b' {"a": "x"} ', b'"top"', b'42', b'-0.5e+3', b'true', b'null', b'[1, "two", {"note": "3"}]',
         b'{"host_ip": "10.0.0.1", "asset": {"mac": "aa:bb:cc:dd:ee:ff", "tags": ["x", "y\\n"]}}',
         b'{"note": "a\\u00e9b\\"c\\\\"}', b'{"note": "\\ud83d\\ude00"}', b'{"k": ""}',
         b'{"a" "b"}', b'{"a": }', b'{"a": 1,}', b'[1 2]', b'{"a": 01}', b'{"a": 1.}', b'{"a": .5}', b'{"a": tru}',
         b'{"a": "x\\q"}', b'{"a": "x\\u12"}', b'{"a": "\x01"}', b'{"a": "x"} extra', b'{"a": "x"', b'"',
         b'{"a": NaN}', b'{"a": [1, 2]]', b'', b'   ', b'{"host_name":"a","host_name":"b"}']


@pytest.mark.parametrize("line", CASES)
def test_hand_cases(line):
    check_line(line)


def test_depth_limit():
    ok = b"[" * J.MAX_DEPTH + b'"x"' + b"]" * J.MAX_DEPTH
    deep = b"[" + ok + b"]"
    assert J.scan_line(ok, KEYS) == ([(J.MAX_DEPTH + 1, 1, len(KEYS))], False)
    assert J.scan_line(deep, KEYS)[1]


def test_mutations(lines):
    rng = np.random.default_rng(5)
    alphabet = b'{}[]":,\\ unt0123456789.-eE+aflsr\n\x01'
    n_bad = 0
    for _ in range(3000):
        line = bytearray(lines[int(rng.integers(len(lines)))][:300])
        for _ in range(int(rng.integers(1, 4))):
            i = int(rng.integers(len(line) + 1))
            op = int(rng.integers(3))
            c = alphabet[int(rng.integers(len(alphabet)))]
            if op == 0 and i < len(line):
                del line[i]
            elif op == 1:
                line.insert(i, c)
            elif i < len(line):
                line[i] = c
        line = bytes(line)
        try:
            line.decode("utf-8")
        except UnicodeDecodeError:
            continue
        check_line(line)
        n_bad += J.scan_line(line, KEYS)[1]
    assert n_bad > 1000
