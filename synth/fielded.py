"""Seeded CSV-like scan records with fields (inputs for the per-field policy).

One record per line of a scan export: columns host address | host name | port |
plugin id | severity | plugin name | description | solution | plugin output,
separated by " | ". Descriptions and solutions are boilerplate text of the
lexicon; the plugin output carries the planted entities at the workload's
density. Field i of a record is column i (the separators are outside every
field). Holds none of the method's arithmetic: it only lays out bytes.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import lexicon as lx
from .records import RecordSet, _Gen, _target_lengths
from .workloads import RecordShape

COLUMNS = ("host_ip", "host_name", "port", "plugin_id", "severity", "plugin_name", "description", "solution",
           "plugin_output")
SEP = b" | "


@dataclass
class FieldedRecords:
    records: RecordSet
    start: np.ndarray   # uint64, absolute byte offset of each field in the arena
    length: np.ndarray  # uint32
    field_id: np.ndarray  # uint32 (column index)

    def fields_of(self, r: int) -> list[tuple[int, int, int]]:
        """Fields of record r relative to the record start (start, length, id)."""
        a, b = int(self.records.offsets[r]), int(self.records.offsets[r + 1])
        lo = int(np.searchsorted(self.start, a, side="left"))
        hi = int(np.searchsorted(self.start, b, side="left"))
        return [(int(self.start[k]) - a, int(self.length[k]), int(self.field_id[k])) for k in range(lo, hi)]


def _text(g: _Gen, n_tok: int, ent_per_1k: float) -> bytes:
    r = g.rng
    out = bytearray()
    used = 0
    n_ent = int(g._np_rng.poisson(ent_per_1k * n_tok / 1000.0))
    slots = sorted(int(r.integers(0, max(n_tok, 1))) for _ in range(n_ent))
    si = 0
    while used < n_tok:
        if si < len(slots) and used >= slots[si]:
            si += 1
            e = g.entity()[0]
            piece = b" " + g.word() + b" " + e
        else:
            piece = b" " + g.word()
        out += piece
        used += g.est(piece)
    return bytes(out[1:])


def make_fielded_records(shape: RecordShape, vocab_words: list[bytes], seed: int = 1001) -> FieldedRecords:
    rng = np.random.default_rng(seed)
    targets = _target_lengths(rng, shape)
    g = _Gen(rng, vocab_words, shape)
    chunks, starts, lens, ids = [], [], [], []
    offsets = np.zeros(shape.n_records + 1, dtype=np.uint64)
    pos = 0
    for ri in range(shape.n_records):
        t = int(targets[ri])
        r = g.rng
        cols = [
            g.ipv4(),
            g.hostname(),
            str(int(r.choice((22, 25, 53, 80, 443, 445, 3306, 5432, 8080)))).encode(),
            str(int(r.integers(10000, 200000))).encode(),
            lx.SEVERITIES[int(r.integers(len(lx.SEVERITIES)))].encode(),
            _text(g, 6, 0.0),
            _text(g, max(4, int(0.3 * t)), 0.0),
            _text(g, max(4, int(0.2 * t)), 0.0),
            _text(g, max(4, int(0.45 * t)), shape.entities_per_1k * 2.0),
        ]
        rec = bytearray()
        for i, c in enumerate(cols):
            if i:
                rec += SEP
            starts.append(pos + len(rec))
            lens.append(len(c))
            ids.append(i)
            rec += c
        chunks.append(bytes(rec))
        pos += len(rec)
        offsets[ri + 1] = pos
    data = np.frombuffer(b"".join(chunks), dtype=np.uint8).copy()
    rs = RecordSet(data=data, offsets=offsets, planted=np.zeros((0, 4), np.int64), target_tokens=targets)
    return FieldedRecords(rs, np.array(starts, np.uint64), np.array(lens, np.uint32), np.array(ids, np.uint32))


JSONL_KEYS = ("host_ip", "host_name", "port", "plugin_id", "severity", "plugin_name", "description", "solution",
              "plugin_output", "mac", "os", "tags", "cves", "asset", "note")


def make_jsonl_records(shape: RecordShape, vocab_words: list[bytes], seed: int = 1001) -> RecordSet:
    """Scan findings as JSON Lines: one JSON object per record (no trailing newline).

    Members: the nine columns of the CSV-like records (port and plugin id as
    numbers), a nested "asset" object with "mac", "os" and a "tags" array, a
    "cves" array, and sometimes a "note" holding escapes (\\n, \\", \\u00e9) or
    raw UTF-8. Lines are written by ``json.dumps`` (key order kept), so they
    are well formed; a few (one in 50) are cut short to exercise malformed lines.
    """
    import json
    rng = np.random.default_rng(seed)
    targets = _target_lengths(rng, shape)
    g = _Gen(rng, vocab_words, shape)
    lines = []
    for ri in range(shape.n_records):
        t = int(targets[ri])
        r = g.rng
        cves = [g.cve().decode() for _ in range(int(r.integers(0, 4)))]
        obj = {
            "host_ip": g.ipv4().decode(),
            "host_name": g.hostname().decode(),
            "port": int(r.choice((22, 25, 53, 80, 443, 445, 3306, 5432, 8080))),
            "plugin_id": int(r.integers(10000, 200000)),
            "severity": lx.SEVERITIES[int(r.integers(len(lx.SEVERITIES)))],
            "plugin_name": _text(g, 6, 0.0).decode(),
            "description": _text(g, max(4, int(0.25 * t)), 0.0).decode(),
            "solution": _text(g, max(4, int(0.15 * t)), 0.0).decode(),
            "plugin_output": _text(g, max(4, int(0.4 * t)), shape.entities_per_1k * 2.0).decode(),
            "asset": {"mac": g.mac().decode(), "os": lx.SERVICES[int(r.integers(len(lx.SERVICES)))],
                      "tags": [g.word().decode() for _ in range(int(r.integers(0, 3)))]},
            "cves": cves,
        }
        k = int(r.integers(6))
        if k == 0:
            obj["note"] = "line one\nline \"two\" at " + g.ipv4().decode() + " café"
        elif k == 1:
            obj["note"] = None
        line = json.dumps(obj, ensure_ascii=bool(r.integers(2))).encode()
        if int(r.integers(50)) == 0:
            line = line[:int(r.integers(1, len(line)))]
        lines.append(line)
    offsets = np.zeros(len(lines) + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum([len(x) for x in lines], dtype=np.uint64)
    data = np.frombuffer(b"".join(lines), dtype=np.uint8).copy()
    return RecordSet(data=data, offsets=offsets, planted=np.zeros((0, 4), np.int64), target_tokens=targets)
