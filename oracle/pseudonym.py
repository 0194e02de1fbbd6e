"""Pseudonyms, substitution and the entity map (oracle).

§2 stage (3): each entity is replaced by an HMAC-SHA256 slug under the
operator's key; the slug keeps 0..64 hex characters and the entity type is
kept as a prefix, as in 100.111.20.23 -> [IP_ADDRESS_48624b5cdc]. Reading:
the HMAC message is the entity's exact bytes (no type, no normalisation);
the slug is the first L lower-case hex characters of the digest (L = 10 by
default, odd L allowed); the replacement is ``[TYPE_slug]``, or ``[TYPE]``
when L = 0.

§2 stage (4): the entity <-> slug map records entity type, original name,
slug, full hash, first and last sighting. Here first_seen / last_seen are
record indices (a deterministic stand-in for timestamps) and each entry also
counts its occurrences. The map key is (type, original bytes). Export order
is type id, then original bytes in lexicographic byte order.

§2 stage (5): only the sensitive values are replaced; every other byte is
copied through unchanged.
"""
from __future__ import annotations

from dataclasses import dataclass

from .hmac_sha256 import hmac_sha256


@dataclass
class MapEntry:
    type: int
    original: bytes
    full_hash: str
    slug: str
    first_seen: int
    last_seen: int
    count: int


def replacement(type_name: str, digest: bytes, slug_len: int) -> tuple[bytes, str]:
    hexd = digest.hex()
    slug = hexd[:slug_len]
    if slug_len == 0:
        return f"[{type_name}]".encode(), slug
    return f"[{type_name}_{slug}]".encode(), slug


def substitute(data: bytes, spans: list[tuple[int, int, int]], key: bytes, type_names: list[str],
               slug_len: int, record_index: int, emap: dict[tuple[int, bytes], MapEntry]) -> bytes:
    """Output bytes of one record; updates ``emap`` with every replaced entity."""
    out = bytearray()
    prev = 0
    for s, n, t in spans:
        out += data[prev:s]
        ent = data[s:s + n]
        digest = hmac_sha256(key, ent)
        rep, slug = replacement(type_names[t - 1], digest, slug_len)
        out += rep
        prev = s + n
        k = (t, ent)
        e = emap.get(k)
        if e is None:
            emap[k] = MapEntry(t, ent, digest.hex(), slug, record_index, record_index, 1)
        else:
            e.first_seen = min(e.first_seen, record_index)
            e.last_seen = max(e.last_seen, record_index)
            e.count += 1
    out += data[prev:]
    return bytes(out)


def export(emap: dict[tuple[int, bytes], MapEntry]) -> list[MapEntry]:
    return [emap[k] for k in sorted(emap)]


def merge_maps(maps: list[list[MapEntry]]) -> list[MapEntry]:
    """Union of maps from shards of one job: min first_seen, max last_seen, summed count."""
    out: dict[tuple[int, bytes], MapEntry] = {}
    for m in maps:
        for e in m:
            k = (e.type, e.original)
            o = out.get(k)
            if o is None:
                out[k] = MapEntry(e.type, e.original, e.full_hash, e.slug, e.first_seen, e.last_seen, e.count)
            else:
                o.first_seen = min(o.first_seen, e.first_seen)
                o.last_seen = max(o.last_seen, e.last_seen)
                o.count += e.count
    return export(out)
