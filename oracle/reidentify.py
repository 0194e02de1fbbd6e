"""Controlled re-identification (oracle).

The paper keeps the entity <-> slug mapping (type, original, slug, full hash,
first / last seen) so that an administrator holding both the database and
the HMAC key can reverse the pseudonymisation (§2 stage (4)). It gives no
procedure; this project reads it as follows.

* A pseudonym is ``[`` NAME ``_`` h ``]`` inside one record, NAME the name of
  an entity type t of the schema and h exactly L lower-case hex characters,
  L the schema's slug length (L >= 1: with L = 0 the replacement carries no
  hash and nothing can be reversed). Type names hold no ``[`` or ``]``, so
  pseudonyms never overlap; at most one type name fits at a position.
* It resolves to the map entry of type t whose full hash begins with h when
  exactly one entry of type t does ("ambiguous" when several do, as two
  entities can share a short slug); and the entry must check out under the
  key: HMAC-SHA256(key, original) equals its full hash ("unverified" when it
  does not, as with a wrong key or an altered row).
* A resolved pseudonym is replaced by the entry's original bytes; every other
  byte, and every pseudonym that does not resolve, is copied unchanged.

So re-identifying the output of an anonymization with its map and key gives
back the input, except where two entities of one type share a slug.

Test infrastructure: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.
"""
from __future__ import annotations

from dataclasses import dataclass

from .hmac_sha256 import hmac_sha256

_HEX = set(b"0123456789abcdef")


@dataclass
class ReidStats:
    pseudonyms: int = 0
    resolved: int = 0
    ambiguous: int = 0
    unverified: int = 0


def match_at(data: bytes, i: int, type_names: list[str], slug_len: int) -> tuple[int, bytes] | None:
    """(type, slug) of the pseudonym starting at ``i``, else None."""
    if data[i:i + 1] != b"[":
        return None
    for t, name in enumerate(type_names, start=1):
        nb = name.encode()
        end = i + 1 + len(nb) + 1 + slug_len
        if data[i + 1:i + 1 + len(nb)] != nb or data[i + 1 + len(nb):i + 2 + len(nb)] != b"_":
            continue
        h = data[i + 2 + len(nb):end]
        if len(h) == slug_len and all(c in _HEX for c in h) and data[end:end + 1] == b"]":
            return t, h
    return None


def reidentify(records: list[bytes], entries, type_names: list[str], slug_len: int, key: bytes,
               stats: ReidStats | None = None) -> list[bytes]:
    """Records with every resolvable pseudonym replaced by its original.

    ``entries``: map entries with ``type``, ``original`` and ``full_hash``
    (64 lower-case hex characters)."""
    if slug_len < 1:
        raise ValueError("pseudonyms without a slug cannot be re-identified")
    for name in type_names:
        if "[" in name or "]" in name:
            raise ValueError("type names must not contain brackets")
    st = ReidStats() if stats is None else stats
    out = []
    for data in records:
        res = bytearray()
        i = 0
        while i < len(data):
            m = match_at(data, i, type_names, slug_len)
            if m is None:
                res.append(data[i])
                i += 1
                continue
            t, h = m
            plen = 3 + len(type_names[t - 1].encode()) + slug_len
            st.pseudonyms += 1
            hits = [e for e in entries if e.type == t and e.full_hash.encode().startswith(h)]
            if len(hits) > 1:
                st.ambiguous += 1
            elif len(hits) == 1 and hmac_sha256(key, hits[0].original).hex() != hits[0].full_hash:
                st.unverified += 1
            elif len(hits) == 1:
                st.resolved += 1
                res += hits[0].original
                i += plen
                continue
            res += data[i:i + plen]
            i += plen
        out.append(bytes(res))
    return out
