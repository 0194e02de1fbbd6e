"""Seeded synthetic vulnerability-scan records.

Each record is a byte string shaped like one finding of a network scan: a
header line with host address, host name, port and plugin id, then free text
(description, solution, plugin output) assembled from the lexicon, with
entities planted at a target density: IPv4 (sometimes with a port), IPv6,
host names (sometimes with a port), CVE ids and MAC addresses, plus
look-alikes that are not entities (version strings, file names, out-of-range
octets). A shape with ``extra_kinds`` also plants URLs, hashes, CPE names,
UUIDs, OIDs, certificate fingerprints and PEM certificate blocks (each PEM
block on lines of its own), and look-alikes of those.

Record length is set in tokens. The generator cannot tokenize (it holds none
of the method's arithmetic), so it sizes text with a conservative count: an
isolated vocabulary word counts as one token, every other alphanumeric run
counts one token per byte, every other byte counts one. The true count is at
most this estimate, and a record whose pieces add up to more than its target
loses trailing pieces until they fit, so records never exceed the length cap;
runs that merge into fewer tokens make a record a few tokens shorter than its
target.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import lexicon as lx
from .workloads import EXTRA_KIND_TYPE, EXTRA_SHARE, RecordShape

T_IP, T_HOST, T_CVE, T_MAC = 1, 2, 3, 4

_HEX = "0123456789abcdef"
_B64 = "ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz0123456789+/"
# share of fresh entities by kind: IPv4, host name, CVE, MAC, IPv6
_KIND_CDF = [0.40, 0.62, 0.80, 0.90, 1.0]


@dataclass
class RecordSet:
    data: np.ndarray        # uint8 byte arena
    offsets: np.ndarray     # uint64 [n+1]
    planted: np.ndarray     # int64 [m, 4]: record, start (within record), length, type
    target_tokens: np.ndarray  # int32 [n]

    @property
    def n(self) -> int:
        return len(self.offsets) - 1

    def record(self, i: int) -> bytes:
        return self.data[int(self.offsets[i]):int(self.offsets[i + 1])].tobytes()

    def records(self) -> list[bytes]:
        return [self.record(i) for i in range(self.n)]


def _is_alnum(c: int) -> bool:
    return (48 <= c <= 57) or (65 <= c <= 90) or (97 <= c <= 122)


class _Rand:
    """Seeded uniform stream drawn in bulk (scalar numpy calls are slow)."""

    def __init__(self, rng: np.random.Generator, block: int = 1 << 20):
        self._rng = rng
        self._block = block
        self._buf = rng.random(block).tolist()
        self._i = 0

    def random(self) -> float:
        if self._i >= self._block:
            self._buf = self._rng.random(self._block).tolist()
            self._i = 0
        v = self._buf[self._i]
        self._i += 1
        return v

    def integers(self, lo: int, hi: int | None = None) -> int:
        if hi is None:
            lo, hi = 0, lo
        return lo + int(self.random() * (hi - lo))

    def choice(self, seq):
        return seq[int(self.random() * len(seq))]

    def weighted(self, cdf: list[float]) -> int:
        u = self.random()
        for i, c in enumerate(cdf):
            if u < c:
                return i
        return len(cdf) - 1

    def poisson(self, lam: float) -> int:
        # inversion by sequential search; lam is at most a few hundred here
        L = np.exp(-lam) if lam < 600 else 0.0
        if L == 0.0:
            return max(0, int(round(lam + np.sqrt(lam) * np.sqrt(-2 * np.log(max(self.random(), 1e-300)))
                                    * np.cos(2 * np.pi * self.random()))))
        k, p, s = 0, L, L
        u = self.random()
        while u > s:
            k += 1
            p *= lam / k
            s += p
        return k


class _Gen:
    def __init__(self, rng: np.random.Generator, vocab_words: list[bytes], shape: RecordShape):
        self.rng = _Rand(rng)
        self._np_rng = rng
        self._est_cache: dict[bytes, int] = {}
        self.vocab_set = set(vocab_words)
        self.shape = shape
        words = [w for w in (lx.NOUNS + lx.VERBS + lx.ADJECTIVES + lx.SERVICES + lx.FUNCTION_WORDS)]
        self.words = [w.encode() for w in words]
        self.cap_words = [w[:1].upper().encode() + w[1:].encode() for w in words]
        self.zipf_pool: list[tuple[bytes, int]] | None = None
        if shape.zipf_distinct > 0:
            self._build_zipf_pool(shape.zipf_distinct, shape.zipf_s)

    # ---- token estimate (upper bound; see module docstring) ----
    def est(self, s: bytes) -> int:
        c = self._est_cache.get(s)
        if c is not None:
            return c
        c = self._est(s)
        if len(s) <= 16:
            self._est_cache[s] = c
        return c

    def _est(self, s: bytes) -> int:
        n = 0
        i = 0
        L = len(s)
        while i < L:
            if _is_alnum(s[i]):
                j = i
                while j < L and _is_alnum(s[j]):
                    j += 1
                n += 1 if s[i:j] in self.vocab_set else (j - i)
                i = j
            else:
                n += 1
                i += 1
        return n

    # ---- entity makers ----
    def ipv4(self) -> bytes:
        r = self.rng
        k = int(r.integers(4))
        if k == 0:
            o = [10, int(r.integers(256)), int(r.integers(256)), int(r.integers(1, 255))]
        elif k == 1:
            o = [192, 168, int(r.integers(256)), int(r.integers(1, 255))]
        elif k == 2:
            o = [172, int(r.integers(16, 32)), int(r.integers(256)), int(r.integers(1, 255))]
        else:
            o = [int(r.integers(1, 224)), int(r.integers(256)), int(r.integers(256)), int(r.integers(256))]
        return ".".join(str(x) for x in o).encode()

    def ipv6(self) -> bytes:
        r = self.rng
        groups = []
        for _ in range(8):
            v = int(r.integers(0, 65536)) if int(r.integers(3)) else int(r.integers(0, 16))
            groups.append(format(v, "x"))
        if int(r.integers(2)) == 0:
            groups[0] = "fe80" if int(r.integers(2)) else "2001"
        if int(r.integers(2)):
            # compress one run of groups with "::"
            a = int(r.integers(0, 8))
            b = int(r.integers(a + 1, 9))
            s = ":".join(groups[:a]) + "::" + ":".join(groups[b:])
        else:
            s = ":".join(groups)
        if int(r.integers(5)) == 0:
            s = s.upper()
        return s.encode()

    def hostname(self) -> bytes:
        r = self.rng
        hw = lx.HOST_WORDS
        first = hw[int(r.integers(len(hw)))]
        if int(r.integers(2)):
            first += format(int(r.integers(0, 100)), "02d")
        if int(r.integers(4)) == 0:
            first += "-" + hw[int(r.integers(len(hw)))]
        labels = [first]
        for _ in range(int(r.integers(0, 3))):
            ow = lx.ORG_WORDS + lx.HOST_WORDS
            labels.append(ow[int(r.integers(len(ow)))])
        labels.append(lx.TLDS[int(r.integers(len(lx.TLDS)))])
        return ".".join(labels).encode()

    def cve(self) -> bytes:
        r = self.rng
        year = int(r.integers(1999, 2027))
        num = int(r.integers(1, 60000))
        width = 4 if num < 10000 else 5
        return f"CVE-{year}-{num:0{width}d}".encode()

    def mac(self) -> bytes:
        r = self.rng
        sep = ":" if int(r.integers(2)) else "-"
        s = sep.join(_HEX[int(r.integers(16))] + _HEX[int(r.integers(16))] for _ in range(6))
        if int(r.integers(3)) == 0:
            s = s.upper()
        return s.encode()

    def _hexs(self, n: int) -> str:
        return "".join(_HEX[int(self.rng.integers(16))] for _ in range(n))

    def url(self) -> bytes:
        r = self.rng
        scheme = r.choice(("http", "https", "https", "ftp", "ldap", "ssh", "smb"))
        host = self.hostname() if int(r.integers(4)) else self.ipv4()
        s = scheme.encode() + b"://" + host
        if int(r.integers(3)) == 0:
            s += f":{r.choice((80, 443, 8080, 8443, 389, 21))}".encode()
        for _ in range(int(r.integers(0, 4))):
            s += b"/" + self.word()
        if int(r.integers(3)) == 0:
            s += b"/" + self.word() + r.choice((b".php", b".html", b".jsp", b".cgi"))
        if int(r.integers(3)) == 0:
            s += b"?" + self.word() + b"=" + str(int(r.integers(1000))).encode()
            if int(r.integers(2)):
                s += b"&" + self.word() + b"=" + self.word() + b"%20" + self.word()
        if int(r.integers(6)) == 0:
            s += b"#" + self.word()
        return s

    def hash_hex(self) -> bytes:
        r = self.rng
        n = r.choice((32, 40, 64, 64, 128))
        h = self._hexs(n)
        return (h.upper() if int(r.integers(4)) == 0 else h).encode()

    def cpe(self) -> bytes:
        r = self.rng
        sv = lx.SERVICES
        vendor = sv[int(r.integers(len(sv)))]
        product = sv[int(r.integers(len(sv)))]
        if int(r.integers(2)):
            product += "_" + r.choice(("server", "http_server", "client", "daemon", "agent"))
        version = f"{int(r.integers(0, 12))}.{int(r.integers(0, 20))}"
        if int(r.integers(2)):
            version += f".{int(r.integers(0, 60))}"
        part = r.choice(("a", "a", "o", "h"))
        if int(r.integers(3)):
            tail = ":".join(r.choice(("*", "*", "*", "-")) for _ in range(7))
            return f"cpe:2.3:{part}:{vendor}:{product}:{version}:{tail}".encode()
        return f"cpe:/{part}:{vendor}:{product}:{version}".encode()

    def uuid(self) -> bytes:
        h = self._hexs(32)
        s = f"{h[:8]}-{h[8:12]}-{h[12:16]}-{h[16:20]}-{h[20:]}"
        return (s.upper() if int(self.rng.integers(5)) == 0 else s).encode()

    def oid(self) -> bytes:
        r = self.rng
        k = int(r.integers(3))
        if k == 0:
            arcs = [1, 3, 6, 1, 4, 1] + [int(r.integers(1, 60000)) for _ in range(int(r.integers(1, 4)))]
        elif k == 1:
            arcs = [1, 2, 840, 113549, 1] + [int(r.integers(1, 20)) for _ in range(int(r.integers(1, 3)))]
        else:
            arcs = [2, 5, 29, int(r.integers(1, 40))] + [int(r.integers(0, 10)) for _ in range(int(r.integers(1, 3)))]
        return ".".join(str(a) for a in arcs).encode()

    def cert_fp(self) -> bytes:
        r = self.rng
        g = r.choice((16, 20, 20, 32))
        s = ":".join(self._hexs(2) for _ in range(g))
        return (s.upper() if int(r.integers(2)) else s).encode()

    def pem(self) -> bytes:
        r = self.rng
        n = int(r.integers(48, 300))
        body = "".join(_B64[int(r.integers(64))] for _ in range(n)) + "=" * int(r.integers(0, 3))
        lines = "\n".join(body[i:i + 64] for i in range(0, len(body), 64))
        return f"-----BEGIN CERTIFICATE-----\n{lines}\n-----END CERTIFICATE-----".encode()

    def extra_entity(self, kind: str) -> bytes:
        return {"url": self.url, "hash": self.hash_hex, "cpe": self.cpe, "uuid": self.uuid, "oid": self.oid,
                "cert_fp": self.cert_fp, "pem": self.pem}[kind]()

    def extra_lookalike(self) -> bytes:
        r = self.rng
        k = int(r.integers(7))
        if k == 0:
            return self._hexs(r.choice((31, 33, 39, 63))).encode()
        if k == 1:
            h = self._hexs(32)
            return f"{h[:8]}-{h[8:13]}-{h[13:16]}-{h[16:20]}-{h[20:]}".encode()
        if k == 2:
            return f"1.{int(r.integers(40, 99))}.{int(r.integers(9))}.{int(r.integers(9))}.{int(r.integers(9))}".encode()
        if k == 3:
            return f"cpe:2.3:a:{lx.SERVICES[int(r.integers(len(lx.SERVICES)))]}:*".encode()
        if k == 4:
            return b"http:/" + self.word()
        if k == 5:
            return ":".join(self._hexs(2) for _ in range(int(r.choice((15, 17))))).encode()
        return f"3.{int(r.integers(9))}.{int(r.integers(9))}.{int(r.integers(9))}.{int(r.integers(9))}".encode()

    def _fresh_entity(self, kind: int) -> bytes:
        return (self.ipv4, self.hostname, self.cve, self.mac, self.ipv6)[kind]()

    def _build_zipf_pool(self, n: int, s: float):
        pool = []
        seen = set()
        while len(pool) < n:
            kind = int(self.rng.integers(5))
            e = self._fresh_entity(kind)
            if e in seen:
                continue
            seen.add(e)
            pool.append((e, (T_IP, T_HOST, T_CVE, T_MAC, T_IP)[kind]))
        self.zipf_pool = pool
        p = 1.0 / np.arange(1, n + 1, dtype=np.float64) ** s
        self.zipf_cdf = np.cumsum(p / p.sum())
        self.zipf_cdf[-1] = 1.0

    def entity(self) -> tuple[bytes, int, bool]:
        """(entity bytes, type, whether a :port suffix may follow it)."""
        if self.zipf_pool is not None:
            k = int(np.searchsorted(self.zipf_cdf, self.rng.random()))
            e, t = self.zipf_pool[min(k, len(self.zipf_pool) - 1)]
            return e, t, False
        extra = self.shape.extra_kinds
        if extra and self.rng.random() < EXTRA_SHARE:
            kind = extra[int(self.rng.integers(len(extra)))]
            return self.extra_entity(kind), EXTRA_KIND_TYPE[kind], False
        kind = self.rng.weighted(_KIND_CDF)
        return self._fresh_entity(kind), (T_IP, T_HOST, T_CVE, T_MAC, T_IP)[kind], kind in (0, 1)

    # ---- text makers ----
    def word(self, cap: bool = False) -> bytes:
        i = int(self.rng.integers(len(self.words)))
        return self.cap_words[i] if cap else self.words[i]

    def lookalike(self) -> bytes:
        r = self.rng
        k = int(r.integers(6))
        if k == 0:
            return f"{int(r.integers(1, 10))}.{int(r.integers(0, 20))}.{int(r.integers(0, 60))}".encode()
        if k == 1:
            return (lx.SERVICES[int(r.integers(len(lx.SERVICES)))] + ".php").encode()
        if k == 2:
            return f"{int(r.integers(256, 999))}.{int(r.integers(256))}.{int(r.integers(256))}.{int(r.integers(256))}".encode()
        if k == 3:
            return f"0{int(r.integers(1, 10))}.{int(r.integers(256))}.{int(r.integers(256))}.{int(r.integers(256))}".encode()
        if k == 4:
            return f"v{int(r.integers(1, 9))}.{int(r.integers(0, 9))}".encode()
        return "Ferrão".encode()   # non-ASCII bytes pass through as single-byte tokens

    def header(self) -> tuple[list[bytes], list[tuple[int, int]]]:
        """Pieces of the header line and the index of planted entities in it."""
        r = self.rng
        ip, ip_t = self.entity()[:2] if self.zipf_pool is not None else (self.ipv4(), T_IP)
        host = self.hostname()
        port = r.choice((21, 22, 25, 53, 80, 110, 143, 389, 443, 445, 3306, 5432, 6379, 8080, 8443, 9200))
        pid = int(r.integers(10000, 200000))
        sev = lx.SEVERITIES[int(r.integers(len(lx.SEVERITIES)))]
        pieces = [b"Host: ", ip, b" Name: ", host, f" Port: {port}/".encode(),
                  lx.PROTOCOLS[int(r.integers(2))].encode(), f" Plugin: {pid} Severity: ".encode(),
                  sev.encode(), b"\n"]
        return pieces, [(1, ip_t), (3, T_HOST)]


def _target_lengths(rng: np.random.Generator, shape: RecordShape) -> np.ndarray:
    n = shape.n_records
    if shape.length_dist == "uniform":
        return rng.integers(shape.lo, shape.hi + 1, size=n).astype(np.int32)
    x = rng.lognormal(mean=np.log(shape.median), sigma=shape.sigma, size=n)
    return np.clip(np.rint(x), shape.lo, shape.hi).astype(np.int32)


def make_records(shape: RecordShape, vocab_words: list[bytes], seed: int = 1001) -> RecordSet:
    rng = np.random.default_rng(seed)
    targets = _target_lengths(rng, shape)
    g = _Gen(rng, vocab_words, shape)
    rng = g.rng
    chunks: list[bytes] = []
    offsets = np.zeros(shape.n_records + 1, dtype=np.uint64)
    planted: list[tuple[int, int, int, int]] = []
    pos = 0
    est = g.est
    for ri in range(shape.n_records):
        target = int(targets[ri])
        parts: list[bytes] = []
        part_tok: list[int] = []
        nbytes = 0
        used = 0

        def put(piece: bytes, n_tok: int):
            nonlocal nbytes, used
            parts.append(piece)
            part_tok.append(n_tok)
            nbytes += len(piece)
            used += n_tok

        # header line, only when it fits
        hp, hent = g.header()
        h_est = sum(est(p) for p in hp)
        if h_est <= target:
            ent_idx = {i: t for i, t in hent}
            for i, p in enumerate(hp):
                if i in ent_idx:
                    planted.append((ri, nbytes, len(p), ent_idx[i]))
                put(p, est(p))
        n_ent = int(rng.poisson(shape.entities_per_1k * target / 1000.0))
        slots = sorted(rng.integers(0, max(target, 1)) for _ in range(n_ent))
        si = 0
        sentence_left = 0
        while True:
            room = target - used
            if room <= 0:
                break
            if si < len(slots) and used >= slots[si]:
                si += 1
                e, et, can_port = g.entity()
                if e.startswith(b"-----BEGIN"):      # a PEM block stands on lines of its own
                    lead, tail = b" " + g.word() + b":\n", b"\n"
                else:
                    lead = b" " + g.word() + b" "
                    tail = b"," if rng.integers(3) == 0 else b""
                n_e = est(e)
                if can_port and rng.integers(5) == 0:
                    port = f":{int(rng.integers(1, 65536))}".encode()
                else:
                    port = b""
                n_tot = est(lead) + n_e + est(port) + est(tail)
                if n_tot <= room:
                    put(lead, est(lead))
                    planted.append((ri, nbytes, len(e), et))
                    put(e, n_e)
                    if port:
                        put(port, est(port))
                    if tail:
                        put(tail, est(tail))
                continue
            if sentence_left <= 0:
                if room >= 3 and used > 0:
                    sep = b".\n" if rng.integers(4) == 0 else b". "
                    put(sep, 2)
                    room = target - used
                sentence_left = int(rng.integers(4, 16))
                room = target - used
                if room >= 2:
                    label = lx.FIELD_LABELS[int(rng.integers(len(lx.FIELD_LABELS)))].encode()
                    if room >= 5 and rng.integers(3) == 0:
                        put(b" " + label + b":", est(label) + 2)
                    else:
                        w = b" " + g.word(cap=True)
                        put(w, est(w))
                elif room == 1:
                    put(b".", 1)
                continue
            if rng.integers(40) == 0 and room >= 12:
                la = g.extra_lookalike() if g.shape.extra_kinds and rng.integers(2) else g.lookalike()
                p = b" " + la
                put(p, est(p))
                sentence_left -= 1
                continue
            w = g.word()
            p = b" " + w
            n_p = est(p)
            if n_p <= room:
                put(p, n_p)
            else:
                put(b".", 1)
            sentence_left -= 1
        # a sentence opener, field label or look-alike can take more than the
        # room left: drop trailing pieces (and the entities planted in them)
        # until the estimate is within the target, after every random draw of
        # the record, so that records which fit are unchanged
        while used > target and parts:
            nbytes -= len(parts.pop())
            used -= part_tok.pop()
            while planted and planted[-1][0] == ri and planted[-1][1] + planted[-1][2] > nbytes:
                planted.pop()
        rec = b"".join(parts)
        chunks.append(rec)
        pos += len(rec)
        offsets[ri + 1] = pos
    data = np.frombuffer(b"".join(chunks), dtype=np.uint8).copy()
    pl = np.array(planted, dtype=np.int64).reshape(-1, 4)
    return RecordSet(data=data, offsets=offsets, planted=pl, target_tokens=targets)


def records_from_list(recs: list[bytes]) -> RecordSet:
    offs = np.zeros(len(recs) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(r) for r in recs], dtype=np.uint64)
    data = np.frombuffer(b"".join(recs), dtype=np.uint8).copy() if recs else np.zeros(0, np.uint8)
    return RecordSet(data=data, offsets=offs, planted=np.zeros((0, 4), np.int64),
                     target_tokens=np.zeros(len(recs), np.int32))
