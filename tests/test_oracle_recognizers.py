"""Pins for the oracle's pattern recognizers.

Independent formulation: Python's ``ipaddress`` for both IP families and
``re`` patterns for the word rule, MAC, CVE and host names, written from the
stated rules rather than from the oracle's character loops. Fuzzing over
adversarial words, and every entity the generator planted must come back
with its exact span and type.
"""
import ipaddress
import re

import numpy as np
import pytest

from oracle import recognizers as R
from rx_fuzz import fuzz_record, rand_extra as _rand_extra, rand_word as _rand_word

WORD_RE = re.compile(rb"[A-Za-z0-9.:\-]+")
STRIP_RE = re.compile(rb"^(.*?)((?:[.\-]|(?<!:):)*)$", re.S)
MAC_RE = re.compile(rb"[0-9A-Fa-f]{2}([:\-])[0-9A-Fa-f]{2}(?:\1[0-9A-Fa-f]{2}){4}")
CVE_RE = re.compile(rb"CVE-[0-9]{4}-[0-9]{4,}")
LABEL = rb"[A-Za-z0-9](?:[A-Za-z0-9\-]{0,61}[A-Za-z0-9])?"
HOST_RE = re.compile(rb"((?:" + LABEL + rb"\.)+[A-Za-z]{2,63})(?::[0-9]{1,5})?")
IP4_PORT_RE = re.compile(rb"([0-9.]+)(?::[0-9]{1,5})?")


def ref_ipv4(w: bytes):
    m = IP4_PORT_RE.fullmatch(w)
    if not m:
        return 0
    try:
        ipaddress.IPv4Address(m.group(1).decode())
    except ValueError:
        return 0
    return len(m.group(1))


def ref_ipv6(w: bytes):
    if b"." in w or b":" not in w:
        return False
    try:
        ipaddress.IPv6Address(w.decode())
        return True
    except ValueError:
        return False


def ref_host(w: bytes):
    m = HOST_RE.fullmatch(w)
    if not m or len(m.group(1)) > 253:
        return 0
    return len(m.group(1))


def ref_recognize(data: bytes):
    out = []
    for m in WORD_RE.finditer(data):
        w = STRIP_RE.fullmatch(m.group(0)).group(1)
        s = m.start()
        if not w:
            continue
        if MAC_RE.fullmatch(w):
            out.append((s, len(w), R.MAC_ADDRESS))
        elif ref_ipv6(w):
            out.append((s, len(w), R.IP_ADDRESS))
        elif (n := ref_ipv4(w)):
            out.append((s, n, R.IP_ADDRESS))
        elif CVE_RE.fullmatch(w):
            out.append((s, len(w), R.CVE_ID))
        elif (n := ref_host(w)):
            out.append((s, n, R.HOSTNAME))
    return out


CASES = [
    (b"100.111.20.23", [(0, 13, 1)]),
    (b"host 10.0.0.1:8080, next", [(5, 8, 1)]),
    (b"01.2.3.4 256.1.1.1 1.2.3 1.2.3.4.5", []),
    (b"0.0.0.0", [(0, 7, 1)]),
    (b"fe80::1 ::1 :: 2001:db8:0:0:0:0:0:1", [(0, 7, 1), (8, 3, 1), (12, 2, 1), (15, 20, 1)]),
    (b"fe80:: then", [(0, 6, 1)]),
    (b"1:2:3:4:5:6:7:8:9 1::2::3 12345::1 a:::b", []),
    (b"aa:bb:cc:dd:ee:ff AA-BB-CC-DD-EE-FF aa:bb-cc:dd:ee:ff", [(0, 17, 4), (18, 17, 4)]),
    (b"see CVE-2021-44228. and cve-2021-44228 CVE-21-1234 CVE-2021-123", [(4, 14, 3)]),
    (b"web01.corp.example.org:443 index.php a.b x.y1 -a.com a-.com", [(0, 22, 2), (27, 9, 2)]),
    (b"db.local.", [(0, 8, 2)]),
    (b"", []),
    (b"...:::---", []),
]


@pytest.mark.parametrize("data,expect", CASES)
def test_hand_cases(data, expect):
    assert R.recognize(data) == expect
    assert ref_recognize(data) == expect


def test_fuzz_against_independent_formulation():
    rng = np.random.default_rng(7)
    n = 0
    for _ in range(6000):
        data = fuzz_record(rng, extended=False)
        got = R.recognize(data)
        assert got == ref_recognize(data), data
        n += len(got)
    assert n > 1000


def test_planted_entities_found(c1_records):
    planted = c1_records.planted
    found = 0
    for ri in range(c1_records.n):
        spans = set(R.recognize(c1_records.record(ri)))
        for _, s, n, t in planted[planted[:, 0] == ri]:
            assert (int(s), int(n), int(t)) in spans, (ri, c1_records.record(ri)[s:s + n])
            found += 1
    assert found == len(planted) > 1000


# ---------------------------------------------------------------- the twelve-kind set
#
# Independent formulation of the extended recognizers: ``re`` patterns written
# from the stated rules, ``uuid.UUID`` and ``bytes.fromhex`` for UUIDs and
# fingerprints, and the left-to-right resolution obtained from ``re.finditer``
# over an alternation of the multi-word patterns (a scanning regex engine
# resumes after each match, which is the rule the oracle states).

import uuid

ALL = (R.MAC_ADDRESS, R.IP_ADDRESS, R.IP_ADDRESS, R.CVE_ID, R.HOSTNAME, 5, 6, 9, 7, 10, 11, 12)
NOT_WORD = rb"(?<![A-Za-z0-9.:\-])"
PEM_RE = rb"(?:(?<=\n)|^)-----BEGIN CERTIFICATE-----[A-Za-z0-9+/=\s]*-----END CERTIFICATE-----"
URL_RE = NOT_WORD + rb"[A-Za-z][A-Za-z0-9]{1,15}://[A-Za-z0-9\-._~:/?#\[\]@!$&*+,;=%]*[A-Za-z0-9\-_~/#\[\]@$&*+=%]"
CPE_COMP = rb"[A-Za-z0-9._~%!*?\-]"
CPE_FS_RE = NOT_WORD + rb"cpe:2\.3:[aoh*\-](?::" + CPE_COMP + rb"+){9}:" + CPE_COMP + rb"*[A-Za-z0-9_~%!*?\-]"
CPE_URI_RE = NOT_WORD + rb"cpe:/[aoh](?::[A-Za-z0-9._~%\-]*){0,6}(?<![.:])"
LONG_RE = re.compile(b"(" + PEM_RE + b")|(" + URL_RE + b")|(" + CPE_FS_RE + b")|(" + CPE_URI_RE + b")")
HASH_RE = re.compile(rb"[0-9A-Fa-f]{32}|[0-9A-Fa-f]{40}|[0-9A-Fa-f]{64}|[0-9A-Fa-f]{128}")
OID_RE = re.compile(rb"(?:0|[1-9][0-9]*)(?:\.(?:0|[1-9][0-9]*)){4,}")


def ref_uuid(w: bytes) -> bool:
    if len(w) != 36:
        return False
    try:
        return str(uuid.UUID(w.decode())) == w.decode().lower()
    except ValueError:
        return False


def ref_fp(w: bytes) -> bool:
    if not re.fullmatch(rb"[0-9A-Fa-f]{2}(?::[0-9A-Fa-f]{2})*", w):
        return False
    return len(bytes.fromhex(w.replace(b":", b"").decode())) in (16, 20, 32)


def ref_oid(w: bytes) -> bool:
    if not OID_RE.fullmatch(w):
        return False
    arcs = [int(a) for a in w.split(b".")]
    return arcs[0] <= 2 and (arcs[0] == 2 or arcs[1] <= 39)


def ref_word_all(w: bytes):
    if MAC_RE.fullmatch(w):
        return len(w), R.MAC_ADDRESS
    if ref_ipv6(w):
        return len(w), R.IP_ADDRESS
    if n := ref_ipv4(w):
        return n, R.IP_ADDRESS
    if CVE_RE.fullmatch(w):
        return len(w), R.CVE_ID
    if n := ref_host(w):
        return n, R.HOSTNAME
    if HASH_RE.fullmatch(w):
        return len(w), 6
    if ref_uuid(w):
        return len(w), 9
    if ref_fp(w):
        return len(w), 11
    if ref_oid(w):
        return len(w), 10
    return 0, 0


def ref_recognize_all(data: bytes):
    longs = []
    for m in LONG_RE.finditer(data):
        t = (12, 5, 7, 7)[m.lastindex - 1]
        longs.append((m.start(), m.end() - m.start(), t))
    out = list(longs)
    for m in WORD_RE.finditer(data):
        s = m.start()
        if any(ls <= s < ls + ln for ls, ln, _ in longs):
            continue
        w = STRIP_RE.fullmatch(m.group(0)).group(1)
        if w:
            n, t = ref_word_all(w)
            if n:
                out.append((s, n, t))
    return sorted(out)


def _at(data: bytes, *hits):
    """Expected spans from (substring, type) pairs, each located after the previous one."""
    out, pos = [], 0
    for sub, t in hits:
        k = data.index(sub, pos)
        out.append((k, len(sub), t))
        pos = k + len(sub)
    return data, out


EXT_CASES = [
    _at(b"d41d8cd98f00b204e9800998ecf8427e and " + b"A" * 40 + b" " + b"f" * 31 + b" " + b"0" * 64,
        (b"d41d8cd98f00b204e9800998ecf8427e", 6), (b"A" * 40, 6), (b"0" * 64, 6)),
    _at(b"{123e4567-e89b-12d3-a456-426614174000} 123e4567e89b-12d3-a456-426614174000",
        (b"123e4567-e89b-12d3-a456-426614174000", 9)),
    _at(b"oid 1.3.6.1.4.1.311 2.5.29.17.1 3.1.2.3.4 1.40.1.2.3 1.39.1.2.3. 01.3.6.1.4 10.3.6.1",
        (b"1.3.6.1.4.1.311", 10), (b"2.5.29.17.1", 10), (b"1.39.1.2.3", 10), (b"10.3.6.1", 1)),
    _at(b"fp 3A:5F:00:11:22:33:44:55:66:77:88:99:AA:BB:CC:DD:EE:FF:00:11 aa:bb:cc:dd:ee:ff:00:11:22:33:44:55:66:77:88",
        (b"3A:5F:00:11:22:33:44:55:66:77:88:99:AA:BB:CC:DD:EE:FF:00:11", 11)),
    _at(b"go to https://web01.example.com:8443/a/b?x=1&y=%20z#frag. Next",
        (b"https://web01.example.com:8443/a/b?x=1&y=%20z#frag", 5)),
    _at(b"(see http://10.0.0.1/index.php), x.http://a.bc",
        (b"http://10.0.0.1/index.php", 5), (b"x.http", 2), (b"a.bc", 2)),
    _at(b"http:// ftp://x, h://x verylongschemename12://x", (b"ftp://x", 5)),
    _at(b"cpe:2.3:a:apache:http_server:2.4.41:*:*:*:*:*:*:*. cpe:/a:apache:tomcat:9.0:. cpe:2.3:x:a:b:c:d:e:f:g:h:i:j",
        (b"cpe:2.3:a:apache:http_server:2.4.41:*:*:*:*:*:*:*", 7), (b"cpe:/a:apache:tomcat:9.0", 7)),
    _at(b"cpe:2.3:a:b:c:d:e:f:g:h:i:j:k:extra.example.com", (b"cpe:2.3:a:b:c:d:e:f:g:h:i:j:k", 7)),
    _at(b"url http://host/?c=cpe:2.3:a:b:c:d:e:f:g:h:i:j:k done", (b"http://host/?c=cpe:2.3:a:b:c:d:e:f:g:h:i:j:k", 5)),
    _at(b"x\n-----BEGIN CERTIFICATE-----\nMIIB+/=\nd41d8cd98f00b204e9800998ecf8427e\n-----END CERTIFICATE-----\ny",
        (b"-----BEGIN CERTIFICATE-----\nMIIB+/=\nd41d8cd98f00b204e9800998ecf8427e\n-----END CERTIFICATE-----", 12)),
    _at(b" -----BEGIN CERTIFICATE-----\nAAAA\n-----END CERTIFICATE-----"),
    _at(b"-----BEGIN CERTIFICATE-----\nAA:AA\n-----END CERTIFICATE-----"),
]


@pytest.mark.parametrize("data,expect", EXT_CASES)
def test_extended_hand_cases(data, expect):
    got = R.recognize(data, ALL)
    assert got == expect, [(s, n, t, data[s:s + n]) for s, n, t in got]
    assert ref_recognize_all(data) == expect


def test_default_table_is_the_five_address_recognizers():
    data = b"10.0.0.1 http://a.com/x d41d8cd98f00b204e9800998ecf8427e cpe:/a:b"
    assert R.recognize(data) == R.recognize(data, R.DEFAULT_TYPES) == [(0, 8, 1), (16, 5, 2)]


def test_switched_off_kinds_fall_through():
    """With the MAC recognizer off a MAC is nothing; with URLs off their host names are found."""
    t = list(ALL)
    t[R.KIND_MAC] = 0
    t[R.KIND_URL] = 0
    assert R.recognize(b"aa:bb:cc:dd:ee:ff http://a.example.com/x", t) == [(25, 13, 2)]


def test_extended_fuzz_against_independent_formulation():
    rng = np.random.default_rng(11)
    n = dropped = 0
    kinds = set()
    for _ in range(6000):
        data = fuzz_record(rng, extended=True)
        got = R.recognize(data, ALL)
        assert got == ref_recognize_all(data), data
        n += len(got)
        dropped += len(R.candidates(data, ALL)) - len(got)
        kinds |= {t for _, _, t in got}
    # candidates inside an accepted multi-word span occur, so resolution is exercised
    assert n > 3000 and dropped > 100 and kinds >= {1, 2, 3, 5, 6, 7, 9, 10, 11, 12}


def test_extended_planted_entities_found(vocab_words):
    import synth
    recs = synth.make_records(synth.C1X.records, vocab_words)
    table = ALL[:11] + (11,)         # both certificate forms to type 11, as the generator plants them
    planted = recs.planted
    found = 0
    for ri in range(recs.n):
        spans = set(R.recognize(recs.record(ri), table))
        for _, s, n, t in planted[planted[:, 0] == ri]:
            assert (int(s), int(n), int(t)) in spans, (ri, recs.record(ri)[s:s + n])
            found += 1
    assert found == len(planted) > 1500
    assert set(planted[:, 3].tolist()) == {1, 2, 3, 4, 5, 6, 7, 9, 10, 11}
