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


def _rand_word(rng):
    k = rng.integers(9)
    hx = "0123456789abcdefABCDEF"
    if k == 0:
        return ".".join(str(rng.integers(0, 300)) if rng.integers(6) else "0" + str(rng.integers(0, 30))
                        for _ in range(rng.integers(2, 6))) + (f":{rng.integers(0, 999999)}" if rng.integers(3) == 0 else "")
    if k == 1:
        groups = ["".join(rng.choice(list(hx), size=rng.integers(0, 6))) for _ in range(rng.integers(1, 10))]
        return ":".join(groups)
    if k == 2:
        sep = rng.choice([":", "-", "."])
        return sep.join("".join(rng.choice(list(hx), size=rng.integers(1, 4))) for _ in range(rng.integers(4, 8)))
    if k == 3:
        return f"{rng.choice(['CVE', 'cve', 'CVE'])}-{rng.integers(0, 99999)}-{rng.integers(0, 9999999)}"
    if k == 4:
        labs = []
        for _ in range(rng.integers(1, 5)):
            n = rng.integers(0, 8)
            labs.append("".join(rng.choice(list("abz09-XY"), size=n)))
        return ".".join(labs) + (f":{rng.integers(0, 99)}" if rng.integers(4) == 0 else "")
    if k == 5:
        return "".join(rng.choice(list("a1.:-f"), size=rng.integers(1, 20)))
    if k == 6:
        return "x" * int(rng.integers(60, 70)) + ".com"
    if k == 7:
        return ".".join(["a" * 63] * 4) + ".org"
    return "".join(rng.choice(list("0123456789:."), size=rng.integers(1, 25)))


def test_fuzz_against_independent_formulation():
    rng = np.random.default_rng(7)
    n = 0
    for _ in range(6000):
        parts = [_rand_word(rng) for _ in range(rng.integers(1, 6))]
        seps = [rng.choice([" ", ", ", "\n", "(", ") ", "/", "=", "\xe9"]) for _ in parts]
        data = "".join(p + s for p, s in zip(parts, seps)).encode("utf-8")
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
