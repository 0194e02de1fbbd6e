"""Pins for the oracle's BIO decoder: exhaustive enumeration.

Every label sequence over the nine labels (four entity types) up to length 6
(9^6 = 531,441 at n = 6) is decoded by the oracle and by a second, different
formulation: group consecutive tokens of the same entity type, then split each
group before every B label. Also: encoding the decoded spans back to strict
IOB2 returns a well-formed input unchanged.
"""
import itertools

import numpy as np

from oracle.bio import decode, label_type


def group_split_decode(labels):
    spans = []
    i = 0
    n = len(labels)
    while i < n:
        t, _ = label_type(labels[i])
        j = i
        while j + 1 < n and label_type(labels[j + 1])[0] == t:
            j += 1
        if t:
            start = i
            for k in range(i + 1, j + 1):
                if label_type(labels[k])[1]:
                    spans.append((start, k - 1, t))
                    start = k
            spans.append((start, j, t))
        i = j + 1
    return spans


def encode(spans, n):
    out = [0] * n
    for a, b, t in spans:
        out[a] = 2 * t - 1
        for k in range(a + 1, b + 1):
            out[k] = 2 * t
    return out


def well_formed(labels):
    prev = 0
    for lab in labels:
        t, begin = label_type(lab)
        if t and not begin:
            pt, _ = label_type(prev)
            if pt != t:
                return False
        prev = lab
    return True


def test_exhaustive_up_to_six():
    count = 0
    wf = 0
    for n in range(0, 7):
        for seq in itertools.product(range(9), repeat=n):
            seq = list(seq)
            got = decode(seq)
            assert got == group_split_decode(seq), seq
            # spans are disjoint, ordered, typed consistently with their first label
            for (a, b, t), nxt in zip(got, got[1:] + [None]):
                assert a <= b and label_type(seq[a])[0] == t
                if nxt is not None:
                    assert b < nxt[0]
            if well_formed(seq):
                assert encode(got, n) == seq
                wf += 1
            count += 1
    assert count == sum(9 ** n for n in range(7))
    assert wf > 1000


def test_seventeen_labels_random():
    rng = np.random.default_rng(3)
    for _ in range(20000):
        seq = rng.integers(0, 17, size=int(rng.integers(0, 40))).tolist()
        assert decode(seq) == group_split_decode(seq)
