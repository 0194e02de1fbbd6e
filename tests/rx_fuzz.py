"""Adversarial inputs for the pattern recognizers (test helper, no recognizer logic).

Words near the edge of each recognizer's rule (wrong lengths, leading zeros,
wrong separators, truncated schemes and PEM blocks), joined by separators
that do and do not end a word.
"""
import numpy as np


def rand_word(rng):
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


def rand_extra(rng):
    hx = "0123456789abcdefABCDEF"
    k = rng.integers(9)
    if k == 0:
        return "".join(rng.choice(list(hx), size=rng.choice([31, 32, 33, 40, 64, 128])))
    if k == 1:
        sizes = [8, 4, 4, 4, 12] if rng.integers(2) else list(rng.integers(3, 13, size=5))
        return "-".join("".join(rng.choice(list(hx), size=int(n))) for n in sizes)
    if k == 2:
        return ".".join(str(rng.choice([0, 1, 2, 3, 39, 40, int(rng.integers(0, 99999))])) if rng.integers(8)
                        else "0" + str(rng.integers(1, 9)) for _ in range(rng.integers(3, 9)))
    if k == 3:
        return ":".join("".join(rng.choice(list(hx), size=2 if rng.integers(12) else 3))
                        for _ in range(rng.choice([15, 16, 20, 21, 32])))
    if k == 4:
        comps = ["".join(rng.choice(list("ab._~%!*?-:"), size=rng.integers(0, 4))) for _ in range(rng.integers(8, 14))]
        return "cpe:2.3:" + rng.choice(["a", "o", "*", "x", "ab"]) + ":" + ":".join(comps)
    if k == 5:
        comps = ["".join(rng.choice(list("ab.1_~%-"), size=rng.integers(0, 4))) for _ in range(rng.integers(0, 9))]
        return "cpe:/" + rng.choice(["a", "h", "x"]) + "".join(":" + c for c in comps)
    if k == 6:
        tail = "".join(rng.choice(list("ab1-._~:/?#[]@!$&*+,;=%'()\"<>"), size=rng.integers(0, 14)))
        return rng.choice(["http", "ftp", "h", "x1", "9p", "Https"]) + rng.choice(["://", ":/", "://"]) + tail
    if k == 7:
        body = "".join(rng.choice(list("AB+/=\n :"), size=rng.integers(0, 20)))
        end = rng.choice(["-----END CERTIFICATE-----", "-----END CERT-----", ""])
        return "\n-----BEGIN CERTIFICATE-----" + body + end
    return rand_word(rng)




def fuzz_record(rng: np.random.Generator, extended: bool) -> bytes:
    """One record of 1..5 adversarial words with separators (UTF-8 bytes)."""
    if extended:
        parts = [rand_extra(rng) for _ in range(rng.integers(1, 6))]
        seps = [rng.choice([" ", ", ", "\n", "(", ") ", "/", "=", "?", "\xe9", ""]) for _ in parts]
    else:
        parts = [rand_word(rng) for _ in range(rng.integers(1, 6))]
        seps = [rng.choice([" ", ", ", "\n", "(", ") ", "/", "=", "\xe9"]) for _ in parts]
    return "".join(p + s for p, s in zip(parts, seps)).encode("utf-8")
