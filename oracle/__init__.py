"""Oracle for the pseudonymization hot path: TEST INFRASTRUCTURE, not product.

A plain, slow CPU restatement of what the method computes (AnonShield, §2
"The AnonShield Framework", stages (2) entity detection, (3) HMAC-SHA256
pseudonymisation, (4) persistence and (5) output), with the encoder in FP64.
Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it. It shares no code with the CUDA path; both read
the same seeded inputs from ``synth``.

Modules, in pipeline order:
  tokenizer      byte pre-tokenization and greedy longest-match subwords
  recognizers    pattern recognizers: MAC, IPv6, IPv4 (+port), CVE, host name (+port), hash,
                 UUID, certificate fingerprint, OID, PEM certificate, URL, CPE
  encoder        encoder-only token classifier, FP64, with sliding windows; BF16 and
                 FP8 E4M3 GEMM-input rounding emulated on request
  lowp           BF16 and E4M3 rounding written from the formats' definitions
  bio            BIO label decoding to token spans
  spans          token -> byte spans, overlap rule, preserve filter
  sha256         SHA-256 written from FIPS 180-4
  hmac_sha256    HMAC written from RFC 2104 on top of ``sha256``
  pseudonym      replacement strings, substitution and the entity map
  pipeline       the whole call: records, schema, key -> output records + map
  fields         per-field policy (detect / exclude / force per field id)
  reidentify     controlled re-identification: pseudonyms -> originals via map + key

Parity status: every function is pinned by tests under ``tests/`` against
brute force, closed forms, invariants or independent library routines,
except the pseudonym VALUE for the paper's worked example (§2 stage (3)),
whose key is not published: that one case is pinned for format only
(parity unpinned for the slug value).
"""
