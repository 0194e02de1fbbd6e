"""Reduced-precision number formats, written from their definitions (oracle).

Test infrastructure: only tests, the smoke entry point and the benchmark's
CPU baseline use this package.

The paper runs its NER model on a GPU and states no arithmetic precision (§2
stage (2), §3). The reduced-precision modes of the encoder are readings of
the workload specification: BF16 GEMM inputs with FP32 accumulation, and
FP8 E4M3 GEMM inputs with static per-tensor scales and FP32 accumulation.
This module gives the two roundings those modes apply, as plain arithmetic
on float64 arrays:

* BF16: 1 sign bit, 8 exponent bits (bias 127), 7 stored mantissa bits, so 8
  significant bits. A finite value x = m * 2^e with 0.5 <= |m| < 1 has the
  spacing 2^(e - 8) between neighbours; below 2^-126 the spacing stays 2^-133
  (subnormals). Round to nearest, ties to the even neighbour.
* E4M3 (the "fn" variant used for FP8 GEMM operands): 1 sign bit, 4 exponent
  bits (bias 7), 3 mantissa bits, no infinities; the largest finite value is
  1.75 * 2^8 = 448 and the code S.1111.111 is NaN. Normal values have 4
  significant bits, spacing 2^(e - 4); below the smallest normal 2^-6 the
  spacing stays 2^-9. Round to nearest, ties to even, and saturate: a
  magnitude above 448 becomes 448 (the conversion a GPU applies to GEMM
  operands with "satfinite").

The results are float64 arrays holding exactly representable values, so the
rest of the computation can stay in float64.
"""
from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0


def _round_to_spacing(x: np.ndarray, sig_bits: int, min_exp: int) -> np.ndarray:
    """Round x to the nearest multiple of its format spacing, ties to even.

    sig_bits: significant bits (implicit bit included); min_exp: exponent of
    the smallest normal value (its spacing is kept below it)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                       # x = m * 2^e, 0.5 <= |m| < 1 (m = 0 for x = 0)
    # the smallest normal 2^min_exp has frexp exponent min_exp + 1
    e = np.maximum(e, min_exp + 1)
    spacing = np.ldexp(1.0, e - sig_bits)
    return np.rint(x / spacing) * spacing    # x / spacing is exact; rint ties to even


def round_bf16(x) -> np.ndarray:
    """Nearest BF16 value (ties to even) of each element, as float64."""
    return _round_to_spacing(x, 8, -126)


def round_e4m3(x) -> np.ndarray:
    """Nearest E4M3 value (ties to even, saturating at +-448) of each element, as float64."""
    y = _round_to_spacing(x, 4, -6)
    return np.clip(y, -E4M3_MAX, E4M3_MAX)


def e4m3_code_values() -> np.ndarray:
    """Value of each of the 256 E4M3 codes from the bit layout (NaN for the two NaN codes)."""
    out = np.empty(256)
    for c in range(256):
        s, ex, mt = c >> 7, (c >> 3) & 0xF, c & 0x7
        if ex == 0xF and mt == 0x7:
            v = np.nan
        elif ex == 0:
            v = mt / 8.0 * 2.0 ** -6
        else:
            v = (1.0 + mt / 8.0) * 2.0 ** (ex - 7)
        out[c] = -v if s else v
    return out


def quantize_e4m3(x, scale: float) -> np.ndarray:
    """Per-tensor scaled E4M3: the E4M3 value of x / scale, times scale (as float64)."""
    return round_e4m3(np.asarray(x, dtype=np.float64) / scale) * scale


def tensor_scale(x) -> float:
    """The per-tensor scale amax / 448 (1 when the tensor is all zero)."""
    a = float(np.max(np.abs(x))) if np.size(x) else 0.0
    return a / E4M3_MAX if a > 0 else 1.0
