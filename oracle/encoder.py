"""Encoder-only token classifier in FP64 (oracle).

The paper tags entities with a transformer token-classification model run on
the GPU (§2 stage (2); the default is an XLM-RoBERTa-base NER model). Trained
weights are not available, so the architecture is kept and the weights are
seeded random (``synth.model``). Reading of the block, in this order:

* X = LN(E[id] + P[pos]) with learned absolute positions 0..L-1;
* per layer (post-LayerNorm): QKV = X Wqkv^T + b, columns [0, d) are Q,
  [d, 2d) K, [2d, 3d) V, head j owning columns j*dh..(j+1)*dh of each;
  A = softmax(Q K^T / sqrt(dh)) V per head over the same sequence only;
  X = LN(X + A Wo^T + bo); X = LN(X + GELU(X W1^T + b1) W2^T + b2);
* logits = X Wc^T + bc.
LayerNorm uses the biased variance (divide by d) and eps = 1e-5; GELU is the
exact form 0.5 x (1 + erf(x / sqrt 2)); no dropout.

Reduced precision (readings of the workload specification; the paper states
no precision): ``precision="bf16"`` rounds every projection weight and every
projection input to BF16; ``precision="fp8"`` quantizes them to E4M3
with one scale per tensor: amax(W) / 448 per weight matrix and, per layer,
four static activation scales given by the caller (QKV input, attention
output, FFN input, GELU output; ``calibrate`` computes amax / 448 over
calibration sequences). In both modes the QKV projection's output is
held in BF16 and so are the attention probabilities that multiply V (taken
against the row maximum, divided by the sum of the unrounded ones);
accumulation, bias, residual stream, LayerNorm, softmax and the classifier
stay exact (float64 here, FP32 on the device). The default ``"fp64"`` rounds
nothing.

Long records: the paper truncates them (§5, "standalone truncation"). Here a
record longer than the window is split into windows starting at 0, S, 2S, ...
(a new window starts while the previous one ends before the record does);
a token in the overlap of windows w and w+1 takes window w's logits if it lies
less than (W - S) / 2 tokens past the start of window w+1, else window w+1's.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

from . import lowp

LN_EPS = 1e-5


class RecordTooLong(ValueError):
    pass


def layer_norm(x: np.ndarray, g: np.ndarray, b: np.ndarray) -> np.ndarray:
    mu = x.mean(axis=-1, keepdims=True)
    var = ((x - mu) ** 2).mean(axis=-1, keepdims=True)
    return (x - mu) / np.sqrt(var + LN_EPS) * g + b


def gelu(x: np.ndarray) -> np.ndarray:
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def softmax(s: np.ndarray) -> np.ndarray:
    m = s.max(axis=-1, keepdims=True)
    e = np.exp(s - m)
    return e / e.sum(axis=-1, keepdims=True)


PROJECTIONS = ("w_qkv", "w_o", "w_1", "w_2")


class Encoder:
    """FP64 copy of the weights and the forward pass of one sequence.

    precision: "fp64" (default), "bf16" or "fp8" (see the module docstring);
    act_scales: for "fp8", 4 scales per layer in the order QKV input,
    attention output, FFN input, GELU output."""

    def __init__(self, dims, weights: dict[str, np.ndarray], precision: str = "fp64", act_scales=None):
        if precision not in ("fp64", "bf16", "fp8"):
            raise ValueError(f"unknown precision {precision!r}")
        if precision == "fp8" and (act_scales is None or len(act_scales) != 4 * dims.n_layers):
            raise ValueError("fp8 needs 4 activation scales per layer")
        self.dims = dims
        self.precision = precision
        self.act_scales = None if act_scales is None else [float(a) for a in act_scales]
        self.w = {k: np.asarray(v, dtype=np.float64) for k, v in weights.items()}
        # the projection weights as the GEMMs see them
        self.wq = {}
        for k, v in self.w.items():
            if k.split(".")[-1] in PROJECTIONS:
                if precision == "bf16":
                    self.wq[k] = lowp.round_bf16(v)
                elif precision == "fp8":
                    self.wq[k] = lowp.quantize_e4m3(v, lowp.tensor_scale(v))
                else:
                    self.wq[k] = v

    def _input(self, x: np.ndarray, layer: int, slot: int) -> np.ndarray:
        """A projection input as the GEMM sees it (slot: 0 QKV, 1 attention out, 2 FFN in, 3 GELU out)."""
        if self.precision == "bf16":
            return lowp.round_bf16(x)
        if self.precision == "fp8":
            return lowp.quantize_e4m3(x, self.act_scales[4 * layer + slot])
        return x

    def hidden(self, ids: list[int] | np.ndarray, probe=None) -> np.ndarray:
        """Last hidden state [L, d]. probe(layer, slot, x), when given, sees every
        projection input before rounding (calibration)."""
        d = self.dims
        w, wq = self.w, self.wq
        low = self.precision != "fp64"
        ids = np.asarray(ids, dtype=np.int64)
        L = len(ids)
        if L > d.max_pos:
            raise RecordTooLong(f"sequence of {L} tokens exceeds {d.max_pos} positions")
        x = w["tok_emb"][ids] + w["pos_emb"][np.arange(L)]
        x = layer_norm(x, w["emb_ln_g"], w["emb_ln_b"])
        m, h, dh = d.d_model, d.n_heads, d.d_head
        scale = 1.0 / np.sqrt(dh)

        def proj(x, i, slot, name):
            if probe is not None:
                probe(i, slot, x)
            return self._input(x, i, slot) @ wq[f"l{i}.{name}"].T

        for i in range(d.n_layers):
            p = f"l{i}."
            qkv = proj(x, i, 0, "w_qkv") + w[p + "b_qkv"]
            if low:
                qkv = lowp.round_bf16(qkv)
            q = qkv[:, 0:m].reshape(L, h, dh).transpose(1, 0, 2)
            k = qkv[:, m:2 * m].reshape(L, h, dh).transpose(1, 0, 2)
            v = qkv[:, 2 * m:3 * m].reshape(L, h, dh).transpose(1, 0, 2)
            s = q @ k.transpose(0, 2, 1) * scale                 # [h, L, L]
            if low:
                e = np.exp(s - s.max(axis=-1, keepdims=True))
                a = (lowp.round_bf16(e) @ v) / e.sum(axis=-1, keepdims=True)
            else:
                a = softmax(s) @ v
            a = a.transpose(1, 0, 2).reshape(L, m)
            x = layer_norm(x + proj(a, i, 1, "w_o") + w[p + "b_o"], w[p + "ln1_g"], w[p + "ln1_b"])
            f = gelu(proj(x, i, 2, "w_1") + w[p + "b_1"])
            x = layer_norm(x + proj(f, i, 3, "w_2") + w[p + "b_2"], w[p + "ln2_g"], w[p + "ln2_b"])
        return x

    def logits(self, ids) -> np.ndarray:
        x = self.hidden(ids)
        return x @ self.w["cls_w"].T + self.w["cls_b"]


def calibrate(enc: Encoder, sequences) -> list[float]:
    """Static FP8 activation scales: amax / 448 of each projection input of each
    layer over the sequences, from an unrounded (float64) pass; 4 per layer in
    the order QKV input, attention output, FFN input, GELU output."""
    amax = [0.0] * (4 * enc.dims.n_layers)

    def probe(layer, slot, x):
        amax[4 * layer + slot] = max(amax[4 * layer + slot], float(np.max(np.abs(x))) if x.size else 0.0)

    ref = Encoder(enc.dims, {k: v for k, v in enc.w.items()})
    for ids in sequences:
        if len(ids):
            ref.hidden(ids, probe=probe)
    return [a / lowp.E4M3_MAX if a > 0 else 1.0 for a in amax]


def window_starts(L: int, window: int, stride: int) -> list[int]:
    starts = [0]
    while starts[-1] + window < L:
        starts.append(starts[-1] + stride)
    return starts


def window_owner(L: int, window: int, stride: int) -> list[int]:
    """For each token, the index of the window whose logits it takes."""
    starts = window_starts(L, window, stride)
    half = (window - stride) // 2
    owner = []
    for t in range(L):
        w = 0
        while w + 1 < len(starts) and t >= starts[w + 1] + half:
            w += 1
        owner.append(w)
    return owner


def record_logits(enc: Encoder, ids: list[int], window: int = 0, stride: int = 0) -> np.ndarray:
    """Logits [L, C] of one record, through sliding windows when ``window`` > 0."""
    L = len(ids)
    if L == 0:
        return np.zeros((0, enc.dims.n_labels))
    if window == 0:
        return enc.logits(ids)
    starts = window_starts(L, window, stride)
    owner = window_owner(L, window, stride)
    per_window = [enc.logits(ids[s:min(s + window, L)]) for s in starts]
    out = np.empty((L, enc.dims.n_labels))
    for t in range(L):
        w = owner[t]
        out[t] = per_window[w][t - starts[w]]
    return out


def encoded_tokens(L: int, window: int, stride: int) -> int:
    """Tokens the encoder runs for a record (window overlaps counted twice)."""
    if L == 0:
        return 0
    if window == 0:
        return L
    return sum(min(s + window, L) - s for s in window_starts(L, window, stride))


def argmax_first(logits: np.ndarray) -> np.ndarray:
    """Label per token: the highest logit, the lowest label index on ties."""
    return np.argmax(logits, axis=-1)
