"""Seeded random-init encoder weights and the HMAC key.

Every matrix and embedding is drawn N(0, 0.02) in FP32; biases are zero,
LayerNorm gains one and shifts zero. The classifier bias of label 0 ("O") is
set to ``o_bias_k * 0.02 * sqrt(d)`` so that an untrained tagger marks a
small share of tokens as entities instead of nearly all of them (logits of a
unit-variance row against N(0, 0.02) weights have standard deviation
0.02 * sqrt(d)). ``random_affine=True`` also draws biases and LayerNorm
parameters at random, so tests can see whether each of them is applied.

The flat blob order (FP32, row-major, nn.Linear [out, in] matrices):
  tok_emb [V, d], pos_emb [P, d], emb_ln_g [d], emb_ln_b [d],
  per layer: w_qkv [3d, d], b_qkv [3d], w_o [d, d], b_o [d], ln1_g [d], ln1_b [d],
             w_1 [f, d], b_1 [f], w_2 [d, f], b_2 [d], ln2_g [d], ln2_b [d],
  cls_w [C, d], cls_b [C].
"""
from __future__ import annotations

import numpy as np

from .workloads import ModelDims

LAYER_KEYS = ("w_qkv", "b_qkv", "w_o", "b_o", "ln1_g", "ln1_b",
              "w_1", "b_1", "w_2", "b_2", "ln2_g", "ln2_b")


def layer_shapes(d: ModelDims) -> dict[str, tuple[int, ...]]:
    m, f = d.d_model, d.d_ffn
    return {"w_qkv": (3 * m, m), "b_qkv": (3 * m,), "w_o": (m, m), "b_o": (m,),
            "ln1_g": (m,), "ln1_b": (m,), "w_1": (f, m), "b_1": (f,),
            "w_2": (m, f), "b_2": (m,), "ln2_g": (m,), "ln2_b": (m,)}


def blob_layout(d: ModelDims) -> list[tuple[str, tuple[int, ...]]]:
    m = d.d_model
    out = [("tok_emb", (d.vocab, m)), ("pos_emb", (d.max_pos, m)), ("emb_ln_g", (m,)), ("emb_ln_b", (m,))]
    ls = layer_shapes(d)
    for i in range(d.n_layers):
        for k in LAYER_KEYS:
            out.append((f"l{i}.{k}", ls[k]))
    out += [("cls_w", (d.n_labels, m)), ("cls_b", (d.n_labels,))]
    return out


def blob_size(d: ModelDims) -> int:
    return int(sum(int(np.prod(s)) for _, s in blob_layout(d)))


def make_weights(d: ModelDims, seed: int = 2002, o_bias_k: float = 3.5,
                 random_affine: bool = False) -> dict[str, np.ndarray]:
    rng = np.random.default_rng(seed)
    w: dict[str, np.ndarray] = {}
    for name, shape in blob_layout(d):
        base = name.split(".")[-1]
        if base.startswith("ln") or base.startswith("emb_ln"):
            if base.endswith("_g"):
                w[name] = (np.ones(shape, np.float32) if not random_affine
                           else (1.0 + 0.1 * rng.standard_normal(shape, dtype=np.float32)))
            else:
                w[name] = (np.zeros(shape, np.float32) if not random_affine
                           else 0.02 * rng.standard_normal(shape, dtype=np.float32))
        elif base.startswith("b_") or base == "cls_b":
            w[name] = (np.zeros(shape, np.float32) if not random_affine
                       else 0.02 * rng.standard_normal(shape, dtype=np.float32))
        else:
            w[name] = (0.02 * rng.standard_normal(shape, dtype=np.float32)).astype(np.float32)
    w["cls_b"] = w["cls_b"].copy()
    w["cls_b"][0] += np.float32(o_bias_k * 0.02 * np.sqrt(d.d_model))
    return w


def pack_blob(d: ModelDims, w: dict[str, np.ndarray]) -> np.ndarray:
    parts = []
    for name, shape in blob_layout(d):
        a = np.ascontiguousarray(w[name], dtype=np.float32)
        if a.shape != tuple(shape):
            raise ValueError(f"{name}: shape {a.shape} != {shape}")
        parts.append(a.reshape(-1))
    return np.concatenate(parts)


def make_key(seed: int = 3003, length: int = 32) -> bytes:
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=length, dtype=np.uint8).tobytes()
