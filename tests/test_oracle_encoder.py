"""Pins for the FP64 encoder oracle.

1. Independent formulation: PyTorch's own post-LayerNorm
   ``nn.TransformerEncoderLayer`` (GELU, no dropout, eps 1e-5) in float64 on
   the CPU, loaded with the same weights, gives the same logits to ~1e-12.
   It fixes the block order, the Q/K/V column layout of the packed
   projection, the head split and the 1/sqrt(dh) scale.
2. Closed forms: a one-token sequence attends only to itself (its attention
   output is its V row); zero classifier weights give logits equal to the
   bias; LayerNorm rows have mean 0 and variance 1; softmax rows sum to 1.
3. Invariance: a record's logits do not depend on windows when it fits one
   window, and each window's logits are those of the window's tokens run
   alone.
4. Windows: the owner of each token, checked against the closed form
   floor((t - (W - S) / 2) / S) clamped to the window range, for many (L, W, S).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import encoder as E

DIMS = synth.ModelDims(vocab=300, d_model=64, n_heads=4, d_ffn=128, n_layers=2, n_labels=9, max_pos=64)


@pytest.fixture(scope="module")
def weights():
    return synth.make_weights(DIMS, seed=11, random_affine=True)


def torch_reference(ids, w, dims):
    d = dims.d_model
    x = torch.tensor(w["tok_emb"], dtype=torch.float64)[ids] + torch.tensor(w["pos_emb"], dtype=torch.float64)[:len(ids)]
    x = torch.nn.functional.layer_norm(x, (d,), torch.tensor(w["emb_ln_g"], dtype=torch.float64),
                                       torch.tensor(w["emb_ln_b"], dtype=torch.float64), eps=1e-5)
    x = x.unsqueeze(0)
    for i in range(dims.n_layers):
        layer = torch.nn.TransformerEncoderLayer(d, dims.n_heads, dims.d_ffn, dropout=0.0, activation="gelu",
                                                 layer_norm_eps=1e-5, batch_first=True, norm_first=False,
                                                 dtype=torch.float64)
        p = f"l{i}."
        sd = {
            "self_attn.in_proj_weight": w[p + "w_qkv"], "self_attn.in_proj_bias": w[p + "b_qkv"],
            "self_attn.out_proj.weight": w[p + "w_o"], "self_attn.out_proj.bias": w[p + "b_o"],
            "linear1.weight": w[p + "w_1"], "linear1.bias": w[p + "b_1"],
            "linear2.weight": w[p + "w_2"], "linear2.bias": w[p + "b_2"],
            "norm1.weight": w[p + "ln1_g"], "norm1.bias": w[p + "ln1_b"],
            "norm2.weight": w[p + "ln2_g"], "norm2.bias": w[p + "ln2_b"],
        }
        layer.load_state_dict({k: torch.tensor(v, dtype=torch.float64) for k, v in sd.items()})
        layer.eval()
        with torch.no_grad():
            x = layer(x)
    x = x[0]
    return (x @ torch.tensor(w["cls_w"], dtype=torch.float64).T + torch.tensor(w["cls_b"], dtype=torch.float64)).numpy()


@pytest.mark.parametrize("L", [1, 2, 7, 33, 64])
def test_matches_torch_transformer_layer(weights, L):
    rng = np.random.default_rng(L)
    ids = rng.integers(1, DIMS.vocab, size=L)
    enc = E.Encoder(DIMS, weights)
    got = enc.logits(ids)
    ref = torch_reference(torch.tensor(ids), weights, DIMS)
    assert np.max(np.abs(got - ref)) < 1e-11


def test_c1_shape_matches_torch():
    w = synth.make_weights(synth.C1.dims, seed=5, random_affine=True)
    rng = np.random.default_rng(0)
    ids = rng.integers(1, 8192, size=120)
    got = E.Encoder(synth.C1.dims, w).logits(ids)
    ref = torch_reference(torch.tensor(ids), w, synth.C1.dims)
    assert np.max(np.abs(got - ref)) < 1e-11


def test_single_token_attention_is_v(weights):
    dims = synth.ModelDims(vocab=300, d_model=64, n_heads=4, d_ffn=128, n_layers=1, n_labels=9, max_pos=64)
    w = {k: v for k, v in weights.items() if not k.startswith("l1.")}
    enc = E.Encoder(dims, w)
    x0 = E.layer_norm(enc.w["tok_emb"][[5]] + enc.w["pos_emb"][[0]], enc.w["emb_ln_g"], enc.w["emb_ln_b"])
    v = (x0 @ enc.w["l0.w_qkv"].T + enc.w["l0.b_qkv"])[:, 128:192]
    x1 = E.layer_norm(x0 + v @ enc.w["l0.w_o"].T + enc.w["l0.b_o"], enc.w["l0.ln1_g"], enc.w["l0.ln1_b"])
    x2 = E.layer_norm(x1 + E.gelu(x1 @ enc.w["l0.w_1"].T + enc.w["l0.b_1"]) @ enc.w["l0.w_2"].T + enc.w["l0.b_2"],
                      enc.w["l0.ln2_g"], enc.w["l0.ln2_b"])
    assert np.max(np.abs(enc.hidden([5]) - x2)) < 1e-13


def test_zero_classifier_gives_bias(weights):
    w = dict(weights)
    w["cls_w"] = np.zeros_like(w["cls_w"])
    enc = E.Encoder(DIMS, w)
    lg = enc.logits(np.arange(1, 30))
    assert np.array_equal(lg, np.broadcast_to(w["cls_b"].astype(np.float64), lg.shape))


def test_layernorm_and_softmax_closed_forms():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((50, 96)) * 3 + 1
    y = E.layer_norm(x, np.ones(96), np.zeros(96))
    assert np.allclose(y.mean(-1), 0, atol=1e-12)
    assert np.allclose(y.var(-1), 1 - 1e-5 / (x.var(-1) + 1e-5), atol=1e-12)
    s = E.softmax(rng.standard_normal((7, 13)) * 10)
    assert np.allclose(s.sum(-1), 1, atol=1e-14) and (s > 0).all()
    g = E.gelu(np.array([0.0, 1.0, -1.0, 10.0]))
    assert g[0] == 0 and abs(g[3] - 10) < 1e-12 and abs(g[1] - g[2] - 1.0) < 1e-15


def test_windows_invariance(weights):
    enc = E.Encoder(DIMS, weights)
    rng = np.random.default_rng(4)
    short = rng.integers(1, 300, size=40).tolist()
    assert np.array_equal(E.record_logits(enc, short, 64, 48), enc.logits(short))
    long = rng.integers(1, 300, size=150).tolist()
    W, S = 64, 48
    lg = E.record_logits(enc, long, W, S)
    starts = E.window_starts(150, W, S)
    owner = E.window_owner(150, W, S)
    for wi, s in enumerate(starts):
        ref = enc.logits(long[s:min(s + W, 150)])
        for t in range(150):
            if owner[t] == wi:
                assert np.array_equal(lg[t], ref[t - s])


def test_window_owner_closed_form():
    for W in range(2, 13):
        for S in range(1, W + 1):
            if (W - S) % 2:
                continue
            half = (W - S) // 2
            for L in range(1, 60):
                starts = E.window_starts(L, W, S)
                assert starts[-1] + W >= L and all(b - a == S for a, b in zip(starts, starts[1:]))
                assert len(starts) == 1 or starts[-2] + W < L
                owner = E.window_owner(L, W, S)
                for t in range(L):
                    w = min(max((t - half) // S, 0), len(starts) - 1)
                    assert owner[t] == w
                    assert starts[w] <= t < starts[w] + W


def test_too_long_without_windows(weights):
    enc = E.Encoder(DIMS, weights)
    with pytest.raises(E.RecordTooLong):
        enc.logits(list(range(1, 66)))
