"""Pins of the oracle's relative-position bias (CPU only): the library attention with an
additive float mask, a closed form that isolates each query with itself, the
orientation of the table (key minus query) by a closed form, and the zero table."""
import math

import numpy as np
import torch
import torch.nn.functional as F

from oracle import inpaint_oracle as O
from paper_2509_10466_gb300 import synthetic as S
from paper_2509_10466_gb300.config import ModelConfig

DT = torch.float64


def rand_qkv(N, d, seed):
    g = torch.Generator().manual_seed(seed)
    return torch.randn(N, 3 * d, generator=g, dtype=DT), g


def test_relpos_attention_matches_library_sdpa():
    heads, dh, Ht, Wt = 2, 32, 16, 24
    d, N = heads * dh, Ht * Wt
    qkv, g = rand_qkv(N, d, 3)
    valid = (torch.rand(N, generator=g) < 0.5).to(torch.uint8)
    table = torch.randn(heads, 15, 15, generator=g, dtype=DT)
    for offset in (0, 4):
        widx = O.window_index(Ht, Wt, 8, offset)
        o, _ = O.window_attention(qkv, valid, heads, widx, table)
        bias = O.relpos_bias(table, 8)                                # [h, 64, 64]
        for wi in range(widx.shape[0]):
            slots = torch.nonzero(widx[wi] >= 0).flatten()
            toks = widx[wi][slots]
            ok = valid[toks] != 0
            if not ok.any():
                continue
            q = qkv[toks, :d].reshape(-1, heads, dh).transpose(0, 1)
            k = qkv[toks, d:2 * d].reshape(-1, heads, dh).transpose(0, 1)
            v = qkv[toks, 2 * d:].reshape(-1, heads, dh).transpose(0, 1)
            m = bias[:, slots][:, :, slots].clone()
            m[:, :, ~ok] = float("-inf")
            ref = F.scaled_dot_product_attention(q, k, v, attn_mask=m)
            assert torch.allclose(o[toks], ref.transpose(0, 1).reshape(len(toks), d), rtol=1e-12, atol=1e-12)


def test_self_only_table_returns_each_tokens_own_value():
    heads, dh, Ht, Wt = 1, 32, 8, 16
    d, N = heads * dh, Ht * Wt
    qkv, _ = rand_qkv(N, d, 5)
    valid = torch.ones(N, dtype=torch.uint8)
    table = torch.full((1, 15, 15), -1e4, dtype=DT)
    table[0, 7, 7] = 0.0
    o, _ = O.window_attention(qkv, valid, heads, O.window_index(Ht, Wt, 8, 0), table)
    assert torch.equal(o, qkv[:, 2 * d:])


def test_table_is_indexed_by_key_minus_query():
    """Zero queries: all scores are the bias.  A table that favours the key one row below
    the query gives that key weight e / (e + 63) in an all-valid window (closed form)."""
    heads, dh = 1, 32
    d, N = 32, 64
    qkv, _ = rand_qkv(N, d, 9)
    qkv[:, :d] = 0.0
    table = torch.zeros(1, 15, 15, dtype=DT)
    table[0, 8, 7] = 1.0                                              # (key row - query row) = +1
    o, _ = O.window_attention(qkv, torch.ones(N, dtype=torch.uint8), heads, O.window_index(8, 8, 8, 0), table)
    v = qkv[:, 2 * d:]
    t = 3 * 8 + 4                                                     # row 3, column 4
    below = 4 * 8 + 4
    ref = (math.e * v[below] + (v.sum(0) - v[below])) / (math.e + 63)
    assert torch.allclose(o[t], ref, rtol=1e-13, atol=1e-13)
    # the bottom row has no key below it: a plain mean
    t = 7 * 8 + 2
    assert torch.allclose(o[t], v.mean(0), rtol=1e-13, atol=1e-13)


def test_zero_table_is_the_model_without_bias():
    cfg = ModelConfig(dim=64, heads=2, window=8, blocks=2, mlp_ratio=2, pos_bias=1)
    cfg0 = ModelConfig(dim=64, heads=2, window=8, blocks=2, mlp_ratio=2)
    w = S.make_weights(cfg, seed=4, perturb=True).astype(np.float64)
    # remove the tables from the blob, and zero them in the biased one
    names = S.param_shapes(cfg)
    parts, pos = [], 0
    wz = w.copy()
    for name, shape in names:
        n = int(np.prod(shape))
        if name.endswith("relpos"):
            wz[pos:pos + n] = 0
        else:
            parts.append(w[pos:pos + n])
        pos += n
    w0 = np.concatenate(parts)
    x = torch.from_numpy(S.make_frames(1, 64, 96, seed=2))
    hole = torch.from_numpy(S.make_hole(1, 64, 96, "polygons", seed=2))
    a = O.forward(x, hole, torch.from_numpy(wz), cfg)
    b = O.forward(x, hole, torch.from_numpy(w0), cfg0)
    assert torch.allclose(a["out"], b["out"], rtol=0, atol=1e-13)
