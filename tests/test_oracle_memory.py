"""Pins of the oracle's temporal-memory attention (CPU only).

The memory reading: with m memory slots the odd blocks are temporal, and their queries
also attend to the keys / values that previous frames of the stream produced in the
same block at the same window positions (where those frames' tokens were usable keys).
Each test ties the oracle to something other than itself: an invariant of softmax
attention (duplicated keys change nothing), a library routine (torch's scaled dot
product attention with a boolean mask), a closed form (a single usable key returns its
value) and the reduction to the spatial model when no memory is present.
"""
import numpy as np
import torch
import torch.nn.functional as F

from oracle import inpaint_oracle as O
from paper_2509_10466_gb300 import synthetic as S
from paper_2509_10466_gb300.config import ModelConfig

DT = torch.float64


def mem_cfg(**kw):
    base = dict(dim=64, heads=2, window=8, blocks=4, mlp_ratio=2, mem_slots=2)
    base.update(kw)
    return ModelConfig(**base)


def frame(seed, H=64, W=96, kind="ellipse_strokes", area=None):
    x = torch.from_numpy(S.make_frames(1, H, W, seed=seed))
    hole = torch.from_numpy(S.make_hole(1, H, W, kind, seed=seed, area=area))
    return x, hole


def weights(cfg, seed=3):
    return torch.from_numpy(S.make_weights(cfg, seed=seed, perturb=True).astype(np.float64))


def test_no_memory_is_the_spatial_model():
    cfg = mem_cfg()
    w = weights(cfg)
    x, hole = frame(1)
    r_mem = O.forward(x, hole, w, cfg)
    r_sp = O.forward(x, hole, w, mem_cfg(mem_slots=0))
    assert torch.allclose(r_mem["out"], r_sp["out"], rtol=0, atol=1e-13)
    assert torch.equal(r_mem["masks"], r_sp["masks"])
    # the memory tensor covers exactly the temporal blocks
    assert sorted(r_mem["memory"][0]) == [1, 3]


def test_memory_of_the_same_frame_changes_nothing():
    """Memory slots holding the frame's own keys, values and key masks duplicate every key
    of every temporal window; softmax attention over duplicated keys is unchanged, so the
    whole pass must reproduce the pass without memory (holes included)."""
    cfg = mem_cfg()
    w = weights(cfg)
    x, hole = frame(2, area=(0.3, 0.5))
    r0 = O.forward(x, hole, w, cfg)
    own = r0["memory"][0]
    r1 = O.forward(x, hole, w, cfg, mem=[[own, own]])
    assert torch.allclose(r1["out"], r0["out"], rtol=0, atol=1e-11)
    assert torch.equal(r1["masks"], r0["masks"])


def test_memory_attention_matches_library_sdpa():
    g = torch.Generator().manual_seed(7)
    heads, dh, Ht, Wt = 2, 32, 16, 24
    d, N = heads * dh, Ht * Wt
    qkv = torch.randn(N, 3 * d, generator=g, dtype=DT)
    valid = (torch.rand(N, generator=g) < 0.4).to(torch.uint8)
    mem = []
    for j in range(2):
        kv = torch.randn(N, 2 * d, generator=g, dtype=DT)
        mask = (torch.rand(N, generator=g) < 0.5).to(torch.uint8)
        mem.append((kv, mask))
    for offset in (0, 4):
        widx = O.window_index(Ht, Wt, 8, offset)
        o, nxt = O.window_attention_mem(qkv, valid, heads, widx, mem + [None])
        for wi in range(widx.shape[0]):
            toks = widx[wi][widx[wi] >= 0]
            keys = [(qkv[toks, d:2 * d], qkv[toks, 2 * d:], valid[toks] != 0)]
            keys += [(kv[toks, :d], kv[toks, d:], mask[toks] != 0) for kv, mask in mem]
            k = torch.cat([a for a, _, _ in keys])
            v = torch.cat([b for _, b, _ in keys])
            ok = torch.cat([c for _, _, c in keys])
            if not ok.any():
                assert torch.all(o[toks] == 0) and torch.all(nxt[toks] == 0)
                continue
            assert torch.all(nxt[toks] == 1)
            q = qkv[toks, :d].reshape(-1, heads, dh).transpose(0, 1)
            kh = k.reshape(-1, heads, dh).transpose(0, 1)
            vh = v.reshape(-1, heads, dh).transpose(0, 1)
            ref = F.scaled_dot_product_attention(q, kh, vh, attn_mask=ok[None, None, :].expand(heads, len(toks), -1))
            assert torch.allclose(o[toks], ref.transpose(0, 1).reshape(len(toks), d), rtol=1e-12, atol=1e-12)


def test_memory_fills_a_window_without_current_keys():
    """A window whose current tokens are all hole but whose memory holds exactly one usable
    key returns that key's value for every query (softmax over one key) and becomes valid."""
    g = torch.Generator().manual_seed(11)
    heads, dh, Ht, Wt = 1, 32, 8, 8
    d, N = heads * dh, Ht * Wt
    qkv = torch.randn(N, 3 * d, generator=g, dtype=DT)
    valid = torch.zeros(N, dtype=torch.uint8)
    kv = torch.randn(N, 2 * d, generator=g, dtype=DT)
    mask = torch.zeros(N, dtype=torch.uint8)
    mask[37] = 1
    widx = O.window_index(Ht, Wt, 8, 0)
    o, nxt = O.window_attention_mem(qkv, valid, heads, widx, [None, (kv, mask)])
    assert torch.equal(o, kv[37, d:].expand(N, d))
    assert torch.all(nxt == 1)
    # and without it the window stays empty
    o0, nxt0 = O.window_attention_mem(qkv, valid, heads, widx, [None, None])
    assert torch.all(o0 == 0) and torch.all(nxt0 == 0)


def test_memory_lets_a_fully_hidden_window_become_valid_in_the_pass():
    """In the pass, a temporal block turns every real token valid whose window has usable
    memory keys; with a fully hidden frame the token masks after block 1 therefore equal
    1 where the previous frame's block-1 key mask covers the window, and stay 0 without
    memory."""
    cfg = mem_cfg(blocks=2)
    w = weights(cfg)
    x, _ = frame(4)
    hole_all = torch.ones(1, 64, 96, dtype=torch.uint8)
    hole_none = torch.zeros(1, 64, 96, dtype=torch.uint8)
    prev = O.forward(x, hole_none, w, cfg)["memory"][0]
    r_mem = O.forward(x, hole_all, w, cfg, mem=[[prev, None]])
    r_nomem = O.forward(x, hole_all, w, cfg)
    assert int(r_nomem["masks"][2].sum()) == 0
    assert torch.all(r_mem["masks"][2] == 1)
    assert torch.all(r_mem["masks"][1] == 0)  # block 0 is spatial: nothing to attend to
