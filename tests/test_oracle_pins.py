"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test checks the oracle against an independent library routine, a closed form, an
invariant of the method, a hand-derived fixture or brute force, so that a dropped term,
a wrong sign, index or transposed operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import inpaint_oracle as O
from paper_2509_10466_gb300 import synthetic as S
from paper_2509_10466_gb300.config import ModelConfig

DT = torch.float64
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_cfg(**kw):
    base = dict(dim=64, heads=2, window=8, blocks=2, mlp_ratio=2)
    base.update(kw)
    return ModelConfig(**base)


# ----------------------------------------------------------------------------- elementary steps

def test_layer_norm_matches_library():
    g = torch.Generator().manual_seed(0)
    x = torch.randn(37, 96, generator=g, dtype=DT) * 3 + 1
    w = torch.randn(96, generator=g, dtype=DT)
    b = torch.randn(96, generator=g, dtype=DT)
    ref = F.layer_norm(x, (96,), w, b, eps=1e-5)
    assert torch.allclose(O.layer_norm(x, w, b), ref, rtol=1e-13, atol=1e-13)


def test_gelu_closed_form():
    xs = torch.linspace(-6, 6, 241, dtype=DT)
    ref = torch.tensor([0.5 * v * (1 + math.erf(v / math.sqrt(2))) for v in xs.tolist()], dtype=DT)
    assert torch.allclose(O.gelu(xs), ref, rtol=0, atol=1e-15)
    assert torch.allclose(O.gelu(xs), F.gelu(xs, approximate="none"), rtol=0, atol=1e-15)


def test_conv3x3_matches_library():
    g = torch.Generator().manual_seed(1)
    f = torch.randn(2, 5, 9, 11, generator=g, dtype=DT)
    w = torch.randn(7, 5, 3, 3, generator=g, dtype=DT)
    b = torch.randn(7, generator=g, dtype=DT)
    assert torch.allclose(O.conv3x3(f, w, b), F.conv2d(f, w, b, padding=1), rtol=1e-12, atol=1e-12)


def test_upsample_matches_library():
    f = torch.randn(2, 3, 5, 7, dtype=DT)
    assert torch.equal(O.upsample2(f), F.interpolate(f, scale_factor=2, mode="nearest"))


def test_patch_embed_is_strided_conv():
    g = torch.Generator().manual_seed(2)
    inp = torch.randn(2, 4, 32, 64, generator=g, dtype=DT)
    w = torch.randn(24, 4, 4, 4, generator=g, dtype=DT)
    b = torch.randn(24, generator=g, dtype=DT)
    ref = F.conv2d(inp, w, b, stride=4)                      # [2, 24, 8, 16]
    got = O.patch_embed(inp, w, b, 4).reshape(2, 8, 16, 24).permute(0, 3, 1, 2)
    assert torch.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_model_input_zeroes_hole_and_appends_mask():
    x = torch.rand(1, 3, 32, 32, dtype=DT)
    hole = (torch.rand(1, 32, 32) < 0.3).to(torch.uint8)
    xp, hp = O.pad_inputs(x, hole, 32)
    inp = O.model_input(xp, hp)
    assert inp.shape == (1, 4, 32, 32)
    assert torch.all(inp[:, :3][hp[:, None].expand(1, 3, 32, 32) == 1] == 0)
    assert torch.equal(inp[:, 3], (1 - hole).to(DT))


def test_pad_inputs_marks_pad_as_hole():
    x = torch.rand(1, 3, 40, 50, dtype=DT)
    hole = torch.zeros(1, 40, 50, dtype=torch.uint8)
    xp, hp = O.pad_inputs(x, hole, 32)
    assert xp.shape == (1, 3, 64, 64) and hp.shape == (1, 64, 64)
    assert torch.all(hp[:, 40:] == 1) and torch.all(hp[:, :, 50:] == 1) and torch.all(hp[:, :40, :50] == 0)
    assert torch.all(xp[:, :, 40:] == 0)


def test_token_mask_init_any_known_pixel():
    hole = torch.ones(1, 32, 32, dtype=torch.uint8)
    hole[0, 5, 9] = 0          # one known pixel -> token (1, 2) of the 8x8 token grid
    v0 = O.token_mask_init(hole, 4).reshape(8, 8)
    expect = torch.zeros(8, 8, dtype=torch.uint8)
    expect[1, 2] = 1
    assert torch.equal(v0, expect)


# ----------------------------------------------------------------------------- windows and masks

@pytest.mark.parametrize("Ht,Wt,off", [(8, 8, 0), (16, 24, 0), (16, 24, 4), (8, 8, 4), (24, 8, 4)])
def test_windows_partition_the_grid(Ht, Wt, off):
    widx = O.window_index(Ht, Wt, 8, off)
    real = widx[widx >= 0]
    assert sorted(real.tolist()) == list(range(Ht * Wt))           # every token exactly once
    expect_n = (math.ceil((Ht + off) / 8)) * (math.ceil((Wt + off) / 8))
    assert widx.shape == (expect_n, 64)
    # a window's real tokens form one rectangle of rows x cols aligned to the offset grid
    for row in widx:
        toks = row[row >= 0]
        ys, xs = toks // Wt, toks % Wt
        assert len(set(((ys + off) // 8).tolist())) == 1 and len(set(((xs + off) // 8).tolist())) == 1


def _or_pool_rule(v, Ht, Wt, ws, off):
    """Independent closed form: window OR = max-pool over the offset grid, broadcast back."""
    g = v.reshape(-1, 1, Ht, Wt).to(DT)
    Hpad = math.ceil((Ht + off) / ws) * ws
    Wpad = math.ceil((Wt + off) / ws) * ws
    gp = F.pad(g, (off, Wpad - Wt - off, off, Hpad - Ht - off))     # void slots = 0: no effect on OR
    pooled = F.max_pool2d(gp, ws, ws)
    up = pooled.repeat_interleave(ws, 2).repeat_interleave(ws, 3)
    return up[:, 0, off:off + Ht, off:off + Wt].reshape(v.shape[0], -1).to(torch.uint8)


def test_mask_rule_exhaustive_4x4_window2():
    """All 2^16 token masks of a 4x4 grid with 2x2 windows, two blocks (second offset by 1)."""
    cfg = ModelConfig(dim=8, heads=1, window=2, blocks=2, mlp_ratio=1, patch=1, shift=1)
    codes = torch.arange(1 << 16)
    v0 = ((codes[:, None] >> torch.arange(16)[None, :]) & 1).to(torch.uint8)      # [65536, 16]
    hole = (1 - v0).reshape(-1, 4, 4)
    masks = O.token_masks(hole, cfg)                                              # [3, 65536, 16]
    assert torch.equal(masks[0], v0)
    exp1 = _or_pool_rule(v0, 4, 4, 2, 0)
    assert torch.equal(masks[1], exp1)
    exp2 = _or_pool_rule(exp1, 4, 4, 2, 1)
    assert torch.equal(masks[2], exp2)
    # invariants: monotone, all-valid is a fixed point, all-hole stays all-hole
    assert torch.all(masks[1] >= masks[0]) and torch.all(masks[2] >= masks[1])
    assert torch.all(masks[:, -1] == 1) and torch.all(masks[:, 0] == 0)


def test_mask_rule_brute_force_sets():
    """Brute force over python sets on random 16x24 grids, windows 8, offset 4 on odd blocks."""
    rng = np.random.default_rng(5)
    cfg = ModelConfig(dim=8, heads=1, window=8, blocks=3, mlp_ratio=1, patch=1, shift=1)
    for _ in range(20):
        v0 = (rng.random((16, 24)) < rng.uniform(0.0, 0.05)).astype(np.uint8)
        masks = O.token_masks(torch.from_numpy(1 - v0)[None], cfg)
        v = {(y, x) for y in range(16) for x in range(24) if v0[y, x]}
        for l in range(3):
            off = 4 if l % 2 else 0
            win = lambda y, x: ((y + off) // 8, (x + off) // 8)
            live = {win(y, x) for (y, x) in v}
            v = {(y, x) for y in range(16) for x in range(24) if win(y, x) in live}
            got = masks[l + 1, 0].reshape(16, 24)
            exp = torch.zeros(16, 24, dtype=torch.uint8)
            for (y, x) in v:
                exp[y, x] = 1
            assert torch.equal(got, exp)


def _read_golden_masks(path):
    with open(path) as f:
        lines = [ln.rstrip("\n") for ln in f if not ln.startswith("#")]
    hdr = lines[0].split()
    H, W = int(hdr[1]), int(hdr[2])
    grids = {}
    i = 1
    while i < len(lines):
        name = lines[i].strip()
        rows = lines[i + 1:i + 1 + H]
        grids[name] = torch.tensor([[1 if c == "X" else 0 for c in r] for r in rows], dtype=torch.uint8)
        i += 1 + H
    return H, W, grids


def test_mask_rule_golden_fixture():
    H, W, grids = _read_golden_masks(os.path.join(GOLDEN, "mask_rule_16x16.txt"))
    cfg = ModelConfig(dim=8, heads=1, window=8, blocks=3, mlp_ratio=1, patch=1, shift=1)
    masks = O.token_masks((1 - grids["v0"])[None], cfg)
    for l in range(4):
        assert torch.equal(masks[l, 0].reshape(H, W), grids[f"v{l}"]), f"v{l}"


# ----------------------------------------------------------------------------- attention

def _sdpa_window_reference(qkv, valid, heads, Ht, Wt, off):
    """Per-window library attention with a boolean key mask (independent window enumeration)."""
    N, d3 = qkv.shape
    d = d3 // 3
    dh = d // heads
    o = torch.zeros(N, d, dtype=DT)
    nxt = torch.zeros(N, dtype=torch.uint8)
    for wy0 in range(-off, Ht, 8):
        for wx0 in range(-off, Wt, 8):
            toks = [y * Wt + x for y in range(max(wy0, 0), min(wy0 + 8, Ht))
                    for x in range(max(wx0, 0), min(wx0 + 8, Wt))]
            if not toks:
                continue
            t = torch.tensor(toks)
            keymask = valid[t] != 0
            if not keymask.any():
                continue
            nxt[t] = 1
            q = qkv[t, :d].reshape(-1, heads, dh).transpose(0, 1)
            k = qkv[t, d:2 * d].reshape(-1, heads, dh).transpose(0, 1)
            v = qkv[t, 2 * d:].reshape(-1, heads, dh).transpose(0, 1)
            a = F.scaled_dot_product_attention(q, k, v, attn_mask=keymask[None, None, :].expand(heads, len(toks), len(toks)))
            o[t] = a.transpose(0, 1).reshape(-1, d)
    return o, nxt


@pytest.mark.parametrize("off", [0, 4])
@pytest.mark.parametrize("density", [0.0, 0.03, 0.3, 1.0])
def test_window_attention_matches_library(off, density):
    Ht, Wt, heads, d = 16, 24, 2, 64
    g = torch.Generator().manual_seed(int(density * 100) + off)
    qkv = torch.randn(Ht * Wt, 3 * d, generator=g, dtype=DT)
    valid = (torch.rand(Ht * Wt, generator=g) < density).to(torch.uint8)
    o, nxt = O.window_attention(qkv, valid, heads, O.window_index(Ht, Wt, 8, off))
    ro, rn = _sdpa_window_reference(qkv, valid, heads, Ht, Wt, off)
    assert torch.equal(nxt, rn)
    assert torch.allclose(o, ro, rtol=1e-12, atol=1e-12)


def test_attention_single_valid_key_returns_its_value():
    Ht = Wt = 8
    d, heads = 32, 1
    qkv = torch.randn(64, 3 * d, dtype=DT)
    valid = torch.zeros(64, dtype=torch.uint8)
    valid[19] = 1
    o, nxt = O.window_attention(qkv, valid, heads, O.window_index(Ht, Wt, 8, 0))
    assert torch.equal(o, qkv[19, 2 * d:].expand(64, d))
    assert torch.all(nxt == 1)


def test_attention_no_valid_key_outputs_zero():
    qkv = torch.randn(64, 96, dtype=DT)
    o, nxt = O.window_attention(qkv, torch.zeros(64, dtype=torch.uint8), 1, O.window_index(8, 8, 8, 0))
    assert torch.all(o == 0) and torch.all(nxt == 0)


def test_attention_brute_force_python():
    """Pure-python softmax attention over a 4x4 grid with one 4x4 window and random key mask."""
    rng = np.random.default_rng(3)
    Ht = Wt = 4
    heads, dh = 2, 3
    d = heads * dh
    qkv = rng.standard_normal((16, 3 * d))
    valid = (rng.random(16) < 0.4).astype(np.uint8)
    valid[0] = 1
    o, _ = O.window_attention(torch.from_numpy(qkv), torch.from_numpy(valid), heads, O.window_index(Ht, Wt, 4, 0))
    for t in range(16):
        for h in range(heads):
            q = qkv[t, h * dh:(h + 1) * dh]
            scores = {s: sum(q[i] * qkv[s, d + h * dh + i] for i in range(dh)) / math.sqrt(dh)
                      for s in range(16) if valid[s]}
            mx = max(scores.values())
            z = sum(math.exp(v - mx) for v in scores.values())
            for i in range(dh):
                ref = sum(math.exp(scores[s] - mx) / z * qkv[s, 2 * d + h * dh + i] for s in scores)
                assert abs(float(o[t, h * dh + i]) - ref) < 1e-12


# ----------------------------------------------------------------------------- whole pass

def _library_network(x, hole, flat, cfg):
    """The same network assembled from torch library layers (independent composition)."""
    w = {}
    pos = 0
    for name, shape in S.param_shapes(cfg):
        n = int(np.prod(shape))
        w[name] = flat[pos:pos + n].reshape(shape)
        pos += n
    B, _, H, W = x.shape
    mult = cfg.patch * cfg.window
    Hp, Wp = -(-H // mult) * mult, -(-W // mult) * mult
    xp = F.pad(x, (0, Wp - W, 0, Hp - H))
    known = F.pad((hole == 0).to(DT), (0, Wp - W, 0, Hp - H))          # pad counts as hole
    inp = torch.cat([xp * known[:, None], known[:, None]], 1)
    feat = F.conv2d(inp, w["embed.w"], w["embed.b"], stride=cfg.patch)  # [B, d, Ht, Wt]
    Ht, Wt = feat.shape[2:]
    v = (F.max_pool2d(known[:, None], cfg.patch) > 0).to(DT)[:, 0]      # [B, Ht, Wt]
    tok = feat.permute(0, 2, 3, 1)                                      # [B, Ht, Wt, d]
    d, heads = cfg.dim, cfg.heads
    for l in range(cfg.blocks):
        off = cfg.window // 2 if (cfg.shift and l % 2) else 0
        y = F.layer_norm(tok, (d,), w[f"blk{l}.ln1.g"], w[f"blk{l}.ln1.b"], eps=1e-5)
        qkv = F.linear(y, w[f"blk{l}.qkv.w"].T, w[f"blk{l}.qkv.b"])
        o = torch.zeros_like(tok)
        vn = torch.zeros_like(v)
        for b in range(B):
            ob, nb = _sdpa_window_reference(qkv[b].reshape(-1, 3 * d), v[b].reshape(-1), heads, Ht, Wt, off)
            o[b] = ob.reshape(Ht, Wt, d)
            vn[b] = nb.reshape(Ht, Wt).to(DT)
        v = vn
        tok = tok + F.linear(o, w[f"blk{l}.proj.w"].T, w[f"blk{l}.proj.b"])
        y2 = F.layer_norm(tok, (d,), w[f"blk{l}.ln2.g"], w[f"blk{l}.ln2.b"], eps=1e-5)
        hid = F.gelu(F.linear(y2, w[f"blk{l}.fc1.w"].T, w[f"blk{l}.fc1.b"]))
        tok = tok + F.linear(hid, w[f"blk{l}.fc2.w"].T, w[f"blk{l}.fc2.b"])
    f = F.layer_norm(tok, (d,), w["lnf.g"], w["lnf.b"], eps=1e-5).permute(0, 3, 1, 2)
    f = F.gelu(F.conv2d(F.interpolate(f, scale_factor=2, mode="nearest"), w["dec1.w"], w["dec1.b"], padding=1))
    f = F.gelu(F.conv2d(F.interpolate(f, scale_factor=2, mode="nearest"), w["dec2.w"], w["dec2.b"], padding=1))
    pred = F.conv2d(f, w["head.w"], w["head.b"], padding=1)[:, :, :H, :W]
    hm = (hole != 0)[:, None].expand_as(x)
    return x * (~hm) + pred * hm, pred


@pytest.mark.parametrize("H,W,shift", [(64, 96, 1), (70, 45, 1), (64, 64, 0)])
def test_forward_matches_library_composition(H, W, shift):
    cfg = small_cfg(shift=shift, blocks=3)
    flat = torch.from_numpy(S.make_weights(cfg, seed=7, perturb=True)).to(DT)
    x = torch.from_numpy(S.make_frames(2, H, W, seed=1)).to(DT)
    hole = torch.from_numpy(S.make_hole(2, H, W, "ellipse_strokes", seed=1, area=(0.2, 0.6)))
    res = O.forward(x, hole, flat, cfg)
    out_ref, pred_ref = _library_network(x, hole, flat, cfg)
    assert torch.allclose(res["pred"], pred_ref, rtol=1e-10, atol=1e-12)
    assert torch.allclose(res["out"], out_ref, rtol=1e-10, atol=1e-12)


def test_known_pixels_pass_through_exactly_and_hole_invariance():
    cfg = small_cfg()
    flat = S.make_weights(cfg, seed=3, perturb=True)
    x = torch.from_numpy(S.make_frames(1, 64, 64, seed=2)).to(DT)
    hole = torch.from_numpy(S.make_hole(1, 64, 64, "ellipse_strokes", seed=2))
    r1 = O.forward(x, hole, flat, cfg)
    known = (hole == 0)[:, None].expand_as(x)
    assert torch.equal(r1["out"][known], x[known])
    x2 = x.clone()
    noise = torch.rand_like(x2) * 100 - 50
    x2[~known] = noise[~known]
    r2 = O.forward(x2, hole, flat, cfg)
    assert torch.equal(r1["out"][~known], r2["out"][~known])
    assert torch.equal(r1["masks"], r2["masks"])
    # composite = m*x + (1-m)*pred for finite pred
    m = known.to(DT)
    assert torch.equal(r1["out"], m * x + (1 - m) * r1["pred"])


def test_all_hole_frame_has_no_attention():
    """All-hole frame: masks stay 0 and the qkv weights cannot influence the output."""
    cfg = small_cfg()
    flat = S.make_weights(cfg, seed=4, perturb=True)
    x = torch.from_numpy(S.make_frames(1, 64, 64, seed=3)).to(DT)
    hole = torch.ones(1, 64, 64, dtype=torch.uint8)
    r1 = O.forward(x, hole, flat, cfg)
    assert torch.all(r1["masks"] == 0)
    flat2 = flat.copy()
    pos = 0
    for name, shape in S.param_shapes(cfg):
        n = int(np.prod(shape))
        if ".qkv." in name:
            flat2[pos:pos + n] = np.random.default_rng(0).standard_normal(n)
        pos += n
    r2 = O.forward(x, hole, flat2, cfg)
    assert torch.equal(r1["out"], r2["out"])
    assert torch.equal(r1["out"], r1["pred"])


def test_no_hole_frame_is_identity():
    cfg = small_cfg()
    flat = S.make_weights(cfg, seed=4)
    x = torch.from_numpy(S.make_frames(1, 64, 64, seed=3)).to(DT)
    res = O.forward(x, torch.zeros(1, 64, 64, dtype=torch.uint8), flat, cfg)
    assert torch.equal(res["out"], x)
    assert torch.all(res["masks"] == 1)


def test_blob_format_matches_generator():
    for cfg in (small_cfg(), ModelConfig(256, 8, 8, 8, 4), ModelConfig(32, 1, 8, 1, 4), ModelConfig(192, 6, 8, 6, 4)):
        assert O.num_params(cfg) == S.num_params(cfg)
        flat = torch.zeros(S.num_params(cfg), dtype=DT)
        O.unpack(flat, cfg)
        with pytest.raises(ValueError):
            O.unpack(torch.zeros(S.num_params(cfg) + 1, dtype=DT), cfg)


# ----------------------------------------------------------------------------- loss and gradient

def test_l1_hole_loss_closed_form():
    out = torch.tensor([[[[0.5, 0.2], [0.9, 0.1]]]] * 1, dtype=DT).expand(1, 3, 2, 2).clone()
    tgt = torch.zeros_like(out)
    tgt[:, 1] = 1.0
    hole = torch.tensor([[[1, 0], [1, 0]]], dtype=torch.uint8)
    loss, grad = O.l1_hole_loss(out, tgt, hole)
    # hole pixels: (0,0) value .5 and (1,0) value .9; channels 0,2 vs 0 and channel 1 vs 1
    expect = ((0.5 + 0.5 + 0.5) + (0.9 + 0.1 + 0.9)) / (3 * 2)
    assert abs(float(loss) - expect) < 1e-15
    assert torch.all(grad[:, :, :, 1] == 0)
    assert float(grad[0, 1, 0, 0]) == -1 / 6 and float(grad[0, 0, 0, 0]) == 1 / 6
    z, gz = O.l1_hole_loss(out, tgt, torch.zeros_like(hole))
    assert float(z) == 0 and torch.all(gz == 0)


def test_weight_vjp_agrees_with_loss_gradient():
    cfg = small_cfg(dim=32, heads=1, blocks=1, mlp_ratio=4)
    flat = S.make_weights(cfg, seed=9, perturb=True)
    x = S.make_frames(1, 64, 64, seed=9)
    hole = S.make_hole(1, 64, 64, "ellipse_strokes", seed=9)
    tgt = S.make_target(1, 64, 64, seed=9)
    loss, g1 = O.loss_and_grad(x, hole, tgt, flat, cfg)
    out = O.forward(x, hole, flat, cfg)["out"]
    _, gout = O.l1_hole_loss(out, tgt, hole)
    g2 = O.weight_vjp(x, hole, gout, flat, cfg)
    assert torch.allclose(g1, g2, rtol=1e-12, atol=1e-15)


@pytest.mark.slow
def test_gradient_central_finite_differences():
    """FP64 central differences on the 64x64, 1-block, d32 (1 head) instance."""
    cfg = ModelConfig(dim=32, heads=1, window=8, blocks=1, mlp_ratio=4)
    flat = S.make_weights(cfg, seed=11, perturb=True).astype(np.float64)
    x = S.make_frames(1, 64, 64, seed=11)
    hole = S.make_hole(1, 64, 64, "ellipse_strokes", seed=11)
    tgt = S.make_target(1, 64, 64, seed=11)
    out = O.forward(x, hole, flat, cfg)["out"]
    gap = (out - torch.from_numpy(tgt).to(DT)).abs()[torch.from_numpy(hole != 0)[:, None].expand_as(out)]
    assert float(gap.min()) > 1e-4, "seed lands on an L1 kink; pick another"
    _, grad = O.loss_and_grad(x, hole, tgt, flat, cfg)
    rng = np.random.default_rng(0)
    pos = 0
    picks = []
    for name, shape in S.param_shapes(cfg):
        n = int(np.prod(shape))
        picks += list(pos + rng.choice(n, size=min(n, 3), replace=False))
        pos += n
    h = 1e-6
    # absolute floor: the loss is a sum of ~3*n_hole terms of size ~0.3, so each FP64
    # evaluation carries a rounding error of about sqrt(3*n_hole)*eps*L ~ 4e-15, and the
    # central difference divides it by 2h -> ~2e-9
    n_terms = 3 * int((hole != 0).sum())
    floor = math.sqrt(n_terms) * 2.2e-16 * 0.5 / (2 * h) * 2
    for i in picks:
        wp = flat.copy(); wp[i] += h
        wm = flat.copy(); wm[i] -= h
        fd = (O.loss_only(x, hole, tgt, wp, cfg) - O.loss_only(x, hole, tgt, wm, cfg)) / (2 * h)
        an = float(grad[i])
        assert abs(fd - an) <= 1e-6 * max(abs(an), abs(fd)) + floor, (i, fd, an, floor)


# ----------------------------------------------------------------------------- full-resolution pre/post

def test_fullres_oracle_against_library_and_sets():
    cfg = small_cfg(blocks=1)
    flat = S.make_weights(cfg, seed=12, perturb=True)
    B, K, H, W = 2, 3, 64, 96
    rng = np.random.default_rng(12)
    x = torch.from_numpy(S.make_frames(B, H, W, seed=12)).to(DT)
    masks = torch.from_numpy((rng.random((B, K, H // 2, W // 2)) < 0.15).astype(np.uint8) * 7)
    sel = torch.tensor([[1, 0, 1], [0, 0, 1]], dtype=torch.uint8)
    r = O.fullres(x, masks, sel, flat, cfg)
    # union of the selected masks, by python sets
    for b in range(B):
        want = set()
        for k in range(K):
            if sel[b, k]:
                want |= {(int(i), int(j)) for i, j in zip(*np.nonzero(masks[b, k].numpy()))}
        got = {(int(i), int(j)) for i, j in zip(*np.nonzero(r["hole_half"][b].numpy()))}
        assert got == want
    # the half-resolution input is the 2x2 mean, and the pass runs on it
    xh = F.avg_pool2d(x, 2)
    ref = O.forward(xh, r["hole_half"], flat, cfg)
    assert torch.allclose(r["pred_half"], ref["pred"], rtol=1e-12, atol=1e-12)
    # composite: nearest x2 of pred on the upscaled hole, known pixels copied exactly
    up = F.interpolate(ref["pred"], scale_factor=2, mode="nearest")
    hup = F.interpolate(r["hole_half"][:, None].to(DT), scale_factor=2, mode="nearest")[:, 0] != 0
    hm = hup[:, None].expand_as(x)
    assert torch.equal(r["out"][~hm], x[~hm])
    assert torch.equal(r["out"][hm], up[hm])
