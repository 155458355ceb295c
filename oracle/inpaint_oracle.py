"""FP64 CPU oracle of the mask-aware windowed-transformer inpainting pass.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or call this module.  The product path
(the CUDA library and its binding) never does, and this module imports nothing from it.

What it computes, in the paper's terms: the inpainting model receives the frame with
its masked (private) regions set to 0 and returns a completed frame (Section
"Inpainting Manager"); the model is a hybrid CNN/transformer (DSTT-derived, Section
"Real-time Digital Inpainting") whose attention is plain scaled dot-product attention
(Section "Inpainting Model", item "Distinct Transformer Blocks"); the transformer
output is turned back into an image by convolutions with a final crop (item "Modified
Vec2Patch Algorithm").  The paper gives no layer sizes or masking rule; the readings
used here are:

* pad H and W up to a multiple of patch*window (32) with x = 0 and hole = 1;
  m = 1 - hole; the model input is [x*m (3 ch), m (1 ch)];
* patch embedding: 4x4 stride-4 convolution, no padding (a GEMM over 64-value patches);
* token mask v0[t] = 1 if any pixel of the token's patch is known;
* pre-LN transformer blocks; block l attends inside 8x8-token windows, offset by half a
  window on odd blocks (shift=1); slots of an offset window that fall outside the grid
  are void (neither keys nor queries); keys are the tokens with v[l] = 1; a window with
  no such key outputs 0; after the attention of block l every real token of a window
  with any usable key becomes valid: v[l+1][t] = OR of v[l] over t's window;
* softmax scale 1/sqrt(d_h); LayerNorm eps 1e-5 with biased variance; exact erf GELU;
* optional relative-position bias (pos_bias = 1): a learned per-head table added to the
  scores of query slot i and key slot j by their row and column offset in the window;
* final LayerNorm, then two stages of (nearest x2 upsample, 3x3 conv pad 1, GELU) with
  d/4 and d/8 channels, then a 3x3 conv to RGB = pred (no output activation);
* composite out = pred on hole pixels and x on known pixels (a select, so known pixels
  are copied exactly), cropped back to H x W;
* temporal memory (mem_slots = m > 0): odd blocks are temporal; a temporal block's
  queries also attend to the keys/values that each of m previous frames produced in
  the same block, at the same window positions, where those frames' tokens were usable
  keys; the window becomes valid if any current or memory key is usable.  A frame's
  memory tensor is its own k | v and usable-key mask in every temporal block;
* fine-tuning loss: L1 over hole pixels only, sum / (3 * number of hole pixels), 0 when
  there are no hole pixels (Section "Training structure", "Loss"; the paper also weights
  known pixels, which this path leaves out).

Everything is float64.  Library primitives (matmul, einsum, exp, erf, autograd for the
reverse mode) serve as steps; there is no blocking or fusion beyond the definitions.
"""
from __future__ import annotations

import math

import torch

DT = torch.float64
LN_EPS = 1e-5


# ----------------------------------------------------------------------------- weights

def unpack(flat: torch.Tensor, cfg) -> dict:
    """Split the flat weight blob into named views (order: embed, blocks, lnf, decoder)."""
    d, r, p = cfg.dim, cfg.mlp_ratio, cfg.patch
    c1 = cfg.dec_c1 or d // 4
    c2 = cfg.dec_c2 or d // 8
    pos = 0
    out = {}

    def take(name, *shape):
        nonlocal pos
        n = 1
        for s in shape:
            n *= s
        out[name] = flat[pos:pos + n].reshape(*shape)
        pos += n

    take("embed.w", d, 4, p, p)
    take("embed.b", d)
    for l in range(cfg.blocks):
        take(f"{l}.ln1.g", d); take(f"{l}.ln1.b", d)
        take(f"{l}.qkv.w", d, 3 * d); take(f"{l}.qkv.b", 3 * d)
        take(f"{l}.proj.w", d, d); take(f"{l}.proj.b", d)
        take(f"{l}.ln2.g", d); take(f"{l}.ln2.b", d)
        take(f"{l}.fc1.w", d, r * d); take(f"{l}.fc1.b", r * d)
        take(f"{l}.fc2.w", r * d, d); take(f"{l}.fc2.b", d)
        if getattr(cfg, "pos_bias", 0):
            take(f"{l}.relpos", cfg.heads, 2 * cfg.window - 1, 2 * cfg.window - 1)
    take("lnf.g", d); take("lnf.b", d)
    take("dec1.w", c1, d, 3, 3); take("dec1.b", c1)
    take("dec2.w", c2, c1, 3, 3); take("dec2.b", c2)
    take("head.w", 3, c2, 3, 3); take("head.b", 3)
    if pos != flat.numel():
        raise ValueError(f"weight blob has {flat.numel()} values, config needs {pos}")
    return out


def num_params(cfg) -> int:
    d, r, p = cfg.dim, cfg.mlp_ratio, cfg.patch
    c1 = cfg.dec_c1 or d // 4
    c2 = cfg.dec_c2 or d // 8
    blk = 2 * d + 3 * d * d + 3 * d + d * d + d + 2 * d + 2 * r * d * d + r * d + d
    if getattr(cfg, "pos_bias", 0):
        blk += cfg.heads * (2 * cfg.window - 1) ** 2
    return (d * 4 * p * p + d + cfg.blocks * blk + 2 * d
            + c1 * d * 9 + c1 + c2 * c1 * 9 + c2 + 3 * c2 * 9 + 3)


# ----------------------------------------------------------------------------- steps

def pad_inputs(x: torch.Tensor, hole: torch.Tensor, multiple: int):
    """Pad [B,3,H,W] frames and [B,H,W] holes on the bottom/right: x = 0, hole = 1."""
    B, _, H, W = x.shape
    Hp = -(-H // multiple) * multiple
    Wp = -(-W // multiple) * multiple
    xp = x.new_zeros(B, 3, Hp, Wp)
    xp[:, :, :H, :W] = x
    hp = torch.ones(B, Hp, Wp, dtype=torch.uint8)
    hp[:, :H, :W] = (hole != 0).to(torch.uint8)
    return xp, hp


def model_input(xp: torch.Tensor, hp: torch.Tensor) -> torch.Tensor:
    """[x*m, m] with m = 1 - hole: the frame with its masked regions set to 0, plus the mask."""
    m = (1 - hp).to(DT)[:, None]
    return torch.cat([xp * m, m], dim=1)


def patch_embed(inp: torch.Tensor, w: torch.Tensor, b: torch.Tensor, p: int) -> torch.Tensor:
    """tok[b, ty*Wt+tx, :] = b + sum_{c,i,j} w[:, c, i, j] * inp[b, c, p*ty+i, p*tx+j]."""
    B, C, Hp, Wp = inp.shape
    Ht, Wt = Hp // p, Wp // p
    patches = inp.reshape(B, C, Ht, p, Wt, p).permute(0, 2, 4, 1, 3, 5).reshape(B, Ht * Wt, C * p * p)
    return patches @ w.reshape(w.shape[0], C * p * p).T + b


def token_mask_init(hp: torch.Tensor, p: int) -> torch.Tensor:
    """v0[b, t] = 1 if any pixel of token t's p x p patch is known (hole == 0)."""
    B, Hp, Wp = hp.shape
    known = (hp == 0).reshape(B, Hp // p, p, Wp // p, p)
    return known.any(dim=4).any(dim=2).reshape(B, -1).to(torch.uint8)


def window_index(Ht: int, Wt: int, ws: int, offset: int) -> torch.Tensor:
    """[n_windows, ws*ws] token indices of each window; -1 marks a void slot.

    Window (wy, wx) covers token rows wy*ws - offset ... wy*ws - offset + ws - 1 (same
    for columns); slots outside the Ht x Wt grid are void.
    """
    nwy = -(-(Ht + offset) // ws)
    nwx = -(-(Wt + offset) // ws)
    rows = []
    for wy in range(nwy):
        for wx in range(nwx):
            slots = []
            for i in range(ws):
                for j in range(ws):
                    ty, tx = wy * ws - offset + i, wx * ws - offset + j
                    slots.append(ty * Wt + tx if (0 <= ty < Ht and 0 <= tx < Wt) else -1)
            rows.append(slots)
    return torch.tensor(rows, dtype=torch.long)


def block_offset(cfg, l: int) -> int:
    return cfg.window // 2 if (cfg.shift and l % 2 == 1) else 0


def layer_norm(x: torch.Tensor, g: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    mu = x.mean(dim=-1, keepdim=True)
    var = ((x - mu) ** 2).mean(dim=-1, keepdim=True)
    return (x - mu) / torch.sqrt(var + LN_EPS) * g + b


def gelu(x: torch.Tensor) -> torch.Tensor:
    return 0.5 * x * (1.0 + torch.erf(x / math.sqrt(2.0)))


def relpos_bias(relpos: torch.Tensor, ws: int) -> torch.Tensor:
    """[heads, 2ws-1, 2ws-1] table -> [heads, S, S] score bias of query slot i and key slot
    j of a window (slot = row * ws + column): relpos[h, rj - ri + ws-1, cj - ci + ws-1]."""
    r = torch.arange(ws * ws) // ws
    c = torch.arange(ws * ws) % ws
    dy = r[None, :] - r[:, None] + ws - 1
    dx = c[None, :] - c[:, None] + ws - 1
    return relpos[:, dy, dx]


def window_attention(qkv: torch.Tensor, valid: torch.Tensor, heads: int, widx: torch.Tensor, relpos=None):
    """Mask-aware windowed multi-head attention of one frame.

    qkv [N, 3d] (q | k | v, head h at columns h*d_h ... within each third), valid [N]
    (1 = usable key).  For query t in window w: o_t = sum over keys s of w with
    valid[s] of softmax_s(q_t . k_s / sqrt(d_h) [+ relative-position bias]) v_s, per
    head; o_t = 0 when w has no valid key.  Returns (o [N, d], next valid [N] = OR of
    valid over t's window).
    """
    N, d3 = qkv.shape
    d = d3 // 3
    dh = d // heads
    nW, S = widx.shape
    real = widx >= 0
    safe = widx.clamp(min=0)
    key_ok = real & (valid[safe] != 0)                     # [nW, S]
    any_w = key_ok.any(dim=1)                              # [nW]
    q = qkv[:, :d][safe].reshape(nW, S, heads, dh).transpose(1, 2)        # [nW, h, S, dh]
    k = qkv[:, d:2 * d][safe].reshape(nW, S, heads, dh).transpose(1, 2)
    v = qkv[:, 2 * d:][safe].reshape(nW, S, heads, dh).transpose(1, 2)
    s = q @ k.transpose(-1, -2) / math.sqrt(dh)                            # [nW, h, S, S]
    if relpos is not None:
        s = s + relpos_bias(relpos, int(round(S ** 0.5)))[None]
    # windows without a usable key get a harmless stand-in key set; their output is zeroed
    allowed = key_ok | ~any_w[:, None]
    s = s.masked_fill(~allowed[:, None, None, :], float("-inf"))
    e = torch.exp(s - s.max(dim=-1, keepdim=True).values)
    pr = e / e.sum(dim=-1, keepdim=True)
    ow = (pr @ v).transpose(1, 2).reshape(nW, S, d) * any_w[:, None, None].to(qkv.dtype)
    o = qkv.new_zeros(N, d)
    o = o.index_put((widx[real],), ow[real])
    nxt = torch.zeros(N, dtype=torch.uint8)
    nxt[widx[real]] = any_w[:, None].expand(nW, S)[real].to(torch.uint8)
    return o, nxt


def temporal_block(cfg, l: int) -> bool:
    """Whether block l is a temporal block: with memory slots, odd blocks (the paper's
    fixed series alternating spatial and temporal blocks, item "Distinct Transformer
    Blocks"; memory tensors of previous frames, Sections "Inpainting Manager" and
    "Minimal memory slots")."""
    return getattr(cfg, "mem_slots", 0) > 0 and l % 2 == 1


def window_attention_mem(qkv: torch.Tensor, valid: torch.Tensor, heads: int, widx: torch.Tensor, mem, relpos=None):
    """window_attention with memory keys: `mem` lists, per memory slot, (kv [N, 2d] =
    k | v of a past frame at this block, mask [N] = that frame's usable-key mask there),
    or None for an empty slot.  Query t of window w attends over w's usable current keys
    and, in every slot, the usable keys at w's positions; o_t = 0 when there is none.
    next valid[t] = 1 iff t's window had any usable key (current or memory)."""
    N, d3 = qkv.shape
    d = d3 // 3
    dh = d // heads
    nW, S = widx.shape
    real = widx >= 0
    safe = widx.clamp(min=0)

    def heads_of(t):  # [N, d] gathered by window -> [nW, h, S, dh]
        return t[safe].reshape(nW, S, heads, dh).transpose(1, 2)

    q = heads_of(qkv[:, :d])
    ks, vs, oks = [heads_of(qkv[:, d:2 * d])], [heads_of(qkv[:, 2 * d:])], [real & (valid[safe] != 0)]
    for slot in mem:
        if slot is None:
            continue
        kv, mask = slot
        ks.append(heads_of(kv[:, :d]))
        vs.append(heads_of(kv[:, d:]))
        oks.append(real & (mask[safe] != 0))
    k = torch.cat(ks, dim=2)                                   # [nW, h, S*(1+m), dh]
    v = torch.cat(vs, dim=2)
    key_ok = torch.cat(oks, dim=1)                             # [nW, S*(1+m)]
    any_w = key_ok.any(dim=1)
    s = q @ k.transpose(-1, -2) / math.sqrt(dh)
    if relpos is not None:  # memory keys sit at the same window positions as current ones
        s = s + relpos_bias(relpos, int(round(S ** 0.5))).repeat(1, 1, len(ks))[None]
    allowed = key_ok | ~any_w[:, None]
    s = s.masked_fill(~allowed[:, None, None, :], float("-inf"))
    e = torch.exp(s - s.max(dim=-1, keepdim=True).values)
    pr = e / e.sum(dim=-1, keepdim=True)
    ow = (pr @ v).transpose(1, 2).reshape(nW, S, d) * any_w[:, None, None].to(qkv.dtype)
    o = qkv.new_zeros(N, d)
    o = o.index_put((widx[real],), ow[real])
    nxt = torch.zeros(N, dtype=torch.uint8)
    nxt[widx[real]] = any_w[:, None].expand(nW, S)[real].to(torch.uint8)
    return o, nxt


def upsample2(f: torch.Tensor) -> torch.Tensor:
    """Nearest-neighbour x2 upsampling of [B, C, H, W]."""
    return f.repeat_interleave(2, dim=2).repeat_interleave(2, dim=3)


def conv3x3(f: torch.Tensor, w: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """out[b,o,y,x] = b[o] + sum_{c,ky,kx} w[o,c,ky,kx] * f[b,c,y+ky-1,x+kx-1], zero outside."""
    B, C, H, W = f.shape
    side = f.new_zeros(B, C, H, 1)
    row = f.new_zeros(B, C, 1, W + 2)
    fp = torch.cat([row, torch.cat([side, f, side], dim=3), row], dim=2)      # zero border of 1
    out = b.reshape(1, -1, 1, 1).expand(B, w.shape[0], H, W)
    for ky in range(3):
        for kx in range(3):
            out = out + torch.einsum("bchw,oc->bohw", fp[:, :, ky:ky + H, kx:kx + W], w[:, :, ky, kx])
    return out


# ----------------------------------------------------------------------------- model

def forward(x, hole, weights, cfg, keep_block_inputs: bool = False, mem=None) -> dict:
    """The whole pass.  x float [B,3,H,W] in [0,1]; hole uint8 [B,H,W] (nonzero = remove).

    Returns out [B,3,H,W], pred [B,3,H,W] (decoder output, cropped), masks
    [(L+1), B, N] uint8 (token masks v0 ... vL) and, on request, the block inputs.
    With memory slots (cfg.mem_slots > 0), `mem[b]` lists frame b's memory slots (each
    a previous frame's "memory" entry, or None), and res["memory"][b] is the memory
    tensor this frame emits: for every temporal block l, (k | v [N, 2d], usable-key
    mask [N]) of its own tokens at that block.
    """
    x = torch.as_tensor(x).to(DT)
    hole = torch.as_tensor(hole)
    flat = torch.as_tensor(weights)
    if flat.dtype != DT:
        flat = flat.to(DT)
    w = unpack(flat, cfg)
    B, _, H, W = x.shape
    p, ws, d = cfg.patch, cfg.window, cfg.dim
    xp, hp = pad_inputs(x, hole, p * ws)
    Hp, Wp = xp.shape[2:]
    Ht, Wt = Hp // p, Wp // p

    tok = patch_embed(model_input(xp, hp), w["embed.w"], w["embed.b"], p)     # [B, N, d]
    v = token_mask_init(hp, p)                                                  # [B, N]
    masks = [v]
    block_inputs = []
    memory = [dict() for _ in range(B)]
    for l in range(cfg.blocks):
        block_inputs.append(tok)
        widx = window_index(Ht, Wt, ws, block_offset(cfg, l))
        y = layer_norm(tok, w[f"{l}.ln1.g"], w[f"{l}.ln1.b"])
        qkv = y @ w[f"{l}.qkv.w"] + w[f"{l}.qkv.b"]
        rp = w[f"{l}.relpos"] if getattr(cfg, "pos_bias", 0) else None
        outs, nxts = [], []
        for bi in range(B):
            if temporal_block(cfg, l):
                slots = [None if mem is None or mem[bi] is None or mem[bi][j] is None else mem[bi][j][l]
                         for j in range(cfg.mem_slots)]
                o, nxt = window_attention_mem(qkv[bi], v[bi], cfg.heads, widx, slots, rp)
                memory[bi][l] = (qkv[bi][:, d:].clone(), v[bi].clone())
            else:
                o, nxt = window_attention(qkv[bi], v[bi], cfg.heads, widx, rp)
            outs.append(o)
            nxts.append(nxt)
        o = torch.stack(outs)
        v = torch.stack(nxts)
        masks.append(v)
        tok = tok + o @ w[f"{l}.proj.w"] + w[f"{l}.proj.b"]
        y2 = layer_norm(tok, w[f"{l}.ln2.g"], w[f"{l}.ln2.b"])
        tok = tok + gelu(y2 @ w[f"{l}.fc1.w"] + w[f"{l}.fc1.b"]) @ w[f"{l}.fc2.w"] + w[f"{l}.fc2.b"]

    y = layer_norm(tok, w["lnf.g"], w["lnf.b"])
    feat = y.reshape(B, Ht, Wt, d).permute(0, 3, 1, 2)                         # [B, d, Ht, Wt]
    h1 = gelu(conv3x3(upsample2(feat), w["dec1.w"], w["dec1.b"]))
    h2 = gelu(conv3x3(upsample2(h1), w["dec2.w"], w["dec2.b"]))
    pred_full = conv3x3(h2, w["head.w"], w["head.b"])                          # [B, 3, Hp, Wp]
    pred = pred_full[:, :, :H, :W]
    out = torch.where((hole != 0)[:, None], pred, x)
    res = {"out": out, "pred": pred, "masks": torch.stack(masks)}
    if getattr(cfg, "mem_slots", 0) > 0:
        res["memory"] = memory
    if keep_block_inputs:
        res["block_inputs"] = block_inputs
        res["final_tokens"] = tok
    return res


def token_masks(hole, cfg) -> torch.Tensor:
    """Masks v0 ... vL only (the integer part of the pass), [(L+1), B, N] uint8."""
    hole = torch.as_tensor(hole)
    B, H, W = hole.shape
    p, ws = cfg.patch, cfg.window
    _, hp = pad_inputs(torch.zeros(B, 3, H, W, dtype=DT), hole, p * ws)
    Ht, Wt = hp.shape[1] // p, hp.shape[2] // p
    v = token_mask_init(hp, p)
    masks = [v]
    for l in range(cfg.blocks):
        widx = window_index(Ht, Wt, ws, block_offset(cfg, l))
        real = widx >= 0
        safe = widx.clamp(min=0)
        nxt = torch.zeros_like(v)
        for bi in range(B):
            any_w = (real & (v[bi][safe] != 0)).any(dim=1)
            nxt[bi][widx[real]] = any_w[:, None].expand_as(widx)[real].to(torch.uint8)
        v = nxt
        masks.append(v)
    return torch.stack(masks)


# ----------------------------------------------------------------------------- loss / gradient

def l1_hole_loss(out, target, hole):
    """L = sum over hole pixels and channels of |out - target| / (3 * n_hole); 0 if no hole.

    Returns (L, dL/dout) with sign(0) = 0 and zero gradient on known pixels.
    """
    out = torch.as_tensor(out).to(DT)
    target = torch.as_tensor(target).to(DT)
    hm = (torch.as_tensor(hole) != 0)[:, None].expand_as(out)
    n_hole = int((torch.as_tensor(hole) != 0).sum())
    if n_hole == 0:
        return torch.zeros((), dtype=DT), torch.zeros_like(out)
    diff = out - target
    loss = diff.abs()[hm].sum() / (3 * n_hole)
    grad = torch.where(hm, torch.sign(diff), torch.zeros_like(diff)) / (3 * n_hole)
    return loss, grad


def weight_vjp(x, hole, grad_out, weights, cfg) -> torch.Tensor:
    """dL/dweights for dL/dout = grad_out (reverse mode of :func:`forward`; masks carry no gradient)."""
    flat = torch.as_tensor(weights).to(DT).clone().requires_grad_(True)
    out = forward(x, hole, flat, cfg)["out"]
    (out * torch.as_tensor(grad_out).to(DT)).sum().backward()
    return flat.grad.detach()


def loss_and_grad(x, hole, target, weights, cfg):
    """Hole-L1 loss of the composite against ``target`` and its gradient w.r.t. the weights."""
    flat = torch.as_tensor(weights).to(DT).clone().requires_grad_(True)
    out = forward(x, hole, flat, cfg)["out"]
    tgt = torch.as_tensor(target).to(DT)
    hm = (torch.as_tensor(hole) != 0)[:, None].expand_as(out)
    n_hole = int((torch.as_tensor(hole) != 0).sum())
    if n_hole == 0:
        return torch.zeros((), dtype=DT), torch.zeros_like(flat)
    loss = (out - tgt).abs()[hm].sum() / (3 * n_hole)
    loss.backward()
    return loss.detach(), flat.grad.detach()


def loss_only(x, hole, target, weights, cfg) -> float:
    with torch.no_grad():
        out = forward(x, hole, torch.as_tensor(weights).to(DT), cfg)["out"]
        return float(l1_hole_loss(out, target, hole)[0])


# ----------------------------------------------------------------------------- full-resolution pre/post

def fullres(x, obj_masks, selected, weights, cfg) -> dict:
    """Half-resolution inpainting of full-resolution frames (Section "Upscaling"), with the
    hole built from the selected objects' masks (Section "Object Control").

    x float [B,3,H,W] (H, W even); obj_masks uint8 [B,K,H/2,W/2]; selected uint8 [B,K].
    hole_half = OR over selected k of (mask != 0); x_half = mean of each 2x2 block;
    out = hole_half[y//2, x//2] ? pred_half[y//2, x//2] : x[y, x].
    """
    x = torch.as_tensor(x).to(DT)
    m = torch.as_tensor(obj_masks) != 0
    sel = torch.as_tensor(selected) != 0
    B, _, H, W = x.shape
    hole_half = (m & sel[:, :, None, None]).any(dim=1).to(torch.uint8)
    x_half = 0.25 * (x[:, :, 0::2, 0::2] + x[:, :, 0::2, 1::2] + x[:, :, 1::2, 0::2] + x[:, :, 1::2, 1::2])
    r = forward(x_half, hole_half, weights, cfg)
    up = r["pred"].repeat_interleave(2, dim=2).repeat_interleave(2, dim=3)
    hole_up = hole_half.repeat_interleave(2, dim=1).repeat_interleave(2, dim=2)
    out = torch.where((hole_up != 0)[:, None], up, x)
    return {"out": out, "hole_half": hole_half, "pred_half": r["pred"], "masks": r["masks"]}
