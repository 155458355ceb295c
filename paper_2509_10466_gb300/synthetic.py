"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and the bench.

Holds no arithmetic of the inpainting method: only random frames, hole masks and the
random initial weights, each drawn from ``numpy.random.default_rng`` with a seed that
is part of the call.  The datasets of the paper (GTA-V, MIT Indoor, SUN3D, DAVIS) are
not available, so these stand in for them with the shapes and mask statistics of the
workloads: frames are i.i.d. uniform [0, 1]; holes are object-like shapes covering a
stated fraction of the frame, like the paper's training masks (rectangles or multi-stroke
shapes grown or shrunk to 5-30 % of the frame, Section "Mask generation").

Hole convention: ``hole[b, y, x] = 1`` marks a private pixel to be removed and
filled; 0 marks a known pixel.

Weight blob: one flat float32 vector; the tensors follow each other in the order of
:func:`param_shapes`, each in C (row-major) order.  Matrices (``*.w``) are N(0, 0.02),
biases and LayerNorm shifts are 0 and LayerNorm scales are 1.  ``perturb=True``
additionally draws biases, shifts and scales at random so that tests see every term.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------- weights

def param_shapes(cfg):
    """Ordered (name, shape) list of the flat weight blob for a config ``cfg``.

    Matrices of linear layers are stored as (in, out): a token row ``y`` maps to
    ``y @ W + b``.  Conv kernels are (out, in, ky, kx).  With ``pos_bias`` each block
    ends with its relative-position bias (heads, 15, 15), indexed by
    (key row - query row + 7, key column - query column + 7) inside a window.  The embedding's 4 input
    channels are R, G, B of the hole-zeroed frame and then the known-pixel mask.
    """
    d, r, p = cfg.dim, cfg.mlp_ratio, cfg.patch
    c1 = cfg.dec_c1 or d // 4
    c2 = cfg.dec_c2 or d // 8
    out = [("embed.w", (d, 4, p, p)), ("embed.b", (d,))]
    for l in range(cfg.blocks):
        out += [
            (f"blk{l}.ln1.g", (d,)), (f"blk{l}.ln1.b", (d,)),
            (f"blk{l}.qkv.w", (d, 3 * d)), (f"blk{l}.qkv.b", (3 * d,)),
            (f"blk{l}.proj.w", (d, d)), (f"blk{l}.proj.b", (d,)),
            (f"blk{l}.ln2.g", (d,)), (f"blk{l}.ln2.b", (d,)),
            (f"blk{l}.fc1.w", (d, r * d)), (f"blk{l}.fc1.b", (r * d,)),
            (f"blk{l}.fc2.w", (r * d, d)), (f"blk{l}.fc2.b", (d,)),
        ]
        if getattr(cfg, "pos_bias", 0):
            out += [(f"blk{l}.relpos", (cfg.heads, 2 * cfg.window - 1, 2 * cfg.window - 1))]
    out += [
        ("lnf.g", (d,)), ("lnf.b", (d,)),
        ("dec1.w", (c1, d, 3, 3)), ("dec1.b", (c1,)),
        ("dec2.w", (c2, c1, 3, 3)), ("dec2.b", (c2,)),
        ("head.w", (3, c2, 3, 3)), ("head.b", (3,)),
    ]
    return out


def num_params(cfg) -> int:
    return int(sum(np.prod(s) for _, s in param_shapes(cfg)))


def make_weights(cfg, seed: int = 0, std: float = 0.02, perturb: bool = False) -> np.ndarray:
    """Flat float32 weight blob drawn in :func:`param_shapes` order from ``default_rng(seed)``."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in param_shapes(cfg):
        n = int(np.prod(shape))
        leaf = name.rsplit(".", 1)[1]
        is_ln = ".ln" in name or name.startswith("ln")
        if leaf == "w":
            a = rng.standard_normal(n) * std
        elif leaf == "relpos":  # relative-position bias of the window softmax
            a = rng.standard_normal(n) * (0.5 if perturb else std)
        elif is_ln and leaf == "g":
            a = np.ones(n) + (rng.standard_normal(n) * 0.1 if perturb else 0.0)
        else:  # biases and LayerNorm shifts
            a = rng.standard_normal(n) * 0.05 if perturb else np.zeros(n)
        parts.append(a.astype(np.float32))
    return np.concatenate(parts)


_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def _splitmix_out(z):
    """The SplitMix64 output function (Steele, Lea and Flood 2014) on uint64 values (wrapping)."""
    z = z + _GOLDEN
    z = (z ^ (z >> np.uint64(30))) * _MIX1
    z = (z ^ (z >> np.uint64(27))) * _MIX2
    return z ^ (z >> np.uint64(31))


def counter_normals(seed: int, start: int, n: int) -> np.ndarray:
    """Standard normals of blob positions start .. start+n-1 from the counter-based stream of
    ``seed``: r = mix(mix(seed) + i), two 32-bit halves -> uniforms in (0, 1) -> Box-Muller
    (FP64).  The library's inpaint_default_weights draws the same stream."""
    with np.errstate(over="ignore"):
        key = _splitmix_out(np.array([seed], dtype=np.uint64))[0]
        r = _splitmix_out(key + np.arange(start, start + n, dtype=np.uint64))
    u1 = ((r >> np.uint64(32)).astype(np.float64) + 0.5) * (1.0 / 4294967296.0)
    u2 = ((r & np.uint64(0xFFFFFFFF)).astype(np.float64) + 0.5) * (1.0 / 4294967296.0)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(6.283185307179586 * u2)


def default_weights(cfg, seed: int = 0, std: float = 0.02) -> np.ndarray:
    """The default blob of the C library (inpaint_init with NULL weights) in numpy: value i of
    the blob is drawn from (seed, i) alone; matrices, conv kernels and relative-position
    tables float32(std * z), LayerNorm scales 1, biases and shifts 0."""
    parts = []
    at = 0
    for name, shape in param_shapes(cfg):
        n = int(np.prod(shape))
        leaf = name.rsplit(".", 1)[1]
        is_ln = ".ln" in name or name.startswith("ln")
        if leaf in ("w", "relpos"):
            a = (std * counter_normals(seed, at, n)).astype(np.float32)
        elif is_ln and leaf == "g":
            a = np.ones(n, np.float32)
        else:
            a = np.zeros(n, np.float32)
        parts.append(a)
        at += n
    return np.concatenate(parts)


# ----------------------------------------------------------------------------- frames

def make_frames(batch: int, height: int, width: int, seed: int = 0) -> np.ndarray:
    """float32 [B, 3, H, W], uniform [0, 1]; frame b drawn from its own stream (seed, b)."""
    out = np.empty((batch, 3, height, width), np.float32)
    for b in range(batch):
        rng = np.random.default_rng([seed, b, 1])
        out[b] = rng.random((3, height, width), dtype=np.float32)
    return out


# ----------------------------------------------------------------------------- masks

def _ellipse(h, w, cy, cx, ry, rx, theta):
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float32)
    c, s = np.cos(theta), np.sin(theta)
    u = (xx - cx) * c + (yy - cy) * s
    v = -(xx - cx) * s + (yy - cy) * c
    return (u / rx) ** 2 + (v / ry) ** 2 <= 1.0


def _stroke(mask, rng, width_lo, width_hi, n_vertices=(4, 10)):
    """Free-form brush stroke: a random polyline drawn with a round brush."""
    h, w = mask.shape
    n = int(rng.integers(n_vertices[0], n_vertices[1] + 1))
    radius = rng.uniform(width_lo, width_hi) / 2.0
    pts = [np.array([rng.uniform(0, h), rng.uniform(0, w)])]
    for _ in range(n - 1):
        ang = rng.uniform(0, 2 * np.pi)
        length = rng.uniform(0.05, 0.25) * max(h, w)
        nxt = pts[-1] + length * np.array([np.sin(ang), np.cos(ang)])
        nxt = np.clip(nxt, [0, 0], [h - 1, w - 1])
        pts.append(nxt)
    for p0, p1 in zip(pts[:-1], pts[1:]):
        y0, y1 = int(max(0, min(p0[0], p1[0]) - radius - 1)), int(min(h, max(p0[0], p1[0]) + radius + 2))
        x0, x1 = int(max(0, min(p0[1], p1[1]) - radius - 1)), int(min(w, max(p0[1], p1[1]) + radius + 2))
        if y1 <= y0 or x1 <= x0:
            continue
        yy, xx = np.mgrid[y0:y1, x0:x1].astype(np.float32)
        dvec = p1 - p0
        L2 = float(dvec @ dvec) or 1.0
        t = np.clip(((yy - p0[0]) * dvec[0] + (xx - p0[1]) * dvec[1]) / L2, 0.0, 1.0)
        dy = yy - (p0[0] + t * dvec[0])
        dx = xx - (p0[1] + t * dvec[1])
        mask[y0:y1, x0:x1] |= dy * dy + dx * dx <= radius * radius


def _polygon(h, w, rng, cy, cx, radius, n_vertices):
    """Random star-shaped polygon around (cy, cx), filled by the even-odd rule."""
    ang = np.sort(rng.uniform(0, 2 * np.pi, n_vertices))
    rad = radius * rng.uniform(0.4, 1.0, n_vertices)
    vy = cy + rad * np.sin(ang)
    vx = cx + rad * np.cos(ang)
    y0, y1 = int(max(0, vy.min() - 1)), int(min(h, vy.max() + 2))
    x0, x1 = int(max(0, vx.min() - 1)), int(min(w, vx.max() + 2))
    out = np.zeros((h, w), bool)
    if y1 <= y0 or x1 <= x0:
        return out
    yy, xx = np.mgrid[y0:y1, x0:x1].astype(np.float64)
    inside = np.zeros(yy.shape, bool)
    for i in range(n_vertices):
        j = (i + 1) % n_vertices
        ya, xa, yb, xb = vy[i], vx[i], vy[j], vx[j]
        crosses = (ya > yy) != (yb > yy)
        with np.errstate(divide="ignore", invalid="ignore"):
            xint = xa + (yy - ya) * (xb - xa) / (yb - ya)
        inside ^= crosses & (xx < xint)
    out[y0:y1, x0:x1] = inside
    return out


def _draw(kind, h, w, rng):
    m = np.zeros((h, w), bool)
    if kind == "ellipse_strokes":      # 1-3 ellipses plus brush strokes 10-30 px wide
        for _ in range(int(rng.integers(1, 4))):
            m |= _ellipse(h, w, rng.uniform(0, h), rng.uniform(0, w),
                          rng.uniform(0.05, 0.2) * h, rng.uniform(0.05, 0.2) * w, rng.uniform(0, np.pi))
        for _ in range(int(rng.integers(1, 4))):
            _stroke(m, rng, 10, 30)
    elif kind == "polygons":           # 1-6 object blobs as random polygons
        for _ in range(int(rng.integers(1, 7))):
            m |= _polygon(h, w, rng, rng.uniform(0, h), rng.uniform(0, w),
                          rng.uniform(0.08, 0.3) * min(h, w), int(rng.integers(5, 12)))
    elif kind == "large_and_thin":     # one large contiguous hole plus 3-10 px strokes
        m |= _ellipse(h, w, rng.uniform(0.3, 0.7) * h, rng.uniform(0.3, 0.7) * w,
                      rng.uniform(0.15, 0.35) * h, rng.uniform(0.15, 0.35) * w, rng.uniform(0, np.pi))
        for _ in range(int(rng.integers(2, 6))):
            _stroke(m, rng, 3, 10)
    else:
        raise ValueError(f"unknown mask kind {kind!r}")
    return m


MASK_AREA = {"ellipse_strokes": (0.15, 0.25), "polygons": (0.05, 0.40), "large_and_thin": (0.05, 0.50)}


def make_hole(batch: int, height: int, width: int, kind: str = "ellipse_strokes", seed: int = 0,
              area=None, max_tries: int = 200) -> np.ndarray:
    """uint8 [B, H, W] hole masks; the hole fraction of each frame is rejection-sampled into ``area``."""
    lo, hi = area if area is not None else MASK_AREA[kind]
    out = np.zeros((batch, height, width), np.uint8)
    for b in range(batch):
        rng = np.random.default_rng([seed, b, 2])
        best = None
        for _ in range(max_tries):
            m = _draw(kind, height, width, rng)
            frac = m.mean()
            if lo <= frac <= hi:
                best = m
                break
            if best is None or abs(frac - (lo + hi) / 2) < abs(best.mean() - (lo + hi) / 2):
                best = m
        out[b] = best
    return out


def make_target(batch: int, height: int, width: int, seed: int = 0) -> np.ndarray:
    """Seeded target frames for the hole-L1 fine-tuning loss (float32 [B, 3, H, W] in [0, 1])."""
    out = np.empty((batch, 3, height, width), np.float32)
    for b in range(batch):
        rng = np.random.default_rng([seed, b, 3])
        out[b] = rng.random((3, height, width), dtype=np.float32)
    return out


class DriftingBlobs:
    """Hole masks of 1-6 blobs that drift 0-8 px per frame and reflect at the borders.

    One instance per collaborator stream of the serving workload.
    """

    def __init__(self, height: int, width: int, seed: int):
        self.h, self.w = height, width
        self.rng = np.random.default_rng([seed, 4])
        n = int(self.rng.integers(1, 7))
        self.pos = np.stack([self.rng.uniform(0, height, n), self.rng.uniform(0, width, n)], 1)
        speed = self.rng.uniform(0, 8, n)
        ang = self.rng.uniform(0, 2 * np.pi, n)
        self.vel = np.stack([speed * np.sin(ang), speed * np.cos(ang)], 1)
        self.rad = np.stack([self.rng.uniform(0.04, 0.15, n) * height, self.rng.uniform(0.04, 0.15, n) * width], 1)

    def next(self) -> np.ndarray:
        m = np.zeros((self.h, self.w), bool)
        for (cy, cx), (ry, rx) in zip(self.pos, self.rad):
            m |= _ellipse(self.h, self.w, cy, cx, ry, rx, 0.0)
        self.pos += self.vel
        for k, lim in ((0, self.h), (1, self.w)):
            low = self.pos[:, k] < 0
            high = self.pos[:, k] > lim
            self.vel[low | high, k] *= -1
            self.pos[:, k] = np.clip(self.pos[:, k], 0, lim)
        return m.astype(np.uint8)
