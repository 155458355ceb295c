"""The sub-pixel form of the decoder stages, checked on the CPU against the oracle.

The decoder (nearest x2 upsampling, then a zero-padded 3x3 convolution) runs on the GPU
as a 2x2 convolution per output parity (a, b) on the low-resolution input, with merged
weights, and, for Cout = 32 / 64, with the parities stacked on the MMA's M side: one
product per input shift (sy, sx) that any parity of a group reads, with zero weights for
the parities that do not read it.  These tests restate that algebra in numpy (FP64) and
compare it with the oracle's `upsample2` + `conv3x3`, so that a wrong tap merge, shift
set or parity-to-row mapping fails here without a GPU.
"""
import numpy as np
import pytest
import torch

from oracle import inpaint_oracle as O


def tap_offset(a, k):
    """Input offset of 3x3 tap k for output parity a after nearest x2 upsampling."""
    return (a + k - 1) // 2


def group_shifts(ng, grp):
    """The input shifts that the parities of a group read (9 for four parities, 6 for two)."""
    if ng == 4:
        return [(sy, sx) for sy in (-1, 0, 1) for sx in (-1, 0, 1)]
    return [(sy, sx) for sy in (grp - 1, grp) for sx in (-1, 0, 1)]


def group_parities(ng, grp):
    return [(g >> 1, g & 1) for g in range(4)] if ng == 4 else [(grp, 0), (grp, 1)]


def stacked_weights(w, ng, grp):
    """[shift][g * Cout + co][ci] with the taps of parity g that land on each shift."""
    cout, cin = w.shape[:2]
    shifts, pars = group_shifts(ng, grp), group_parities(ng, grp)
    ws = np.zeros((len(shifts), ng * cout, cin))
    for s, (sy, sx) in enumerate(shifts):
        for g, (a, b) in enumerate(pars):
            for ky in range(3):
                for kx in range(3):
                    if tap_offset(a, ky) == sy and tap_offset(b, kx) == sx:
                        ws[s, g * cout:(g + 1) * cout] += w[:, :, ky, kx]
    return ws


def stacked_stage(x, w, bias):
    """out[2i+a, 2j+b, co] from the parity-stacked products (x [Hi, Wi, Cin], no activation)."""
    hi, wi, _ = x.shape
    cout = w.shape[0]
    ng = 4 if cout * 4 <= 128 else 2
    out = np.zeros((2 * hi, 2 * wi, cout))
    xp = np.zeros((hi + 2, wi + 2, x.shape[2]))
    xp[1:-1, 1:-1] = x
    for grp in range(4 // ng):
        ws = stacked_weights(w, ng, grp)
        d = np.zeros((hi, wi, ng * cout))
        for s, (sy, sx) in enumerate(group_shifts(ng, grp)):
            d += xp[1 + sy:1 + sy + hi, 1 + sx:1 + sx + wi] @ ws[s].T
        for g, (a, b) in enumerate(group_parities(ng, grp)):
            out[a::2, b::2] = d[:, :, g * cout:(g + 1) * cout] + bias
    return out


def oracle_stage(x, w, bias):
    f = torch.from_numpy(x).permute(2, 0, 1)[None]
    y = O.conv3x3(O.upsample2(f), torch.from_numpy(w), torch.from_numpy(bias))
    return y[0].permute(1, 2, 0).numpy()


@pytest.mark.parametrize("hi,wi,cin,cout", [(5, 7, 6, 32), (4, 3, 5, 64), (1, 1, 3, 32), (6, 2, 4, 64)])
def test_parity_stacked_sub_pixel_form_is_upsample_then_conv(hi, wi, cin, cout):
    rng = np.random.default_rng(hi * 100 + wi * 10 + cout)
    x = rng.standard_normal((hi, wi, cin))
    w = rng.standard_normal((cout, cin, 3, 3))
    bias = rng.standard_normal(cout)
    got, ref = stacked_stage(x, w, bias), oracle_stage(x, w, bias)
    assert np.allclose(got, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))


def test_each_parity_reads_four_of_the_shifts():
    """A parity's merged weights are nonzero on exactly its 2 x 2 input shifts, and the nine
    3x3 taps are each merged into exactly one of them (4/9 of the direct products)."""
    w = np.ones((1, 1, 3, 3))
    for ng, groups in ((4, 1), (2, 2)):
        for grp in range(groups):
            ws = stacked_weights(w, ng, grp)[:, :, 0]  # [shift][g]
            for g, (a, b) in enumerate(group_parities(ng, grp)):
                used = [s for s in range(ws.shape[0]) if ws[s, g] != 0]
                assert len(used) == 4
                assert ws[:, g].sum() == 9
