"""VarDCT pixel reconstruction of entropy-decoded data, in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Order of the steps (9.7-9.13 of the draft):
  F.2  DC dequantisation          dc = m_DC[c] * q
  G    DC chroma-from-luma        X += kX_dc * Y, B += kB_dc * Y
  I.2.7 LLF from DC               exact inverse of the 8x8 box mean (I.2.6)
  F.3  AC dequantisation          bias, * AcMul, * matrix (C.6.1)
  G    AC chroma-from-luma        per 64x64 tile factors
  I.2.4 inverse transforms        per varblock
  J.2  edge-preserving filter     (optional)
  J.4  Gaborish                   (optional)
  L.2  XYB -> linear RGB, then /255 to [0, 1]

Inputs follow the library's layout: ``coeffs[c][y][x]`` int16, where the
quantised coefficient (u, v) of the varblock whose top-left sample is
(x0, y0) sits at (x0 + u, y0 + v), and its LLF slots (u < W/8, v < H/8) hold
the quantised DC samples of the 8x8 blocks (x0/8 + u, y0/8 + v).
``vmap[by][bx]`` holds the DctSelect code at a varblock's top-left block and
0xFF on the other blocks it covers; ``acmul[by][bx]`` is AcMul (C.5.5);
``cfl[ty][tx] = (kX, kB)`` per 64x64 tile; ``sharpness[by][bx]`` (C.5.6).

Decisions that turn a real number into an integer inside the EPF (the guide
quantisation and the sigma truncation of J.2.2/J.2.4) are taken in binary32
arithmetic, operation by operation, exactly as the CUDA kernels take them,
so that both sides see the same integers for the same input samples.
"""
import math

import numpy as np

from . import tables as T
from . import transforms as TR


class Params:
    """Reconstruction parameters; defaults are the draft's (C.4, C.10, L.2)."""

    def __init__(self, **kw):
        self.m_dc = (0.02 / (64 * math.sqrt(2)), 0.2 / (64 * math.sqrt(2)),
                     0.2 / (64 * math.sqrt(2)))
        self.kx_dc = 0.0
        self.kb_dc = 0.0
        self.gab = False
        self.gab_w1 = T.GAB_W1
        self.gab_w2 = T.GAB_W2
        self.epf = False
        self.epf_weight_min = T.EPF_WEIGHT_MIN
        self.epf_scale = T.EPF_SCALE
        self.epf_sharp_lut = T.EPF_SHARP_LUT
        self.epf_range_max = T.EPF_RANGE_MAX
        self.epf_range_mul = T.EPF_RANGE_MUL
        self.epf_quant_mul = T.EPF_QUANT_MUL
        self.epf_sigma_max = T.EPF_SIGMA_MAX
        self.inv_opsin = T.INV_OPSIN
        self.opsin_bias = T.OPSIN_BIAS
        self.target_nits_div50 = T.TARGET_NITS_DIV50
        for k, v in kw.items():
            if not hasattr(self, k):
                raise KeyError(k)
            setattr(self, k, v)


# ---------------------------------------------------------------------------
# 6.5 mirroring
# ---------------------------------------------------------------------------
def mirror(coord, size):
    c = np.array(coord, dtype=np.int64, copy=True)
    while True:
        lo = c < 0
        hi = c >= size
        if not (lo.any() or hi.any()):
            return c
        c = np.where(lo, -c - 1, c)
        c = np.where(hi, 2 * size - 1 - c, c)


# ---------------------------------------------------------------------------
# Varblock geometry
# ---------------------------------------------------------------------------
def varblocks(vmap):
    """List of (code, bx0, by0) for every varblock top-left block."""
    out = []
    bh, bw = vmap.shape
    for by in range(bh):
        for bx in range(bw):
            code = int(vmap[by, bx])
            if code != T.COVERED:
                out.append((code, bx, by))
    return out


def owner_map(vmap):
    """Per 8x8 block: (code, bx0, by0) of the varblock covering it."""
    bh, bw = vmap.shape
    code = np.full((bh, bw), -1, dtype=np.int64)
    ox = np.zeros((bh, bw), dtype=np.int64)
    oy = np.zeros((bh, bw), dtype=np.int64)
    for c, bx, by in varblocks(vmap):
        W, H = T.SHAPE_WH[c]
        code[by:by + H // 8, bx:bx + W // 8] = c
        ox[by:by + H // 8, bx:bx + W // 8] = bx
        oy[by:by + H // 8, bx:bx + W // 8] = by
    return code, ox, oy


# ---------------------------------------------------------------------------
# F.2 + G + I.2.7 + F.3 + G: coefficients of every varblock
# ---------------------------------------------------------------------------
def dequantize(coeffs, vmap, acmul, cfl, params):
    """Dequantised, chroma-from-luma-corrected coefficient planes (FP64), in
    the same footprint layout as ``coeffs``, with each varblock's LLF slots
    holding its LLF coefficients."""
    _, Hp, Wp = coeffs.shape
    q = coeffs.astype(np.float64)
    code, ox, oy = owner_map(vmap)
    # per-sample varblock description
    code_s = np.repeat(np.repeat(code, 8, 0), 8, 1)
    x0 = np.repeat(np.repeat(ox, 8, 0), 8, 1) * 8
    y0 = np.repeat(np.repeat(oy, 8, 0), 8, 1) * 8
    xs = np.arange(Wp)[None, :]
    ys = np.arange(Hp)[:, None]
    u = xs - x0
    v = ys - y0
    Wv = np.zeros_like(code_s)
    Hv = np.zeros_like(code_s)
    for c_, (W, H) in T.SHAPE_WH.items():
        Wv[code_s == c_] = W
        Hv[code_s == c_] = H
    llf = (u < Wv // 8) & (v < Hv // 8)
    # AcMul of the varblock (READING: constant per varblock, C.5.5)
    acm = np.repeat(np.repeat(acmul.astype(np.float64), 8, 0), 8, 1)[y0, x0]
    # F.3 bias adjustment
    out = np.zeros((3, Hp, Wp))
    for c in range(3):
        qc = q[c]
        with np.errstate(divide='ignore', invalid='ignore'):
            biased = np.where(np.abs(qc) <= 1, qc * (1 - T.K_ONE_BIAS[c]),
                              qc - T.K_BIAS_NUMER / qc)
        val = np.zeros((Hp, Wp))
        for c_ in T.SHAPE_WH:
            sel = code_s == c_
            if sel.any():
                m = T.dequant_matrix(c_, c)
                val[sel] = m[v[sel], u[sel]]
        out[c] = np.where(llf, 0.0, biased * acm * val)
    # G for AC: per 64x64 tile of the coefficient's position
    kx = np.repeat(np.repeat(cfl[..., 0].astype(np.float64), 64, 0), 64, 1)[:Hp, :Wp]
    kb = np.repeat(np.repeat(cfl[..., 1].astype(np.float64), 64, 0), 64, 1)[:Hp, :Wp]
    out[0] = out[0] + kx * out[1]
    out[2] = out[2] + kb * out[1]
    # F.2 DC dequantisation and G for DC
    dc = np.stack([params.m_dc[c] * q[c] for c in range(3)])
    dc[0] = dc[0] + params.kx_dc * dc[1]
    dc[2] = dc[2] + params.kb_dc * dc[1]
    # I.2.7 LLF from DC, per varblock
    for c_, bx, by in varblocks(vmap):
        W, H = T.SHAPE_WH[c_]
        x_0, y_0 = 8 * bx, 8 * by
        for c in range(3):
            d = dc[c, y_0:y_0 + H // 8, x_0:x_0 + W // 8]
            out[c, y_0:y_0 + H // 8, x_0:x_0 + W // 8] = TR.llf_from_dc(d)
    return out


# ---------------------------------------------------------------------------
# I.2.4: coefficients to samples
# ---------------------------------------------------------------------------
_OPERATOR_8X8 = {}


def _operator_8x8(code):
    """The 8x8-class procedures are linear; their 64x64 operator is built
    once by running the step-by-step procedure on each unit coefficient."""
    if code not in _OPERATOR_8X8:
        op = np.zeros((64, 64))
        for j in range(64):
            e = np.zeros(64)
            e[j] = 1.0
            op[:, j] = TR.idct_8x8_class(code, e.reshape(8, 8)).reshape(-1)
        _OPERATOR_8X8[code] = op
    return _OPERATOR_8X8[code]


def inverse_transform(dq, vmap):
    """XYB samples (padded size) from dequantised coefficient planes."""
    _, Hp, Wp = dq.shape
    out = np.zeros_like(dq)
    by_code = {}
    for c_, bx, by in varblocks(vmap):
        by_code.setdefault(c_, []).append((bx, by))
    for c_, origins in by_code.items():
        W, H = T.SHAPE_WH[c_]
        blocks = np.stack([dq[:, 8 * by:8 * by + H, 8 * bx:8 * bx + W]
                           for bx, by in origins])          # n, 3, H, W
        if c_ in T.DCT_SHAPES:
            pix = TR._IDCT[H] @ blocks @ TR._IDCT[W].T
        else:
            op = _operator_8x8(c_)
            pix = (blocks.reshape(-1, 64) @ op.T).reshape(blocks.shape)
        for i, (bx, by) in enumerate(origins):
            out[:, 8 * by:8 * by + H, 8 * bx:8 * bx + W] = pix[i]
    return out


def inverse_transform_literal(dq, vmap):
    """Same as inverse_transform, one varblock at a time through the
    step-by-step procedures (slow; used to pin the batched form)."""
    out = np.zeros_like(dq)
    for c_, bx, by in varblocks(vmap):
        W, H = T.SHAPE_WH[c_]
        for c in range(3):
            blk = dq[c, 8 * by:8 * by + H, 8 * bx:8 * bx + W]
            if c_ in T.DCT_SHAPES:
                pix = TR.idct_2d(blk)
            else:
                pix = TR.idct_8x8_class(c_, blk)
            out[c, 8 * by:8 * by + H, 8 * bx:8 * bx + W] = pix
    return out


def reconstruct_xyb(coeffs, vmap, acmul, cfl, params):
    """Steps F, G, I: XYB samples of the padded image (FP64)."""
    return inverse_transform(dequantize(coeffs, vmap, acmul, cfl, params), vmap)


# ---------------------------------------------------------------------------
# J.2 edge-preserving filter
# ---------------------------------------------------------------------------
K_SIGMA_SHIFT = 2  # READING: undefined in the draft; 2 makes mul = -32768 the
                   # exact bound for the smallest sigma


def weight_bits(sad, mul4):
    """Weight() of J.2.4 as binary32 bit patterns, in exact integers.
    ``mul4`` is 4 * mul (mul is a multiple of 1/4 after interpolation)."""
    sad = np.minimum(np.asarray(sad, dtype=np.int64), 507)
    prescaled = sad << 6
    # (prescaled * mul) >> 16 == floor(prescaled * mul4 / 2^18)
    high16 = ((prescaled * np.asarray(mul4, dtype=np.int64)) >> 18) + (127 << 7)
    return (high16 << 16).astype(np.uint32)


def weight(sad, mul4):
    return weight_bits(sad, mul4).view(np.float32).astype(np.float64)


def mul_table4():
    """4 * mul_table[sigma] for sigma in [0, 672] (entries < 16 unused)."""
    tab = np.zeros(673, dtype=np.int64)
    gap = 4
    mul = -32768
    for sigma in range(16, 673, gap):
        while mul < 0:
            w = weight(sigma >> K_SIGMA_SHIFT, 4 * mul)
            if w > 0.5:
                break
            mul += 1
        tab[sigma] = 4 * mul
    for sigma in range(16, 672, gap):
        step4 = (tab[sigma + gap] - tab[sigma]) // gap  # exact: mul_step * 4
        assert (tab[sigma + gap] - tab[sigma]) % gap == 0
        for i in range(1, gap):
            tab[sigma + i] = tab[sigma] + i * step4
    return tab


def _f32(x):
    return np.asarray(x, dtype=np.float32)


def guide_scaled(img, params):
    """J.2.2 `scaled`, binary32 operation by operation: (in - min) * scale."""
    im3 = (params.target_nits_div50 * 50.0 / 250.0) ** (1.0 / 3.0)
    out = np.zeros(img.shape, dtype=np.float32)
    for c in range(3):
        mn = (-0.03 if c == 0 else 0.0) * im3
        t = _f32(img[c]) - np.float32(mn)
        out[c] = t * np.float32(params.epf_scale[c])
    return out


def guide(img, params):
    s = guide_scaled(img, params)
    return np.trunc(np.clip(s, np.float32(0), np.float32(255))).astype(np.int64)


def epf_sigma(img, vmap, acmul, sharpness, params):
    """Per 8x8 block sigma of J.2.4 (binary32 arithmetic), for the cropped
    image ``img`` (3, ysize, xsize).  READING: only in-image samples count
    toward a block's range."""
    _, ys, xs = img.shape
    s = guide_scaled(img, params)
    bh, bw = (ys + 7) // 8, (xs + 7) // 8
    r = np.zeros((bh, bw), dtype=np.float32)
    for by in range(bh):
        for bx in range(bw):
            blk = s[:, 8 * by:8 * by + 8, 8 * bx:8 * bx + 8]
            rc = [np.float32(blk[c].max() - blk[c].min()) for c in range(3)]
            r[by, bx] = max(rc)
    code, ox, oy = owner_map(vmap)
    rng = np.zeros((bh, bw), dtype=np.float32)
    for c_, bx0, by0 in varblocks(vmap):
        W, H = T.SHAPE_WH[c_]
        sl = (slice(by0, min(by0 + H // 8, bh)), slice(bx0, min(bx0 + W // 8, bw)))
        if sl[0].start >= bh or sl[1].start >= bw:
            continue
        rng[sl] = r[sl].max()
    sig = np.minimum(rng, np.float32(params.epf_range_max))
    sig = sig * np.float32(params.epf_range_mul)
    lut = _f32(params.epf_sharp_lut)[sharpness[:bh, :bw].astype(np.int64)]
    sig = sig * lut
    quant = np.float32(1.0) / _f32(acmul[:bh, :bw])
    sig = np.minimum(sig, quant * np.float32(params.epf_quant_mul))
    sig = np.minimum(sig, np.float32(params.epf_sigma_max))
    sigma = np.trunc(sig).astype(np.int64)
    return np.minimum(sigma, 672)   # READING: table ends at 672


EPF_OFFSETS = [(cx, cy) for cy in range(-3, 4) for cx in range(-3, 5)]


def epf(img, vmap, acmul, sharpness, params, region=None):
    """J.2 on the cropped image img (3, ysize, xsize), FP64.  ``region``
    (x0, y0, x1, y1) restricts the output to a window (sampled checks of
    large images); the result covers that window only."""
    _, ys, xs = img.shape
    if region is None:
        region = (0, 0, xs, ys)
    x0, y0, x1, y1 = region
    g = guide(img, params)
    sigma_blk = epf_sigma(img, vmap, acmul, sharpness, params)
    mt4 = mul_table4()
    px = np.arange(x0, x1)[None, :]
    py = np.arange(y0, y1)[:, None]

    def at(arr, dx, dy):
        return arr[..., mirror(py + dy, ys), mirror(px + dx, xs)]

    sad = np.zeros((56, y1 - y0, x1 - x0), dtype=np.int64)
    for i, (cx, cy) in enumerate(EPF_OFFSETS):
        acc = np.zeros((y1 - y0, x1 - x0), dtype=np.int64)
        for c in range(3):
            for iy in (-1, 0, 1):
                for ix in (-1, 0, 1, 2):
                    acc += np.abs(at(g[c], ix, iy) - at(g[c], cx + ix, cy + iy))
        sad[i] = acc
    sigma = sigma_blk[py // 8, px // 8]
    mul4 = mt4[np.maximum(sigma, 16)]
    w = weight(sad, mul4[None])
    w = np.where(w < params.epf_weight_min, 0.0, w)
    num = np.zeros((3, y1 - y0, x1 - x0))
    den = w.sum(axis=0)
    for i, (cx, cy) in enumerate(EPF_OFFSETS):
        num += at(img, cx, cy) * w[i][None]
    out = num / den[None]
    # READING: mul_table is undefined below sigma 16; such pixels pass through
    keep = sigma < 16
    return np.where(keep[None], img[:, y0:y1, x0:x1], out)


# ---------------------------------------------------------------------------
# J.4 Gaborish
# ---------------------------------------------------------------------------
def gaborish(img, params, region=None):
    """READING: the weights are used as given by C.10 (no 1e-6 factor)."""
    _, ys, xs = img.shape
    if region is None:
        region = (0, 0, xs, ys)
    x0, y0, x1, y1 = region
    px = np.arange(x0, x1)[None, :]
    py = np.arange(y0, y1)[:, None]
    out = np.zeros((3, y1 - y0, x1 - x0))
    for c in range(3):
        w1, w2 = params.gab_w1[c], params.gab_w2[c]
        norm = 1.0 + 4 * w1 + 4 * w2
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                taxi = abs(dx) + abs(dy)
                wt = (1.0, w1, w2)[taxi] / norm
                out[c] += wt * img[c][mirror(py + dy, ys), mirror(px + dx, xs)]
    return out


# ---------------------------------------------------------------------------
# L.2 XYB -> linear RGB, and the output encodings
# ---------------------------------------------------------------------------
def xyb_to_linear01(xyb, params):
    """(3, h, w) XYB -> (h, w, 3) linear RGB divided by 255 (range [0, 1])."""
    X, Y, B = xyb[0], xyb[1], xyb[2]
    gam = (Y + X, Y - X, B)
    mix = [gam[i] ** 3 + params.opsin_bias[i] for i in range(3)]
    M = params.inv_opsin
    div = params.target_nits_div50 * 50.0 / 250.0
    rgb = [(M[3 * r] * mix[0] + M[3 * r + 1] * mix[1] + M[3 * r + 2] * mix[2]) / div
           for r in range(3)]
    return np.stack(rgb, axis=-1) / 255.0


def srgb_u8(lin01):
    """IEC 61966-2-1 encoding to 8 bits, round half up (READING)."""
    x = np.clip(lin01, 0.0, 1.0)
    enc = np.where(x <= 0.0031308, 12.92 * x, 1.055 * np.power(x, 1 / 2.4) - 0.055)
    return np.floor(enc * 255.0 + 0.5).astype(np.uint8)


# ---------------------------------------------------------------------------
# Whole path
# ---------------------------------------------------------------------------
def reconstruct(inp, params):
    """Returns a dict with the padded XYB before filters, the cropped XYB
    after filters, and linear RGB in [0, 1] (h, w, 3)."""
    xyb = reconstruct_xyb(inp['coeffs'], inp['vmap'], inp['acmul'], inp['cfl'], params)
    ys, xs = inp['ysize'], inp['xsize']
    img = xyb[:, :ys, :xs]
    if params.epf:
        img = epf(img, inp['vmap'], inp['acmul'], inp['sharpness'], params)
    if params.gab:
        img = gaborish(img, params)
    return {'xyb_padded': xyb, 'xyb': img, 'rgb01': xyb_to_linear01(img, params)}
