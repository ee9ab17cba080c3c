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

Decisions that turn a real number into an integer (the guide bytes and the
sigma truncation of J.2.2/J.2.4, the window test of the F.2 smoothing) are
taken in real (FP64) arithmetic, as the draft writes them (5.4).  For
comparisons with an implementation in binary32, epf_decision_bounds,
epf_undetermined and dc_smooth_margin give the decisions that a bounded
perturbation of the input could change.
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
        self.dc_smooth = False        # F.2 adaptive DC smoothing
        self.lf_predict = False       # Annex H AC prediction
        self.qco = False              # J.3 quantization constraint (with EPF)
        self.qco_interval_mul = T.QCO_INTERVAL_MUL
        self.noise = False            # K.5 noise synthesis
        self.noise_lut = (0.0,) * 16  # C.4.8 LUT (u(10) / 1024 each)
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


def mirror_pad(arr, pad):
    """``arr`` (..., h, w) extended by ``pad`` samples on every side with the
    6.5 mirroring, so that shifted windows become plain slices."""
    h, w = arr.shape[-2:]
    rows = mirror(np.arange(-pad, h + pad), h)
    cols = mirror(np.arange(-pad, w + pad), w)
    return arr[..., rows[:, None], cols[None, :]]


def shifted(padded, pad, region, dx, dy):
    """The samples at (x + dx, y + dy) for (x, y) in ``region`` (x0, y0, x1,
    y1), read from an array made by mirror_pad with the same ``pad``."""
    x0, y0, x1, y1 = region
    return padded[..., pad + y0 + dy:pad + y1 + dy, pad + x0 + dx:pad + x1 + dx]


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
def dequantize(coeffs, vmap, acmul, cfl, params, diag=None):
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
    # F.2 DC dequantisation per 8x8 block (and adaptive smoothing), then G
    if params.dc_smooth:
        dcf = dc_smooth(dc_image(coeffs, vmap, params), params)
    else:
        dcf = dc_image(coeffs, vmap, params)
    dcf[0] = dcf[0] + params.kx_dc * dcf[1]
    dcf[2] = dcf[2] + params.kb_dc * dcf[1]
    # I.2.7 LLF from DC, per varblock
    for c_, bx, by in varblocks(vmap):
        W, H = T.SHAPE_WH[c_]
        for c in range(3):
            out[c, 8 * by:8 * by + H // 8, 8 * bx:8 * bx + W // 8] = \
                TR.llf_from_dc(dcf[c, by:by + H // 8, bx:bx + W // 8])
    # Annex H: prediction of the remaining W/4 x H/4 coefficients
    if params.lf_predict:
        info = ac_prediction(out, vmap, dcf, params)
        if diag is not None:
            diag.update(info)
    return out


# ---------------------------------------------------------------------------
# F.2 adaptive DC smoothing
# ---------------------------------------------------------------------------
DC_SMOOTH_W = (0.05226273532324128, 0.20345139757231578, 0.0334829185968739)


def dc_image(coeffs, vmap, params, dtype=np.float64):
    """Dequantised DC samples per 8x8 block, (3, Hp/8, Wp/8), before chroma
    from luma (F.2 with extra_levels 0): the DC of block (bx0+u, by0+v) of a
    varblock sits at its LLF slot (u, v)."""
    bh, bw = vmap.shape
    out = np.zeros((3, bh, bw), dtype=dtype)
    for c_, bx, by in varblocks(vmap):
        W, H = T.SHAPE_WH[c_]
        for c in range(3):
            q = coeffs[c, 8 * by:8 * by + H // 8, 8 * bx:8 * bx + W // 8].astype(dtype)
            out[c, by:by + H // 8, bx:bx + W // 8] = q * dtype(params.m_dc[c])
    return out


def _dc_window(dc, params):
    """The F.2 weighted average wa of the 3x3 neighbourhood of every sample
    off the border (weights for the centre, the 4 edge and the 4 corner
    neighbours), the centre s, and the half window dcq/2 per channel."""
    w0, w1, w2 = DC_SMOOTH_W
    d = np.asarray(dc, np.float64)
    s_ = d[:, 1:-1, 1:-1]
    edges = d[:, :-2, 1:-1] + d[:, 1:-1, :-2] + d[:, 1:-1, 2:] + d[:, 2:, 1:-1]
    corners = d[:, :-2, :-2] + d[:, :-2, 2:] + d[:, 2:, :-2] + d[:, 2:, 2:]
    wa = w0 * s_ + w1 * edges + w2 * corners
    half = 0.5 * np.asarray(params.m_dc, np.float64)[:, None, None]
    return wa, s_, half


def dc_smooth(dc, params):
    """F.2: each DC sample not on the first/last row/column of the DC image
    becomes the 3x3 weighted average wa of its neighbourhood when
    s - dcq/2 <= wa <= s + dcq/2 (real arithmetic).  READINGS: the averages
    read the unsmoothed image; dcq, the DcQuantField of C.5.2, is m_DC of
    the channel (no extra levels)."""
    out = np.array(dc, dtype=np.float64, copy=True)
    if out.shape[1] < 3 or out.shape[2] < 3:
        return out
    wa, s_, half = _dc_window(out, params)
    keep = (s_ - half <= wa) & (wa <= s_ + half)
    out[:, 1:-1, 1:-1] = np.where(keep, wa, s_)
    return out


def dc_smooth_margin(dc, params):
    """Distance of each sample's wa from the nearer end of its F.2 window
    [s - dcq/2, s + dcq/2] (infinite on the border, where no test is made):
    an evaluation whose error is below the margin takes the same decision."""
    d = np.asarray(dc, np.float64)
    out = np.full(d.shape, np.inf)
    if d.shape[1] < 3 or d.shape[2] < 3:
        return out
    wa, s_, half = _dc_window(d, params)
    out[:, 1:-1, 1:-1] = np.minimum(np.abs(wa - (s_ - half)), np.abs(s_ + half - wa))
    return out


# ---------------------------------------------------------------------------
# Annex H AC prediction (with I.2.6 / I.2.7 at N = 4)
# ---------------------------------------------------------------------------
LF_SMOOTH_W = (0.12, 0.2, 0.02)
LF_SMOOTH_RANGE = 1.7
GROUP_BLOCKS = 32            # 256 x 256 sample groups (6.2), in 8x8 blocks
_DCT_SHAPES = (T.DCT8, T.DCT16, T.DCT32, 6, 7, 8, 9, 10, 11)


def downsample4(code, llf):
    """I.2.6 with N = 4 from the LLF coefficients alone (the other
    coefficients zero): the 4x4 box means of that reconstruction, the
    reading pinned at N = 8 against the printed ScaleF form; for the 8x8-class
    shapes every cell is the (0, 0) coefficient (I.2.6.3)."""
    W, H = T.SHAPE_WH[code]
    if code in _DCT_SHAPES:
        coef = np.zeros((H, W))
        coef[:H // 8, :W // 8] = llf
        return TR.idct_2d(coef).reshape(H // 4, 4, W // 4, 4).mean(axis=(1, 3))
    return np.full((2, 2), llf[0, 0])


_LF4_INV = {}


def half_mean_scale():
    """The coefficient of frequency 1 of the 8-point IDCT whose two 4-sample
    halves average to +1 and -1 (the factor I.2.7.3 writes ScaleF(2, 8, 1);
    READING: the exact inverse of the half means, as the LLF-from-DC step
    at N = 8 takes the exact inverse of the 8x8 box mean)."""
    return 1.0 / TR.idct_matrix(8)[:4, 1].mean()


def lf_from_image4(code, img):
    """I.2.7 with N = 4: the top-left H/4 x W/4 coefficients from an
    H/4 x W/4 image of 4x4 means.  DCT shapes: the exact inverse of the 4x4
    box mean of the reconstruction from those coefficients (I.2.7.1 defines
    I.2.7 as the inverse of I.2.6).  Identity, DCT2, DCT4, AFV: AuxDCT2x2
    (I.2.3.2).  DCT8x4 / DCT4x8: half means and half differences
    (I.2.7.3; READING: the second formula printed for "DCT 8 x 4" is the
    4x8 one and its block11 is input(1, 1))."""
    W, H = T.SHAPE_WH[code]
    if code in _DCT_SHAPES:
        if code not in _LF4_INV:
            cx, cy = W // 4, H // 4
            M = np.zeros((cx * cy, cx * cy))
            for j in range(cx * cy):
                coef = np.zeros((H, W))
                coef[j // cx, j % cx] = 1.0
                M[:, j] = TR.idct_2d(coef).reshape(cy, 4, cx, 4).mean(axis=(1, 3)).reshape(-1)
            _LF4_INV[code] = np.linalg.inv(M)
        return (_LF4_INV[code] @ img.reshape(-1)).reshape(H // 4, W // 4)
    if code in (T.IDENTITY, T.DCT2, T.DCT4, T.AFV):
        return TR.aux_dct2x2(img, 2)
    s = half_mean_scale()
    tl, tr, bl, br = img[0, 0], img[0, 1], img[1, 0], img[1, 1]
    out = np.zeros((2, 2))
    if code == T.DCT8X4:          # two 8-tall, 4-wide halves side by side
        dc0, ac0 = (tl + bl) / 2, (tl - bl) / 2
        dc1, ac1 = (tr + br) / 2, (tr - br) / 2
        out[0, 0], out[0, 1] = (dc0 + dc1) / 2, (dc0 - dc1) / 2
        out[1, 0], out[1, 1] = ac0 * s, ac1 * s
    else:                         # DCT4x8: two 4-tall, 8-wide halves stacked
        dc0, ac0 = (tl + tr) / 2, (tl - tr) / 2
        dc1, ac1 = (bl + br) / 2, (bl - br) / 2
        out[0, 0], out[1, 0] = (dc0 + dc1) / 2, (dc0 - dc1) / 2
        out[0, 1], out[1, 1] = ac0 * s, ac1 * s
    return out


def lf_smooth(img, dcq):
    """Annex H smoothing of one group's DC2x2 image (2-sample ring
    included): samples off the 2-wide ring become the 3x3 weighted average
    wa when |wa - s| <= 1.7 dcq.  Returns the smoothed interior and the
    distance of wa from the nearer threshold (for tests)."""
    wc, we, wd = LF_SMOOTH_W
    s_ = img[2:-2, 2:-2]
    edges = img[1:-3, 2:-2] + img[2:-2, 1:-3] + img[2:-2, 3:-1] + img[3:-1, 2:-2]
    corners = img[1:-3, 1:-3] + img[1:-3, 3:-1] + img[3:-1, 1:-3] + img[3:-1, 3:-1]
    wa = wc * s_ + we * edges + wd * corners
    t = LF_SMOOTH_RANGE * dcq
    keep = (s_ - t <= wa) & (wa <= s_ + t)
    margin = np.minimum(np.abs(wa - (s_ - t)), np.abs(s_ + t - wa))
    return np.where(keep, wa, s_), margin


def ac_prediction(out, vmap, dcf, params):
    """Annex H on the dequantised coefficient planes ``out`` (in place):
    per 256 x 256 group, the DC2x2 image of the varblocks' 4x downsamples
    with a ring of the 1-block border of DC samples (mirrored at the image
    bounds, 6.5), each repeated 2x2; smoothing; then the W/4 x H/4
    coefficients of I.2.7 (N = 4) added outside the LLF corner.
    READINGS: the group size is counted in 8x8 blocks of the padded image;
    the ring and the DC2x2 image use the DC samples after F.2 and G; the
    prediction is added to coefficients after G, in the same colour
    space as the DC it derives from.  Returns the smoothed image and the
    threshold margins, (3, 2 bh, 2 bw) each."""
    bh, bw = vmap.shape
    U = np.zeros((3, 2 * bh, 2 * bw))
    for code, bx, by in varblocks(vmap):
        W, H = T.SHAPE_WH[code]
        for c in range(3):
            llf = out[c, 8 * by:8 * by + H // 8, 8 * bx:8 * bx + W // 8]
            U[c, 2 * by:2 * by + H // 4, 2 * bx:2 * bx + W // 4] = downsample4(code, llf)
    Us = np.zeros_like(U)
    margin = np.zeros_like(U)
    G = GROUP_BLOCKS
    for gy0 in range(0, bh, G):
        for gx0 in range(0, bw, G):
            gbw, gbh = min(G, bw - gx0), min(G, bh - gy0)
            ys = mirror(np.arange(gy0 - 1, gy0 + gbh + 1), bh)
            xs = mirror(np.arange(gx0 - 1, gx0 + gbw + 1), bw)
            sl = (slice(2 * gy0, 2 * (gy0 + gbh)), slice(2 * gx0, 2 * (gx0 + gbw)))
            for c in range(3):
                ring = dcf[c][np.ix_(ys, xs)]
                img = np.repeat(np.repeat(ring, 2, 0), 2, 1)
                img[2:-2, 2:-2] = U[c][sl]
                Us[c][sl], margin[c][sl] = lf_smooth(img, params.m_dc[c])
    for code, bx, by in varblocks(vmap):
        W, H = T.SHAPE_WH[code]
        mask = np.ones((H // 4, W // 4), dtype=bool)
        mask[:H // 8, :W // 8] = False
        for c in range(3):
            lf = lf_from_image4(code, Us[c, 2 * by:2 * by + H // 4, 2 * bx:2 * bx + W // 4])
            blk = out[c, 8 * by:8 * by + H // 4, 8 * bx:8 * bx + W // 4]
            blk[mask] += lf[mask]
    return {'lf_image': Us, 'lf_margin': margin}


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


def reconstruct_xyb(coeffs, vmap, acmul, cfl, params, diag=None):
    """Steps F, G, H, I: XYB samples of the padded image (FP64).  ``diag``
    (a dict) receives the Annex H intermediates when that step runs."""
    return inverse_transform(dequantize(coeffs, vmap, acmul, cfl, params, diag), vmap)


# ---------------------------------------------------------------------------
# J.2 edge-preserving filter
# ---------------------------------------------------------------------------
K_SIGMA_SHIFT = 2  # READING: undefined in the draft; 2 makes mul = -32768 the
                   # exact bound for the smallest sigma (Weight(16 >> 2, -32768)
                   # is exactly 0.5)


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


def guide_scaled(img, params):
    """J.2.2 `scaled` in real (FP64) arithmetic: (in - min[c]) * epf_scale[c],
    with min[c] = -0.03 * intensity_multiplier3 for X and 0 otherwise."""
    im3 = (params.target_nits_div50 * 50.0 / 250.0) ** (1.0 / 3.0)
    out = np.zeros(img.shape, dtype=np.float64)
    for c in range(3):
        mn = (-0.03 if c == 0 else 0.0) * im3
        out[c] = (np.asarray(img[c], np.float64) - mn) * params.epf_scale[c]
    return out


def guide_from_scaled(s):
    """J.2.2 guide sample: the scaled value clamped to [0, 255] and stored
    in 8 bits.  READING: the conversion truncates (C++ semantics, 5.4)."""
    return np.trunc(np.clip(s, 0.0, 255.0)).astype(np.int64)


def guide(img, params):
    return guide_from_scaled(guide_scaled(img, params))


def block_ranges(scaled, vmap):
    """J.2.4 `range` per 8x8 block of the cropped image: r[c] is the largest
    minus the smallest `scaled` sample of channel c in the block, all_r the
    largest of the three, and a block's range the largest all_r over the
    blocks of its varblock.  READING: only in-image samples count toward a
    block's r.  Accepts a pair (low, high) of scaled images instead of one:
    r is then taken as max(high) - min(low), the largest range that inputs
    between the two can have, or max(low) - min(high), the smallest (the
    pair is returned as (smallest, largest))."""
    if isinstance(scaled, tuple):
        lo, hi = scaled
        return (_block_ranges(lo, hi, vmap, smallest=True),
                _block_ranges(lo, hi, vmap, smallest=False))
    return _block_ranges(scaled, scaled, vmap, smallest=False)


def _block_ranges(lo, hi, vmap, smallest):
    _, ys, xs = lo.shape
    bh, bw = (ys + 7) // 8, (xs + 7) // 8
    r = np.zeros((bh, bw))
    for by in range(bh):
        for bx in range(bw):
            sl = (slice(None), slice(8 * by, 8 * by + 8), slice(8 * bx, 8 * bx + 8))
            a, b = lo[sl], hi[sl]
            if smallest:
                rc = [max(a[c].max() - b[c].min(), 0.0) for c in range(3)]
            else:
                rc = [b[c].max() - a[c].min() for c in range(3)]
            r[by, bx] = max(rc)
    rng = np.zeros((bh, bw))
    for c_, bx0, by0 in varblocks(vmap):
        W, H = T.SHAPE_WH[c_]
        if by0 >= bh or bx0 >= bw:
            continue
        sl = (slice(by0, min(by0 + H // 8, bh)), slice(bx0, min(bx0 + W // 8, bw)))
        rng[sl] = r[sl].max()
    return rng


def sigma_terms(rng, acmul, sharpness, params):
    """The two terms of J.2.4 sigma, per block, in real arithmetic: the
    range term min(range, range_max) * range_mul * sharp_lut[sharpness] and
    the quant term quant * quant_mul, quant = 1 / AcMul of the block."""
    bh, bw = rng.shape
    a = np.minimum(rng, params.epf_range_max) * params.epf_range_mul
    lut = np.asarray(params.epf_sharp_lut, np.float64)[sharpness[:bh, :bw].astype(np.int64)]
    a = a * lut
    q = (1.0 / np.asarray(acmul[:bh, :bw], np.float64)) * params.epf_quant_mul
    return a, q


def sigma_real(rng, acmul, sharpness, params):
    """J.2.4 sigma before truncation: min(range term, quant term, sigma_max)."""
    a, q = sigma_terms(rng, acmul, sharpness, params)
    return np.minimum(np.minimum(a, q), params.epf_sigma_max)


def sigma_from_real(sig):
    """truncate(), then READING: the mul table ends at 672."""
    return np.minimum(np.trunc(sig).astype(np.int64), 672)


def epf_sigma(img, vmap, acmul, sharpness, params):
    """Per 8x8 block sigma of J.2.4 (real arithmetic) for the cropped image
    ``img`` (3, ysize, xsize)."""
    rng = block_ranges(guide_scaled(img, params), vmap)
    return sigma_from_real(sigma_real(rng, acmul, sharpness, params))


# ---------------------------------------------------------------------------
# Decisions of J.2 under uncertain input (for comparisons with binary32)
# ---------------------------------------------------------------------------
def epf_decision_bounds(img, vmap, acmul, sharpness, params, slack=0.0, guide_alt=None,
                        sigma_alt=None):
    """The J.2 decisions for every input whose scaled guide samples lie
    within +-slack of those of ``img`` (slack: scalar or per sample, in
    guide units), joined with the decisions of another evaluation (for
    instance binary32 arithmetic on another image of the same content):
    ``guide_alt`` its guide bytes (3, h, w), ``sigma_alt`` its block sigmas.
    Returns (g_lo, g_hi, s_lo, s_hi): the smallest and largest guide bytes
    and block sigmas reachable.  A decision is fixed where the two agree;
    where they differ the input lies within the bound of a threshold and
    either outcome is correct."""
    s = guide_scaled(img, params)
    lo, hi = s - slack, s + slack
    r_lo, r_hi = block_ranges((lo, hi), vmap)
    g_lo, g_hi = guide_from_scaled(lo), guide_from_scaled(hi)
    s_lo = sigma_from_real(sigma_real(r_lo, acmul, sharpness, params))
    s_hi = sigma_from_real(sigma_real(r_hi, acmul, sharpness, params))
    if guide_alt is not None:
        g_lo, g_hi = np.minimum(g_lo, guide_alt), np.maximum(g_hi, guide_alt)
    if sigma_alt is not None:
        s_lo, s_hi = np.minimum(s_lo, sigma_alt), np.maximum(s_hi, sigma_alt)
    return g_lo, g_hi, s_lo, s_hi


def epf_undetermined(img, vmap, acmul, sharpness, params, slack=0.0, region=None,
                     guide_alt=None, sigma_alt=None):
    """Pixels of the J.2 output (over ``region``) that the input does not
    determine when its guide samples and sigmas are known only within the
    bounds of epf_decision_bounds: a pixel is undetermined if its block's
    sigma is not fixed and some outcome filters it with a non-centre weight
    at or above the cut-off, or if its sigma is fixed at >= 16 and for some
    offset the guide bytes that are not fixed could bring the patch SAD to
    a weight at or above the cut-off (each byte that is not fixed moves the
    SAD by at most 1).  Everywhere else every reachable set of decisions
    gives the same weights, hence the same output."""
    _, ys, xs = img.shape
    if region is None:
        region = (0, 0, xs, ys)
    x0, y0, x1, y1 = region
    g_lo, g_hi, s_lo, s_hi = epf_decision_bounds(img, vmap, acmul, sharpness, params,
                                                 slack, guide_alt, sigma_alt)
    g = guide(img, params).astype(np.int32)
    loose = (g_lo != g_hi).astype(np.int32)
    mt4 = mul_table4()
    px = np.arange(x0, x1)[None, :]
    py = np.arange(y0, y1)[:, None]
    P = _EPF_PAD
    gp, lp = mirror_pad(g, P), mirror_pad(loose, P)
    blo = s_lo[py // 8, px // 8]
    bhi = s_hi[py // 8, px // 8]
    mul_hi = mt4[np.clip(bhi, 16, 672)]       # the largest weights: largest sigma

    def one(i, off):
        cx, cy = off
        if cx == 0 and cy == 0:
            return None                       # the centre's SAD is 0 on any input
        sad = _patch_sad(gp, P, region, cx, cy)
        # guide bytes that are not fixed, counted over both patches
        k = np.zeros_like(sad)
        for c in range(3):
            for iy in (-1, 0, 1):
                for ix in (-1, 0, 1, 2):
                    k += (shifted(lp[c], P, region, ix, iy)
                          + shifted(lp[c], P, region, cx + ix, cy + iy))
        live = weight(np.maximum(sad - k, 0), mul_hi) >= params.epf_weight_min
        return (((bhi >= 16) & (blo != bhi) & live)
                | ((blo >= 16) & (blo == bhi) & (k > 0) & live))

    out = np.zeros((y1 - y0, x1 - x0), dtype=bool)
    for m in _map_offsets(one):
        if m is not None:
            out |= m
    return out


EPF_OFFSETS = [(cx, cy) for cy in range(-3, 4) for cx in range(-3, 5)]
_EPF_PAD = 8        # reach of a patch at the farthest offset: x - 4 .. x + 6, y +- 4


def _patch_sad(gp, P, region, cx, cy):
    """J.2.3 distance for one offset (cx, cy) at every pixel of ``region``:
    the sum over the 3 channels and the 3x4 patch (rows -1..1, columns
    -1..2 around the origin) of |g(p + d) - g(p + (cx, cy) + d)|."""
    x0, y0, x1, y1 = region
    acc = np.zeros((y1 - y0, x1 - x0), dtype=np.int32)
    for c in range(3):
        for iy in (-1, 0, 1):
            for ix in (-1, 0, 1, 2):
                acc += np.abs(shifted(gp[c], P, region, ix, iy)
                              - shifted(gp[c], P, region, cx + ix, cy + iy))
    return acc


THREADS = None      # worker threads of the J.2 offset loop; None: every host core


def _map_offsets(fn):
    """fn(i, (cx, cy)) for the 56 offsets, evaluated on a thread pool of
    THREADS workers (the work is numpy array arithmetic); results in offset
    order."""
    import concurrent.futures as cf
    import os
    n = THREADS or os.cpu_count() or 1
    if n == 1:
        return [fn(i, off) for i, off in enumerate(EPF_OFFSETS)]
    with cf.ThreadPoolExecutor(max_workers=n) as ex:
        return list(ex.map(lambda a: fn(*a), enumerate(EPF_OFFSETS)))


def epf(img, vmap, acmul, sharpness, params, region=None, decide=None):
    """J.2 on the cropped image img (3, ysize, xsize), FP64.  ``region``
    (x0, y0, x1, y1) restricts the output to a window (sampled checks of
    large images); the result covers that window only.  ``decide`` (an image
    of the same shape, for tests) supplies the guide and the sigmas instead
    of ``img``; the weighted samples are always those of ``img``."""
    _, ys, xs = img.shape
    if region is None:
        region = (0, 0, xs, ys)
    x0, y0, x1, y1 = region
    d = img if decide is None else decide
    g = guide(d, params).astype(np.int32)
    sigma_blk = epf_sigma(d, vmap, acmul, sharpness, params)
    mt4 = mul_table4()
    px = np.arange(x0, x1)[None, :]
    py = np.arange(y0, y1)[:, None]
    P = _EPF_PAD
    gp, ip = mirror_pad(g, P), mirror_pad(np.asarray(img, np.float64), P)
    sigma = sigma_blk[py // 8, px // 8]
    mul4 = mt4[np.maximum(sigma, 16)]

    def one(i, off):
        # J.2.4 weight of this offset, zero below the cut-off; J.2.5 terms
        cx, cy = off
        w = weight(_patch_sad(gp, P, region, cx, cy), mul4)
        w = np.where(w < params.epf_weight_min, 0.0, w)
        return w, shifted(ip, P, region, cx, cy) * w[None]

    parts = _map_offsets(one)
    den = np.zeros((y1 - y0, x1 - x0))
    num = np.zeros((3, y1 - y0, x1 - x0))
    for w, t in parts:                 # J.2.5 sums in offset order
        den += w
        num += t
    out = num / den[None]
    # READING: mul_table is undefined below sigma 16; such pixels pass through
    keep = sigma < 16
    return np.where(keep[None], img[:, y0:y1, x0:x1], out)


# ---------------------------------------------------------------------------
# J.3 quantization constraint
# ---------------------------------------------------------------------------
_FORWARD_8X8 = {T.DCT2: TR.dct_dct2, T.DCT4: TR.dct_dct4, T.IDENTITY: TR.dct_identity,
                T.DCT8X4: TR.dct_dct8x4, T.DCT4X8: TR.dct_dct4x8, T.AFV: TR.dct_afv}


def forward_transform(code, samples):
    """I.2.3: the coefficients whose I.2.4 reconstruction is ``samples``
    (the DCT shapes: the 2-D DCT divided by the sample count, the exact
    inverse of the IDCT's orthogonal cosine sums)."""
    if code in _DCT_SHAPES:
        H, W = samples.shape
        return TR.dct_2d(samples) / (H * W)
    return _FORWARD_8X8[code](samples)


def inverse_any(code, coef):
    """I.2.4 for one varblock of any shape."""
    return TR.idct_2d(coef) if code in _DCT_SHAPES else TR.idct_8x8_class(code, coef)


def qco(filtered, original, vmap, acmul, params):
    """J.3 on the EPF output ``filtered`` (3, ys, xs) with the EPF input
    ``original`` (padded, 3 x Hp x Wp): per varblock and channel, the DCT of
    the filter residual (I.2.3), its LLF turned into DC samples (I.2.6), each
    value clamped to +-qco_interval_mul x interval, DC back to LLF (I.2.7),
    the inverse transform (I.2.4) added to the EPF input.  READINGS: the
    interval of an HF coefficient is the dequantisation step of F.3, AcMul x
    the C.6.1 matrix entry (the text divides by AcMul while F.3 multiplies);
    that of a DC sample is m_DC (DcQuantField without extra levels); samples
    of a varblock outside the cropped image have zero residual.  Returns the
    cropped result."""
    _, ys, xs = filtered.shape
    _, Hp, Wp = original.shape
    res = np.zeros((3, Hp, Wp))
    res[:, :ys, :xs] = filtered - original[:, :ys, :xs]
    out = original.copy()
    mul = params.qco_interval_mul
    for code, bx, by in varblocks(vmap):
        W, H = T.SHAPE_WH[code]
        cx, cy = W // 8, H // 8
        sl = (slice(8 * by, 8 * by + H), slice(8 * bx, 8 * bx + W))
        am = float(acmul[by, bx])
        for c in range(3):
            coef = forward_transform(code, res[c][sl])
            lim = mul * am * T.dequant_matrix(code, c)
            clamped = np.clip(coef, -lim, lim)
            if code in _DCT_SHAPES:
                dc = (TR.box_mean_map(W, H) @ coef[:cy, :cx].reshape(-1)).reshape(cy, cx)
            else:
                dc = coef[:1, :1].copy()
            t = mul * params.m_dc[c]
            dc = np.clip(dc, -t, t)
            clamped[:cy, :cx] = TR.llf_from_dc(dc) if code in _DCT_SHAPES else dc
            out[c][sl] = original[c][sl] + inverse_any(code, clamped)
    return out[:, :ys, :xs]


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
def reconstruct(inp, params, diag=None):
    """Returns a dict with the padded XYB before filters, the cropped XYB
    after filters, and linear RGB in [0, 1] (h, w, 3)."""
    xyb = reconstruct_xyb(inp['coeffs'], inp['vmap'], inp['acmul'], inp['cfl'], params, diag)
    ys, xs = inp['ysize'], inp['xsize']
    img = xyb[:, :ys, :xs]
    if params.epf:
        img = epf(img, inp['vmap'], inp['acmul'], inp['sharpness'], params)
        if params.qco:
            img = qco(img, xyb, inp['vmap'], inp['acmul'], params)
    if params.gab:
        img = gaborish(img, params)
    if params.noise:                  # K.5, after Gaborish (9.12 ordering)
        from . import noise as NZ
        img = NZ.add_noise(img, params.noise_lut)
    return {'xyb_padded': xyb, 'xyb': img, 'rgb01': xyb_to_linear01(img, params)}
