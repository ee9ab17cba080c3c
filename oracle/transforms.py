"""Inverse (and, for the pins, forward) integral transforms of I.2, in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Matrices are indexed [row][column] = [y][x]; a varblock of width W and height
H is an H x W array.  The coefficient at array position [v][u] has horizontal
frequency u and vertical frequency v (READING: I.2.2 prints the square case
without the final transpose of the non-square case; this oracle reads every
shape in the orientation of the non-square case).

The DCT-based shapes use the plain definition: cosine sums with the
per-frequency scale of the draft's one-dimensional transforms,

    IDCT_N[n][k] = S_N(k) * cos((2n + 1) k pi / (2N)),
    S_N(0) = 1,  S_8(k) = 1 / cos(k pi / 16),  S_N(k) = 2 cos(k pi / 2N), N != 8

(I.2.1 butterflies for N = 8, the Annex R generator for N = 2, 4, 16, 32).
The 8x8-class shapes (DCT2, DCT4, Identity, 8x4, 4x8, AFV) follow their
I.2.4 procedures step by step.
"""
import math

import numpy as np

from . import tables as T


# ---------------------------------------------------------------------------
# One-dimensional transforms (I.2.1, Annex R)
# ---------------------------------------------------------------------------
def idct_scale(N, k):
    if k == 0:
        return 1.0
    if N == 8:
        return 1.0 / math.cos(k * math.pi / 16.0)
    return 2.0 * math.cos(k * math.pi / (2.0 * N))


def idct_matrix(N):
    """IDCT_N[n][k]: sample n from frequency k."""
    m = np.zeros((N, N))
    for n in range(N):
        for k in range(N):
            m[n, k] = idct_scale(N, k) * math.cos((2 * n + 1) * k * math.pi / (2.0 * N))
    return m


def dct_matrix(N):
    """Forward transform paired with idct_matrix: DCT_N @ IDCT_N = N * I."""
    return N * np.linalg.inv(idct_matrix(N))


_IDCT = {N: idct_matrix(N) for N in (1, 2, 4, 8, 16, 32)}
_DCT = {N: dct_matrix(N) for N in (1, 2, 4, 8, 16, 32)}


def idct_2d(coef):
    """IDCT_2D of I.2.2 for an H x W coefficient array (orientation above)."""
    H, W = coef.shape
    return _IDCT[H] @ coef @ _IDCT[W].T


def dct_2d(samples):
    H, W = samples.shape
    return _DCT[H] @ samples @ _DCT[W].T


def idct_2d_bruteforce(coef):
    """The O(N^4) cosine-sum definition, used by the pins only."""
    H, W = coef.shape
    out = np.zeros((H, W))
    for m in range(H):
        for n in range(W):
            s = 0.0
            for v in range(H):
                for u in range(W):
                    s += (coef[v, u] * idct_scale(W, u) * idct_scale(H, v)
                          * math.cos((2 * n + 1) * u * math.pi / (2.0 * W))
                          * math.cos((2 * m + 1) * v * math.pi / (2.0 * H)))
            out[m, n] = s
    return out


# ---------------------------------------------------------------------------
# I.2.3.2 / I.2.4.2 two-by-two pyramid steps.  A(x, y) is a[y][x].
# ---------------------------------------------------------------------------
def aux_dct2x2(block, S):
    out = block.copy()
    h = S // 2
    for y in range(h):
        for x in range(h):
            c00 = block[2 * y, 2 * x]
            c01 = block[2 * y, 2 * x + 1]
            c10 = block[2 * y + 1, 2 * x]
            c11 = block[2 * y + 1, 2 * x + 1]
            out[y, x] = (c00 + c01 + c10 + c11) / 4
            out[y, h + x] = (c00 + c01 - c10 - c11) / 4
            out[y + h, x] = (c00 - c01 + c10 - c11) / 4
            out[y + h, h + x] = (c00 - c01 - c10 + c11) / 4
    return out


def aux_idct2x2(block, S):
    out = block.copy()
    h = S // 2
    for y in range(h):
        for x in range(h):
            c00 = block[y, x]
            c01 = block[y, h + x]
            c10 = block[y + h, x]
            c11 = block[y + h, h + x]
            out[2 * y, 2 * x] = c00 + c01 + c10 + c11
            out[2 * y, 2 * x + 1] = c00 + c01 - c10 - c11
            out[2 * y + 1, 2 * x] = c00 - c01 + c10 - c11
            out[2 * y + 1, 2 * x + 1] = c00 - c01 - c10 + c11
    return out


# ---------------------------------------------------------------------------
# I.2.4 coefficients to samples for the 8x8-class shapes
# ---------------------------------------------------------------------------
def idct_dct2(coef):
    b = aux_idct2x2(coef, 2)
    b = aux_idct2x2(b, 4)
    return aux_idct2x2(b, 8)


def idct_dct4(coef):
    dcs = aux_idct2x2(coef, 2)
    out = np.zeros((8, 8))
    for y in range(2):
        for x in range(2):
            block = np.zeros((4, 4))
            for iy in range(4):
                for ix in range(4):
                    if ix == 0 and iy == 0:
                        continue
                    block[iy, ix] = coef[y + 2 * iy, x + 2 * ix]
            block[0, 0] = dcs[y, x]
            out[4 * y:4 * y + 4, 4 * x:4 * x + 4] = idct_2d(block)
    return out


def idct_identity(coef):
    dcs = aux_idct2x2(coef, 2)
    out = np.zeros((8, 8))
    for y in range(2):
        for x in range(2):
            block_dc = dcs[y, x]
            residual_sum = 0.0
            for iy in range(4):
                for ix in range(4):
                    if ix == 0 and iy == 0:
                        continue
                    residual_sum += coef[y + 2 * iy, x + 2 * ix]
            s11 = block_dc - residual_sum / 16.0
            out[4 * y + 1, 4 * x + 1] = s11
            for iy in range(4):
                for ix in range(4):
                    if ix == 1 and iy == 1:
                        continue
                    out[4 * y + iy, 4 * x + ix] = coef[y + 2 * iy, x + 2 * ix] + s11
            out[4 * y, 4 * x] = coef[y + 2, x + 2] + s11
    return out


def idct_dct8x4(coef):
    """Two 8-tall, 4-wide blocks side by side (I.2.4.5)."""
    c0, c1 = coef[0, 0], coef[0, 1]
    dcs = (c0 + c1, c0 - c1)
    out = np.zeros((8, 8))
    for x in range(2):
        blk = np.zeros((8, 4))
        for iy in range(8):
            for ix in range(4):
                if ix == 0 and iy == 0:
                    continue
                blk[iy, ix] = coef[iy, x + 2 * ix]
        blk[0, 0] = dcs[x]
        out[:, 4 * x:4 * x + 4] = idct_2d(blk)
    return out


def idct_dct4x8(coef):
    """Two 4-tall, 8-wide blocks stacked (I.2.4.6).  READING: the DC of the
    y-th block is dcs[y] (the draft prints dcs[x] inside the y loop)."""
    c0, c1 = coef[0, 0], coef[1, 0]
    dcs = (c0 + c1, c0 - c1)
    out = np.zeros((8, 8))
    for y in range(2):
        blk = np.zeros((4, 8))
        for iy in range(4):
            for ix in range(8):
                if ix == 0 and iy == 0:
                    continue
                blk[iy, ix] = coef[y + 2 * iy, ix]
        blk[0, 0] = dcs[y]
        out[4 * y:4 * y + 4, :] = idct_2d(blk)
    return out


def afv_idct(coeffs16):
    """AFV_IDCT of I.2.2: samples[i] = sum_j coefficients[j] * AFVBasis[j][i]."""
    return coeffs16 @ T.AFV_BASIS


def afv_dct(samples16):
    return T.AFV_BASIS @ samples16


def idct_afv(coef):
    c1, c2, c3, c4 = (coef[0, 0] * 4.0, coef[0, 1] * 4.0,
                      coef[1, 0] * 4.0, coef[1, 1] * 4.0)
    dcs = (c1 + c2 + c3 + c4, c1 + c2 - c3 - c4,
           c1 - c2 + c3 - c4, c1 - c2 - c3 + c4)
    out = np.zeros((8, 8))
    for y in range(2):
        for x in range(2):
            ca = np.zeros(16)
            for iy in range(4):
                for ix in range(4):
                    if ix == 0 and iy == 0:
                        continue
                    ca[4 * iy + ix] = coef[y + 2 * iy, x + 2 * ix]
            ca[0] = dcs[2 * y + x]
            sa = afv_idct(ca)
            for iy in range(4):
                for ix in range(4):
                    sx = 3 - ix if x else ix
                    sy = 3 - iy if y else iy
                    out[4 * y + iy, 4 * x + ix] = sa[4 * sy + sx]
    return out


# ---------------------------------------------------------------------------
# Forward transforms of I.2.3 for the 8x8-class shapes (pins only)
# ---------------------------------------------------------------------------
def dct_dct2(samples):
    t = aux_dct2x2(samples, 8)
    t = aux_dct2x2(t, 4)
    return aux_dct2x2(t, 2)


def dct_dct4(samples):
    out = np.zeros((8, 8))
    for y in range(2):
        for x in range(2):
            sub = dct_2d(samples[4 * y:4 * y + 4, 4 * x:4 * x + 4]) / 16.0
            for iy in range(4):
                for ix in range(4):
                    out[y + 2 * iy, x + 2 * ix] = sub[iy, ix]
    return aux_dct2x2(out, 2)


def dct_identity(samples):
    out = np.zeros((8, 8))
    for y in range(2):
        for x in range(2):
            blk = samples[4 * y:4 * y + 4, 4 * x:4 * x + 4]
            block_dc = blk.sum() / 16.0
            for iy in range(4):
                for ix in range(4):
                    if ix == 1 and iy == 1:
                        continue
                    out[y + 2 * iy, x + 2 * ix] = blk[iy, ix] - blk[1, 1]
            out[y + 2, x + 2] = out[y, x]
            out[y, x] = block_dc
    return aux_dct2x2(out, 2)


def idct_8x8_class(code, coef):
    if code == T.DCT2:
        return idct_dct2(coef)
    if code == T.DCT4:
        return idct_dct4(coef)
    if code == T.IDENTITY:
        return idct_identity(coef)
    if code == T.DCT8X4:
        return idct_dct8x4(coef)
    if code == T.DCT4X8:
        return idct_dct4x8(coef)
    if code == T.AFV:
        return idct_afv(coef)
    raise ValueError(code)


# ---------------------------------------------------------------------------
# I.2.6 / I.2.7 LLF <-> DC.  The DC sample of an 8x8 sub-block is the mean of
# the LLF-only reconstruction over that sub-block; the LLF coefficients are
# the exact inverse of that map (READING: I.2.7.1 defines I.2.7 as the
# inverse of I.2.6; the printed I.2.7.2 formula differs from it by the number
# of 8x8 sub-blocks).
# ---------------------------------------------------------------------------
def box_mean_map(W, H):
    """Matrix M with dc = M @ llf (both flattened row-major, cy x cx)."""
    cx, cy = W // 8, H // 8
    M = np.zeros((cx * cy, cx * cy))
    for j in range(cy * cx):
        coef = np.zeros((H, W))
        coef[j // cx, j % cx] = 1.0
        pix = idct_2d(coef)
        means = pix.reshape(cy, 8, cx, 8).mean(axis=(1, 3))
        M[:, j] = means.reshape(-1)
    return M


_LLF_FROM_DC = {}


def llf_from_dc(dc):
    """dc: cy x cx array of DC samples of one varblock -> LLF coefficients."""
    cy, cx = dc.shape
    key = (cx, cy)
    if key not in _LLF_FROM_DC:
        _LLF_FROM_DC[key] = np.linalg.inv(box_mean_map(8 * cx, 8 * cy))
    return (_LLF_FROM_DC[key] @ dc.reshape(-1)).reshape(cy, cx)


def downsample_scalef(coef, N=8):
    """I.2.6.2 as printed: the LF coefficients scaled by ScaleF, then an
    IDCT of the LF size.  Used only to pin box_mean_map."""
    H, W = coef.shape
    cx, cy = W // N, H // N
    llf = np.zeros((cy, cx))
    for y in range(cy):
        for x in range(cx):
            llf[y, x] = coef[y, x] * T.ScaleF(H, cy, y) * T.ScaleF(W, cx, x)
    return idct_2d(llf)


def dct_dct8x4(samples):
    """I.2.3.5, divided by the 32 samples of each half so that it inverts
    idct_dct8x4 exactly."""
    out = np.zeros((8, 8))
    for x in range(2):
        c84 = dct_2d(samples[:, 4 * x:4 * x + 4]) / 32.0
        for iy in range(8):
            for ix in range(4):
                out[iy, x + 2 * ix] = c84[iy, ix]
    c0, c1 = out[0, 0], out[0, 1]
    out[0, 0] = (c0 + c1) * 0.5
    out[0, 1] = (c0 - c1) * 0.5
    return out


def dct_dct4x8(samples):
    """I.2.3.6, normalised like dct_dct8x4."""
    out = np.zeros((8, 8))
    for y in range(2):
        c48 = dct_2d(samples[4 * y:4 * y + 4, :]) / 32.0
        for iy in range(4):
            for ix in range(8):
                out[y + 2 * iy, ix] = c48[iy, ix]
    c0, c1 = out[0, 0], out[1, 0]
    out[0, 0] = (c0 + c1) * 0.5
    out[1, 0] = (c0 - c1) * 0.5
    return out


def dct_afv(samples):
    """I.2.3.7 (four mirrored 4x4 quadrants through AFV_DCT)."""
    out = np.zeros((8, 8))
    for y in range(2):
        for x in range(2):
            sa = np.zeros(16)
            for iy in range(4):
                for ix in range(4):
                    sx = 3 - ix if x else ix
                    sy = 3 - iy if y else iy
                    sa[4 * sy + sx] = samples[4 * y + iy, 4 * x + ix]
            ca = afv_dct(sa)
            for iy in range(4):
                for ix in range(4):
                    out[y + 2 * iy, x + 2 * ix] = ca[4 * iy + ix]
    c1, c2 = out[0, 0] * 0.25, out[0, 1] * 0.25
    c3, c4 = out[1, 0] * 0.25, out[1, 1] * 0.25
    out[0, 0] = (c1 + c2 + c3 + c4) * 0.25
    out[0, 1] = (c1 + c2 - c3 - c4) * 0.25
    out[1, 0] = (c1 - c2 + c3 - c4) * 0.25
    out[1, 1] = (c1 - c2 - c3 + c4) * 0.25
    return out
