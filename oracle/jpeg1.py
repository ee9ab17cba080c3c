"""JPEG1 direct rasterisation (M.6 of the draft), in FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Steps, per component, then per pixel:
  M.6.1  dequantisation  dst[8u + v] = src[8u + v] * Q[8u + v] * I(8, u) * I(8, v)
  M.6.2  IDCT_2D of I.2.2 per 8x8 block
  M.6.3  block-conditional Gaborish (optional side channel)
  M.6.4  2x linear upsampling of subsampled components, horizontal first,
         mirrored so that index -1 reads index 1
  M.6.5  YCbCr -> RGB
  M.6.6  crop to the image size

Coefficients are given per component as ``coeffs[by][bx][64]`` in the
natural order of M.6.1 (index 8u + v: u the vertical, v the horizontal
frequency).  The DC/AC conditioning of M.6.1.1 runs when a component
carries ``cond = (max_gap, min_step)``.  The HDR colour-space transform of
M.6.5.1 is outside this path.

READINGS (M.6.1.1): the garbled indices dc(y, start), ac_h(x, start - 1) and
has_v[v, u] are dc(start, y), ac_h(start - 1, y) and has_v[x, y]; the bullet
"abs(to - from) > min_step" is a third condition of is_sane;
dc_multiplier is Q[0] I(8, 0) I(8, 0) for the three replaced coefficients
(it is defined once, before the loop; with it a slope of -delta/2 per block
makes the block's samples change by about delta across its width).  The
plateau arithmetic (from, to, the sanity tests, the interpolation) is done
in binary32, operation by operation, as in the kernels, because its
comparisons decide which coefficients are replaced.
"""
import numpy as np

from . import tables as T
from . import transforms as TR


def dequantize_block(src, quant):
    """M.6.1 for one block: 8x8 array [u][v] of dequantised coefficients."""
    out = np.zeros((8, 8))
    for u in range(8):
        for v in range(8):
            k = 8 * u + v
            out[u, v] = float(src[k]) * float(quant[k]) * T.I(8, u) * T.I(8, v)
    return out


def _plateaus(dc, ac, q_ratio, max_gap, min_step):
    """M.6.1.1 along the rows of dc / ac ((n, m) int arrays; rows are
    independent): approximations, slopes and the flags, binary32."""
    f32 = np.float32
    n, m = dc.shape
    approx = np.zeros((n, m), f32)
    slope = np.zeros((n, m), f32)
    has = np.zeros((n, m), bool)
    q = f32(q_ratio)
    for y in range(n):
        x = 0
        while x < m:
            end = x
            while end + 1 < m and dc[y, end + 1] == dc[y, x]:
                end += 1
            start = x
            x = end + 1
            if start == 0 and end == m - 1:
                continue
            if np.any(ac[y, start:end + 1] != 0):
                continue
            cur = f32(dc[y, start])
            if start == 0:
                frm = cur
            else:
                frm = f32(0.5) * f32(f32(cur + f32(dc[y, start - 1])) + f32(q * f32(ac[y, start - 1])))
            if end == m - 1:
                to = cur
            else:
                to = f32(0.5) * f32(f32(cur + f32(dc[y, end + 1])) + f32(q * f32(ac[y, end + 1])))
            sane = (abs(f32(to - cur)) <= f32(max_gap) and abs(f32(cur - frm)) <= f32(max_gap)
                    and abs(f32(to - frm)) > f32(min_step))
            if not sane:
                continue
            span = f32(end - start + 1)
            ratio = f32(f32(to - frm) / span)
            for xx in range(start, end + 1):
                i = f32(xx - start)
                approx[y, xx] = f32(frm + f32(f32(f32(0.5) + i) * ratio))
                slope[y, xx] = f32(f32(-0.5) * ratio)
                has[y, xx] = True
    return approx, slope, has


def conditioning(coeffs, quant, max_gap, min_step):
    """M.6.1.1: per block the DC to use (in DC quantisation steps) and the
    replacements of coefficients 1 and 8 (in the same units), or None."""
    dc = coeffs[:, :, 0].astype(np.int64)
    hq = float(np.float32(quant[1]) / np.float32(quant[0]))
    vq = float(np.float32(quant[8]) / np.float32(quant[0]))
    ha, hs, hh = _plateaus(dc, coeffs[:, :, 1].astype(np.int64), hq, max_gap, min_step)
    va, vs, vh = _plateaus(dc.T, coeffs[:, :, 8].astype(np.int64).T, vq, max_gap, min_step)
    va, vs, vh = va.T, vs.T, vh.T
    f32 = np.float32
    approx = np.where(hh & vh, f32(0.5) * (ha + va), np.where(hh, ha, np.where(vh, va, dc.astype(f32))))
    return approx.astype(np.float64), hs.astype(np.float64), hh, vs.astype(np.float64), vh


def component_pixels(coeffs, quant, cond=None):
    """M.6.1 (+ M.6.1.1 when cond = (max_gap, min_step)) + M.6.2: the
    component's sample plane (8 bh, 8 bw); values are level-shifted (about
    -128..127)."""
    bh, bw = coeffs.shape[:2]
    plane = np.zeros((8 * bh, 8 * bw))
    if cond is not None:
        approx, hs, hh, vs, vh = conditioning(coeffs, quant, *cond)
        mult = float(quant[0]) * T.I(8, 0) * T.I(8, 0)
    for by in range(bh):
        for bx in range(bw):
            blk = dequantize_block(coeffs[by, bx], quant)
            if cond is not None:
                blk[0, 0] = approx[by, bx] * mult
                if hh[by, bx]:
                    blk[0, 1] = hs[by, bx] * mult
                if vh[by, bx]:
                    blk[1, 0] = vs[by, bx] * mult
            plane[8 * by:8 * by + 8, 8 * bx:8 * bx + 8] = TR.idct_2d(blk)
    return plane


def _mirror(i, n):
    """6.5 mirroring at the plane bounds."""
    while i < 0 or i >= n:
        i = -i - 1 if i < 0 else 2 * n - 1 - i
    return i


def gaborish_plane(plane, w1, w2):
    """J.4 on one plane with the weights (1, w1, w2) normalised to sum 1,
    mirrored at the plane bounds (6.5)."""
    h, w = plane.shape
    norm = 1.0 + 4 * w1 + 4 * w2
    ys = np.array([[_mirror(y + d, h) for y in range(h)] for d in (-1, 0, 1)])
    xs = np.array([[_mirror(x + d, w) for x in range(w)] for d in (-1, 0, 1)])
    out = np.zeros_like(plane)
    for dy in range(3):
        for dx in range(3):
            wt = 1.0 if (dy == 1 and dx == 1) else (w1 if (dy == 1 or dx == 1) else w2)
            out += wt * plane[np.ix_(ys[dy], xs[dx])]
    return out / norm


def conditional_gaborish(plane, w1, w2, threshold, limit):
    """M.6.3: a block takes the smoothed samples when fewer than ``limit`` of
    its 36 inner samples (offsets 1..6 in both directions) differ from them
    by more than ``threshold``."""
    smooth = gaborish_plane(plane, w1, w2)
    out = plane.copy()
    h, w = plane.shape
    for by in range(h // 8):
        for bx in range(w // 8):
            p = plane[8 * by:8 * by + 8, 8 * bx:8 * bx + 8]
            s = smooth[8 * by:8 * by + 8, 8 * bx:8 * bx + 8]
            count = int(np.sum(np.abs(p[1:7, 1:7] - s[1:7, 1:7]) > threshold))
            if count < limit:
                out[8 * by:8 * by + 8, 8 * bx:8 * bx + 8] = s
    return out


def upsample2(x, axis):
    """M.6.4 along one axis: sample 2i is 3/4 x[i] + 1/4 x[i-1], sample 2i+1
    is 3/4 x[i] + 1/4 x[i+1], where x[-1] = x[1] and x[n] = x[n-2]."""
    x = np.moveaxis(np.asarray(x, dtype=np.float64), axis, 0)
    n = x.shape[0]

    def at(i):
        if i < 0:
            i = -i
        if i >= n:
            i = 2 * n - 2 - i
        return x[min(max(i, 0), n - 1)]

    out = np.zeros((2 * n,) + x.shape[1:])
    for i in range(n):
        out[2 * i] = 0.75 * x[i] + 0.25 * at(i - 1)
        out[2 * i + 1] = 0.75 * x[i] + 0.25 * at(i + 1)
    return np.moveaxis(out, 0, axis)


def ycbcr_to_rgb(y, cb, cr):
    """M.6.5 on level-shifted samples."""
    r = 1.402 * cr + (y + 128.0)
    g = -0.71414 * cr - 0.34414 * cb + (y + 128.0)
    b = 1.772 * cb + (y + 128.0)
    return r, g, b


def rasterize(stream):
    """The whole of M.6: (ysize, xsize,
    3) RGB samples on the nominal 0..255 scale, unclamped.  ``stream``:
    xsize, ysize and a list of components, each a dict with coeffs
    (bh, bw, 64), quant (64,), h_samp, v_samp, an optional 'gab' tuple
    (w1, w2, threshold, limit) and an optional 'cond' tuple (max_gap,
    min_step)."""
    comps = stream['components']
    hmax = max(c['h_samp'] for c in comps)
    vmax = max(c['v_samp'] for c in comps)
    planes = []
    for c in comps:
        p = component_pixels(c['coeffs'], c['quant'], c.get('cond'))
        if c.get('gab') is not None:
            p = conditional_gaborish(p, *c['gab'])
        if c['h_samp'] != hmax:
            p = upsample2(p, 1)
        if c['v_samp'] != vmax:
            p = upsample2(p, 0)
        planes.append(p)
    ys, xs = stream['ysize'], stream['xsize']
    planes = [p[:ys, :xs] for p in planes]
    if len(planes) == 1:
        g = planes[0] + 128.0
        return np.stack([g, g, g], axis=-1)
    r, g, b = ycbcr_to_rgb(*planes)
    return np.stack([r, g, b], axis=-1)


def to_u8(rgb):
    """8-bit output: clamp to [0, 255] and round half up (READING: the
    draft leaves the rounding of the rasterised samples open)."""
    return np.floor(np.clip(rgb, 0.0, 255.0) + 0.5).astype(np.uint8)
