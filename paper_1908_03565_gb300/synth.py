"""Seeded synthetic inputs for VarDCT reconstruction.

The draft measures on no dataset, so every workload here is synthetic. This
module only draws numbers: it holds none of the reconstruction arithmetic,
and both the CUDA library's tests/benchmark and the FP64 oracle take their
inputs from it.

Statistics (per image):

* varblock tiling, per naturally aligned 32x32 cell in raster order:
  DCT32 p=0.10; a pair of 32x16 (or 16x32) p=0.05; four 32x8 (or 8x32)
  p=0.05; otherwise four 16x16 cells.  Per 16x16 cell: DCT16 p=0.1875, a
  pair of 16x8 (or 8x16) p=0.0625, otherwise four 8x8 blocks: DCT8 2/3,
  DCT4 1/6, DCT2 1/12, Identity 1/12.  Cells that do not fit inside the
  padded image fall through to the smaller cells.  Expected area: DCT8 40%,
  DCT16 15%, DCT32 10%, rectangles 15%, DCT4 10%, DCT2 5%, Identity 5%.
* quantised coefficients: Laplace(0, 64 / (1 + u + v)) rounded to int16, where
  (u, v) is the position in the varblock's coefficient matrix (the 8x8 matrix
  for the 8x8-class shapes), the LLF slots included (zero-mean DC);
* quant field (AcMul): log-uniform in [0.5, 4] per varblock, replicated to
  all its 8x8 blocks;
* chroma-from-luma factors kX, kB: uniform in [-0.5, 0.5] per 64x64 tile;
* sharpness: uniform in {0..7} per 8x8 block.

DctSelect codes (C.5.4 of the draft): 0 DCT8, 1 Identity, 2 DCT2, 3 DCT4,
4 DCT16, 5 DCT32, 6 16x8 (16 tall), 7 8x16, 8 32x8 (32 tall), 9 8x32,
10 32x16 (32 tall), 11 16x32, 12 4x8, 13 8x4, 14 AFV; 0xFF marks a block
covered by a varblock that starts elsewhere.
"""
import math

import numpy as np

COVERED = 0xFF
# (width, height) of each DctSelect code
SHAPE_WH = {0: (8, 8), 1: (8, 8), 2: (8, 8), 3: (8, 8), 4: (16, 16),
            5: (32, 32), 6: (8, 16), 7: (16, 8), 8: (8, 32), 9: (32, 8),
            10: (16, 32), 11: (32, 16), 12: (8, 8), 13: (8, 8), 14: (8, 8)}


def _place(vmap, code, bx, by):
    w, h = SHAPE_WH[code]
    vmap[by:by + h // 8, bx:bx + w // 8] = COVERED
    vmap[by, bx] = code


def tiling(bw, bh, rng, mix='mixed'):
    """DctSelect map of bh x bw blocks.  mix: 'mixed' (statistics above),
    'dct8' (all DCT8), or a single code (every block that code where it fits,
    DCT8 elsewhere)."""
    vmap = np.full((bh, bw), COVERED, dtype=np.uint8)
    if mix == 'dct8':
        vmap[:] = 0
        return vmap
    if isinstance(mix, int):
        w, h = SHAPE_WH[mix]
        cw, ch = w // 8, h // 8
        for by in range(0, bh, ch):
            for bx in range(0, bw, cw):
                if by + ch <= bh and bx + cw <= bw:
                    _place(vmap, mix, bx, by)
                else:
                    for yy in range(by, min(by + ch, bh)):
                        for xx in range(bx, min(bx + cw, bw)):
                            vmap[yy, xx] = 0
        return vmap

    def small(bx, by):
        r = rng.random()
        code = 0 if r < 2 / 3 else 3 if r < 2 / 3 + 1 / 6 else 2 if r < 11 / 12 else 1
        vmap[by, bx] = code

    def cell16(bx, by):
        if bx + 2 <= bw and by + 2 <= bh:
            r = rng.random()
            if r < 0.1875:
                _place(vmap, 4, bx, by)
                return
            if r < 0.25:
                if rng.random() < 0.5:   # two 16-tall, 8-wide
                    _place(vmap, 6, bx, by)
                    _place(vmap, 6, bx + 1, by)
                else:                    # two 8-tall, 16-wide
                    _place(vmap, 7, bx, by)
                    _place(vmap, 7, bx, by + 1)
                return
        for yy in range(by, min(by + 2, bh)):
            for xx in range(bx, min(bx + 2, bw)):
                small(xx, yy)

    for cy in range(0, bh, 4):
        for cx in range(0, bw, 4):
            if cx + 4 <= bw and cy + 4 <= bh:
                r = rng.random()
                if r < 0.10:
                    _place(vmap, 5, cx, cy)
                    continue
                if r < 0.15:
                    if rng.random() < 0.5:   # 32 tall, 16 wide
                        _place(vmap, 10, cx, cy)
                        _place(vmap, 10, cx + 2, cy)
                    else:
                        _place(vmap, 11, cx, cy)
                        _place(vmap, 11, cx, cy + 2)
                    continue
                if r < 0.20:
                    if rng.random() < 0.5:   # 32 tall, 8 wide
                        for k in range(4):
                            _place(vmap, 8, cx + k, cy)
                    else:
                        for k in range(4):
                            _place(vmap, 9, cx, cy + k)
                    continue
            for yy in range(cy, min(cy + 4, bh), 2):
                for xx in range(cx, min(cx + 4, bw), 2):
                    cell16(xx, yy)
    return vmap


def coefficient_positions(vmap):
    """Per-sample (u, v) position inside the varblock's coefficient matrix,
    with the 8x8 matrix of 8x8-class shapes; and the top-left block of each
    block's varblock."""
    bh, bw = vmap.shape
    ox = np.zeros((bh, bw), dtype=np.int64)
    oy = np.zeros((bh, bw), dtype=np.int64)
    for code, (w, h) in SHAPE_WH.items():
        ty, tx = np.nonzero(vmap == code)
        for dy in range(h // 8):
            for dx in range(w // 8):
                ox[ty + dy, tx + dx] = tx
                oy[ty + dy, tx + dx] = ty
    Hp, Wp = 8 * bh, 8 * bw
    x0 = np.repeat(np.repeat(ox, 8, 0), 8, 1) * 8
    y0 = np.repeat(np.repeat(oy, 8, 0), 8, 1) * 8
    u = np.arange(Wp)[None, :] - x0
    v = np.arange(Hp)[:, None] - y0
    return u, v, ox, oy


def llf_slots(vmap, u, v, ox, oy):
    """Boolean (Hp, Wp) mask of the LLF slots (u < W/8 and v < H/8 of the
    sample's varblock), which hold the quantised DC samples."""
    bh, bw = vmap.shape
    wv = np.zeros((bh, bw), dtype=np.int64)
    hv = np.zeros((bh, bw), dtype=np.int64)
    for code, (w, h) in SHAPE_WH.items():
        sel = vmap[oy, ox] == code
        wv[sel], hv[sel] = w, h
    wv = np.repeat(np.repeat(wv, 8, 0), 8, 1)
    hv = np.repeat(np.repeat(hv, 8, 0), 8, 1)
    return (u < wv // 8) & (v < hv // 8)


def make_image(xsize, ysize, seed, mix='mixed', acmul=None, cfl=True,
               coef_scale=64.0, y_dc_offset_q=0, dc='noise', ac=True):
    """One synthetic image.  Returns a dict with xsize, ysize, coeffs
    (int16, 3 x Hp x Wp), vmap (uint8, Hp/8 x Wp/8), acmul (float32, per
    block), cfl (float32, ceil(Hp/64) x ceil(Wp/64) x 2), sharpness (uint8).
    ``acmul`` None draws the log-uniform quant field, a number fixes it;
    ``cfl`` False sets kX = kB = 0; ``y_dc_offset_q`` adds a constant to the
    quantised DC of the Y channel.  ``dc='smooth'`` replaces the quantised
    DC samples by a slowly varying field (amplitude 40 steps, period 48
    blocks) plus Gaussian noise of 0.7 steps, so that the DC and DC2x2
    smoothing steps keep some samples and change others; ``ac=False``
    zeroes every coefficient outside the LLF slots."""
    rng = np.random.default_rng(seed)
    Wp, Hp = 8 * ((xsize + 7) // 8), 8 * ((ysize + 7) // 8)
    bw, bh = Wp // 8, Hp // 8
    vmap = tiling(bw, bh, rng, mix)
    u, v, ox, oy = coefficient_positions(vmap)
    scale = coef_scale / (1.0 + u + v)
    lap = rng.laplace(0.0, 1.0, size=(3, Hp, Wp)) * scale[None]
    coeffs = np.clip(np.rint(lap), -32768, 32767).astype(np.int16)
    llf = None
    if dc == 'smooth' or not ac:
        llf = llf_slots(vmap, u, v, ox, oy)
    if dc == 'smooth':
        # block index of the DC sample in each LLF slot
        bxs = np.repeat(np.repeat(ox, 8, 0), 8, 1) + u
        bys = np.repeat(np.repeat(oy, 8, 0), 8, 1) + v
        phase = rng.uniform(0, 2 * math.pi, size=(3, 2))
        for c in range(3):
            f = 40.0 * np.sin(2 * math.pi * bxs / 48.0 + phase[c, 0]) * \
                np.cos(2 * math.pi * bys / 48.0 + phase[c, 1])
            f = np.rint(f + rng.normal(0.0, 0.7, size=f.shape)).astype(np.int16)
            coeffs[c] = np.where(llf, f, coeffs[c])
    if not ac:
        coeffs = np.where(llf[None], coeffs, 0).astype(np.int16)
    if y_dc_offset_q:
        if llf is None:
            llf = llf_slots(vmap, u, v, ox, oy)
        y = coeffs[1].astype(np.int64)
        coeffs[1] = np.where(llf, np.clip(y + y_dc_offset_q, -32768, 32767), y)
    if acmul is None:
        per_vb = np.exp(rng.uniform(math.log(0.5), math.log(4.0), size=(bh, bw)))
        am = per_vb[oy, ox].astype(np.float32)
    else:
        am = np.full((bh, bw), acmul, dtype=np.float32)
    th, tw = (Hp + 63) // 64, (Wp + 63) // 64
    if cfl:
        cf = rng.uniform(-0.5, 0.5, size=(th, tw, 2)).astype(np.float32)
    else:
        cf = np.zeros((th, tw, 2), dtype=np.float32)
    sharp = rng.integers(0, 8, size=(bh, bw)).astype(np.uint8)
    return {'xsize': xsize, 'ysize': ysize, 'coeffs': coeffs, 'vmap': vmap,
            'acmul': am, 'cfl': cf, 'sharpness': sharp}


def shape_area_fractions(vmap):
    """Fraction of the padded area covered by each DctSelect code."""
    tot = {}
    for by, bx in np.argwhere(vmap != COVERED):
        c = int(vmap[by, bx])
        w, h = SHAPE_WH[c]
        tot[c] = tot.get(c, 0) + w * h
    area = 64 * vmap.size
    return {c: a / area for c, a in sorted(tot.items())}


def make_jpeg(xsize, ysize, seed, sampling='420', gab=False, ac_scale=6.0, plateaus=False,
              cond=None):
    """A synthetic JPEG1 coefficient stream (the input of direct
    rasterisation).  ``sampling``: '420' (Y 2x2, Cb and Cr 1x1), '444' or
    'grey'.  Quantisation tables: 3 + 2 (u + v) for Y and 4 + 3 (u + v) for
    chroma (synthetic, index 8u + v).  Quantised DC: a slow field of
    amplitude 200 steps (period 40 blocks) plus Gaussian noise of 2 steps;
    AC: Laplace(0, ac_scale / (1 + u + v)) rounded.  ``gab`` adds the block-
    conditional Gaborish side channel (w1 118/1024, w2 63/1024, threshold
    2.5, limit 20) to every component.  ``plateaus`` makes the quantised DC
    a coarse staircase (the field / 20, rounded: long runs of equal values)
    and zeroes coefficients 1 and 8 in 80% of the blocks, the inputs the DC
    / AC conditioning of M.6.1.1 acts on; ``cond`` = (max_gap, min_step)
    requests that conditioning.  Returns a dict with xsize, ysize and
    components (coeffs int16 (bh, bw, 64), quant uint16 (64,), h_samp,
    v_samp, gab, cond)."""
    rng = np.random.default_rng(seed)
    if sampling == '420':
        samp = [(2, 2), (1, 1), (1, 1)]
    elif sampling == '444':
        samp = [(1, 1), (1, 1), (1, 1)]
    elif sampling == 'grey':
        samp = [(1, 1)]
    else:
        raise ValueError(sampling)
    hmax = max(s[0] for s in samp)
    vmax = max(s[1] for s in samp)
    mx = -(-xsize // (8 * hmax))
    my = -(-ysize // (8 * vmax))
    uu, vv = np.divmod(np.arange(64), 8)
    comps = []
    for ci, (h, v) in enumerate(samp):
        bw, bh = mx * h, my * v
        base = 3 if ci == 0 else 4
        step = 2 if ci == 0 else 3
        quant = (base + step * (uu + vv)).astype(np.uint16)
        ac = rng.laplace(0.0, 1.0, size=(bh, bw, 64)) * (ac_scale / (1.0 + uu + vv))
        q = np.rint(ac)
        by, bx = np.mgrid[0:bh, 0:bw]
        ph = rng.uniform(0, 2 * math.pi, size=2)
        dc = 200.0 * np.sin(2 * math.pi * bx / 40.0 + ph[0]) * np.cos(2 * math.pi * by / 40.0 + ph[1])
        if plateaus:
            q[:, :, 0] = np.rint(dc / 20.0)
            zero = rng.random(size=(bh, bw)) < 0.8
            q[:, :, 1] = np.where(zero, 0, q[:, :, 1])
            q[:, :, 8] = np.where(zero, 0, q[:, :, 8])
        else:
            q[:, :, 0] = np.rint(dc + rng.normal(0.0, 2.0, size=(bh, bw)))
        comps.append({'coeffs': np.clip(q, -32768, 32767).astype(np.int16), 'quant': quant,
                      'h_samp': h, 'v_samp': v,
                      'gab': (118 / 1024, 63 / 1024, 40 / 16, 20) if gab else None,
                      'cond': cond})
    return {'xsize': xsize, 'ysize': ysize, 'components': comps}
