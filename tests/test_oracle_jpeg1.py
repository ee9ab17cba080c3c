"""Pins of the JPEG1 direct-rasterisation oracle (M.6) against what the draft
and the mathematics fix."""
import math
import os

import numpy as np
import pytest

from oracle import jpeg1 as J
from paper_1908_03565_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), 'golden')


def test_upsampling_worked_example():
    """M.6.4 EXAMPLE: {0, 4, 12, 8} -> {1, 1, 3, 6, 10, 11, 9, 9}."""
    with open(os.path.join(GOLDEN, 'm6_4_upsampling_example.txt')) as f:
        rows = [list(map(float, l.split())) for l in f if l.strip() and not l.startswith('#')]
    np.testing.assert_allclose(J.upsample2(np.array(rows[0]), 0), rows[1], atol=1e-12)


def test_upsampling_2d_is_separable_and_keeps_constants():
    x = np.random.default_rng(0).normal(size=(5, 7))
    a = J.upsample2(J.upsample2(x, 1), 0)
    b = J.upsample2(J.upsample2(x, 0), 1)
    np.testing.assert_allclose(a, b, atol=1e-12)     # linear: order does not matter
    np.testing.assert_allclose(J.upsample2(np.full((3, 4), 2.5), 1), 2.5, atol=1e-15)


def _textbook_idct_basis(u, v):
    """The orthonormal 8x8 DCT-III basis function (u vertical, v horizontal)."""
    cu = math.sqrt(0.5) if u == 0 else 1.0
    cv = math.sqrt(0.5) if v == 0 else 1.0
    out = np.zeros((8, 8))
    for y in range(8):
        for x in range(8):
            out[y, x] = 0.25 * cu * cv * math.cos((2 * x + 1) * v * math.pi / 16) * \
                math.cos((2 * y + 1) * u * math.pi / 16)
    return out


@pytest.mark.parametrize('u,v', [(0, 0), (0, 1), (1, 0), (3, 5), (7, 7), (2, 6)])
def test_dequant_idct_is_the_orthonormal_basis(u, v):
    """M.6.1 + M.6.2: I(8,u) I(8,v) IDCT_2D is the orthonormal 2-D DCT-III
    (the textbook JPEG inverse transform), u the vertical frequency."""
    q = np.zeros((1, 1, 64), np.int16)
    q[0, 0, 8 * u + v] = 3
    quant = np.full(64, 5, np.uint16)
    got = J.component_pixels(q, quant)
    np.testing.assert_allclose(got, 15 * _textbook_idct_basis(u, v), atol=1e-12)


def test_dc_only_block_is_constant():
    q = np.zeros((2, 3, 64), np.int16)
    q[..., 0] = np.arange(6).reshape(2, 3) * 7
    quant = np.arange(1, 65).astype(np.uint16)
    p = J.component_pixels(q, quant)
    for by in range(2):
        for bx in range(3):
            np.testing.assert_allclose(p[8 * by:8 * by + 8, 8 * bx:8 * bx + 8],
                                       q[by, bx, 0] * quant[0] / 8.0, atol=1e-12)


def test_ycbcr_values():
    """M.6.5: zero chroma is grey Y + 128; unit chroma moves R, G, B by the
    printed factors."""
    assert J.ycbcr_to_rgb(0.0, 0.0, 0.0) == (128.0, 128.0, 128.0)
    r, g, b = J.ycbcr_to_rgb(10.0, 1.0, 2.0)
    assert r == pytest.approx(138 + 2 * 1.402)
    assert g == pytest.approx(138 - 0.71414 * 2 - 0.34414)
    assert b == pytest.approx(138 + 1.772)


def test_conditional_gaborish_limits():
    """M.6.3: limit 0 never replaces a block; limit 37 always does (36 inner
    samples); a huge threshold with limit 1 replaces every block; the
    normalised kernel keeps constants."""
    rng = np.random.default_rng(1)
    p = rng.normal(0, 20, size=(24, 16))
    w1, w2 = 118 / 1024, 63 / 1024
    np.testing.assert_array_equal(J.conditional_gaborish(p, w1, w2, 2.5, 0), p)
    np.testing.assert_allclose(J.conditional_gaborish(p, w1, w2, 2.5, 37),
                               J.gaborish_plane(p, w1, w2), atol=1e-12)
    np.testing.assert_allclose(J.conditional_gaborish(p, w1, w2, 1e9, 1),
                               J.gaborish_plane(p, w1, w2), atol=1e-12)
    np.testing.assert_allclose(J.gaborish_plane(np.full((9, 9), 3.0), w1, w2), 3.0, atol=1e-14)


def test_gaborish_plane_brute_force():
    """J.4 at one interior and one corner sample, by the definition."""
    p = np.random.default_rng(2).normal(size=(8, 8))
    w1, w2 = 0.2, 0.05
    s = J.gaborish_plane(p, w1, w2)
    y, x = 3, 4
    want = (p[y, x] + w1 * (p[y - 1, x] + p[y + 1, x] + p[y, x - 1] + p[y, x + 1]) +
            w2 * (p[y - 1, x - 1] + p[y - 1, x + 1] + p[y + 1, x - 1] + p[y + 1, x + 1])) / (1 + 4 * w1 + 4 * w2)
    assert s[y, x] == pytest.approx(want)
    # corner: index -1 mirrors to 0 (6.5)
    want0 = (p[0, 0] + w1 * (p[0, 0] + p[1, 0] + p[0, 0] + p[0, 1]) +
             w2 * (p[0, 0] + p[0, 1] + p[1, 0] + p[1, 1])) / (1 + 4 * w1 + 4 * w2)
    assert s[0, 0] == pytest.approx(want0)


def test_rasterize_shapes_and_grey():
    st = synth.make_jpeg(45, 30, 3, sampling='420')
    rgb = J.rasterize(st)
    assert rgb.shape == (30, 45, 3)
    grey = synth.make_jpeg(20, 12, 4, sampling='grey')
    g = J.rasterize(grey)
    np.testing.assert_array_equal(g[..., 0], g[..., 1])
    assert J.to_u8(np.array([-3.0, 0.5, 254.5, 300.0])).tolist() == [0, 1, 255, 255]


def test_conditioning_staircase_by_hand():
    """M.6.1.1 on one row of DC 0 0 0 1 1 1 2 2 2 with zero AC: the first run
    has |to - from| = 0.5, not above min_step 0.5; the middle run from 0.5 to
    1.5 over 3 blocks gives 0.5 + (0.5 + i) / 3 and slopes -1/6; the last run
    is symmetric to the first."""
    dc = np.array([[0, 0, 0, 1, 1, 1, 2, 2, 2]])
    ac = np.zeros_like(dc)
    a, s, h = J._plateaus(dc, ac, 5 / 3, 0.5, 0.5)
    assert h.tolist() == [[False] * 3 + [True] * 3 + [False] * 3]
    np.testing.assert_allclose(a[0, 3:6], [0.5 + 0.5 / 3, 1.0, 1.5 - 0.5 / 3], rtol=1e-6)
    np.testing.assert_allclose(s[0, 3:6], -1 / 6, rtol=1e-6)
    # a whole-row run is never a range; a nonzero AC in the run disables it
    assert not J._plateaus(np.zeros((1, 5), int), np.zeros((1, 5), int), 1.0, 0.5, 0.5)[2].any()
    ac2 = ac.copy()
    ac2[0, 4] = 1
    assert not J._plateaus(dc, ac2, 5 / 3, 0.5, 0.5)[2][0, 3:6].any()


def test_conditioning_makes_a_ramp():
    """With the replaced DC and slope the middle run's samples rise
    monotonically from about 0.5 to 1.5 DC steps (the reading of
    dc_multiplier): no step larger than a third of a DC step."""
    q = np.zeros((1, 9, 64), np.int16)
    q[0, :, 0] = [0, 0, 0, 1, 1, 1, 2, 2, 2]
    quant = np.full(64, 8, np.uint16)
    plain = J.component_pixels(q, quant)
    cond = J.component_pixels(q, quant, (0.5, 0.5))
    row = cond[3, 24:48] / (8 / 8.0)                    # in DC steps (Q0 / 8 per step)
    assert np.all(np.diff(row) >= -1e-6)
    assert np.abs(np.diff(row)).max() < 1 / 3
    assert row[0] == pytest.approx(0.5, abs=0.1) and row[-1] == pytest.approx(1.5, abs=0.1)
    np.testing.assert_allclose(cond[:, :24], plain[:, :24], atol=1e-12)   # first run untouched


def test_conditioning_stream_statistics():
    st = synth.make_jpeg(200, 136, 8, sampling='420', plateaus=True, cond=(0.5, 0.5))
    c = st['components'][0]
    approx, hs, hh, vs, vh = J.conditioning(c['coeffs'], c['quant'], 0.5, 0.5)
    assert 0.05 < hh.mean() < 0.95 and 0.05 < vh.mean() < 0.95
