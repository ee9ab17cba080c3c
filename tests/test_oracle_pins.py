"""Pins of the FP64 oracle against what the draft and mathematics fix.

Each test names the passage it relies on. None of them re-derives a value
with the oracle's own formula: they use closed forms, round trips through
the draft's forward procedures (I.2.3), invariants the draft states
(orthonormal AFV basis, weights summing to one, constants preserved), the
draft's independent I.2.6 downsampling formula, and brute force.
"""
import math
import os

import numpy as np
import pytest

from oracle import recon as R
from oracle import tables as T
from oracle import transforms as TR
from paper_1908_03565_gb300 import synth

RNG = np.random.default_rng(1234)
DCT_SHAPES = [T.SHAPE_WH[c] for c in T.DCT_SHAPES]


# --------------------------------------------------------------------------
# I.2.1 / I.2.2 / Annex R: the inverse DCTs
# --------------------------------------------------------------------------
@pytest.mark.parametrize("W,H", DCT_SHAPES)
def test_separable_idct_equals_cosine_sum_bruteforce(W, H):
    """I.2.2 separable form == the O(N^4) cosine-sum definition (catches
    transposed operands and swapped axes)."""
    c = RNG.standard_normal((H, W))
    np.testing.assert_allclose(TR.idct_2d(c), TR.idct_2d_bruteforce(c),
                               rtol=0, atol=1e-11)


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32])
def test_numerator_scaled_idct_is_orthonormal(N):
    """I.2.6.1 defines I(N,u) as the DCT scaling factor used by the C.6.1
    numerators; with it every 1-D inverse DCT becomes the orthonormal
    DCT-III basis.  A wrong per-frequency scale S_N (I.2.1, Annex R) breaks
    this for that frequency."""
    B = TR.idct_matrix(N) * np.array([T.I(N, u) for u in range(N)])[None, :]
    np.testing.assert_allclose(B.T @ B, np.eye(N), atol=1e-13)
    # and the basis is the textbook one
    ref = np.array([[math.sqrt((1 if u == 0 else 2) / N)
                     * math.cos((2 * n + 1) * u * math.pi / (2 * N))
                     for u in range(N)] for n in range(N)])
    np.testing.assert_allclose(B, ref, atol=1e-13)


@pytest.mark.parametrize("W,H", [(16, 16), (32, 32), (8, 16), (16, 8),
                                 (8, 32), (32, 8), (16, 32), (32, 16)])
def test_box_mean_matches_draft_downsampling(W, H):
    """I.2.6.2 (ScaleF, then a small IDCT) yields the 8x downsampled image;
    it must equal the exact mean of each 8x8 sub-block of the LLF-only
    reconstruction.  Pins S_N of the large and the small transforms."""
    cx, cy = W // 8, H // 8
    llf = RNG.standard_normal((cy, cx))
    coef = np.zeros((H, W))
    coef[:cy, :cx] = llf
    pix = TR.idct_2d(coef)
    means = pix.reshape(cy, 8, cx, 8).mean(axis=(1, 3))
    np.testing.assert_allclose(TR.downsample_scalef(coef), means, atol=1e-12)
    # and llf_from_dc inverts it
    np.testing.assert_allclose(TR.llf_from_dc(means), llf, atol=1e-11)


@pytest.mark.parametrize("W,H", [(16, 16), (32, 32), (8, 16), (32, 16)])
def test_printed_llf_formula_is_blockcount_times_inverse(W, H):
    """I.2.7.2 as printed (DCT of the DC block, times ScaleF) differs from
    the exact inverse of I.2.6.2 by the number of 8x8 sub-blocks; the oracle
    uses the exact inverse (I.2.7.1 calls the step the inverse of I.2.6)."""
    cx, cy = W // 8, H // 8
    dc = RNG.standard_normal((cy, cx))
    Cm = TR.dct_2d(dc)
    printed = np.array([[Cm[y, x] * T.ScaleF(cy, H, y) * T.ScaleF(cx, W, x)
                         for x in range(cx)] for y in range(cy)])
    np.testing.assert_allclose(printed, cx * cy * TR.llf_from_dc(dc), atol=1e-11)


# --------------------------------------------------------------------------
# I.2.3 / I.2.4: the 8x8-class procedures, through their forward partners
# --------------------------------------------------------------------------
@pytest.mark.parametrize("S", [2, 4, 8])
def test_aux_2x2_round_trip(S):
    b = RNG.standard_normal((8, 8))
    np.testing.assert_allclose(TR.aux_idct2x2(TR.aux_dct2x2(b, S), S), b, atol=1e-14)


@pytest.mark.parametrize("fwd,inv", [
    (TR.dct_dct2, TR.idct_dct2), (TR.dct_dct4, TR.idct_dct4),
    (TR.dct_identity, TR.idct_identity), (TR.dct_dct8x4, TR.idct_dct8x4),
    (TR.dct_dct4x8, TR.idct_dct4x8), (TR.dct_afv, TR.idct_afv)])
def test_8x8_class_round_trip(fwd, inv):
    """I.2.3.x forward procedure then I.2.4.x inverse returns the samples.
    For 4x8 this pins the dcs[y] reading of I.2.4.6."""
    s = RNG.standard_normal((8, 8))
    np.testing.assert_allclose(inv(fwd(s)), s, atol=1e-12)


def test_identity_round_trip_exact_on_integers():
    s = RNG.integers(-100, 100, (8, 8)).astype(np.float64) * 16
    np.testing.assert_array_equal(TR.idct_identity(TR.dct_identity(s)), s)


def test_afv_basis_orthonormal():
    """I.2.2 calls the AFV basis orthonormal; this pins the repair of the
    two rows printed with 17 entries."""
    B = T.AFV_BASIS
    assert B.shape == (16, 16)
    np.testing.assert_allclose(B @ B.T, np.eye(16), atol=1e-13)


@pytest.mark.parametrize("code", sorted(T.SHAPE_WH))
def test_dc_only_varblock(code):
    """A varblock with only DC samples (I.2.6/I.2.7 are each other's
    inverse): every 8x8 sub-block of the result averages to its DC sample,
    and equal DC samples give a constant varblock."""
    W, H = T.SHAPE_WH[code]
    vmap = np.full((H // 8, W // 8), T.COVERED, np.uint8)
    vmap[0, 0] = code
    p = R.Params(m_dc=(0.01, 0.002, 0.003))
    ones = np.ones((H // 8, W // 8), np.float32)
    nocfl = np.zeros((1, 1, 2), np.float32)
    coeffs = np.zeros((3, H, W), np.int16)
    q = RNG.integers(-300, 300, (3, H // 8, W // 8))
    coeffs[:, :H // 8, :W // 8] = q
    xyb = R.reconstruct_xyb(coeffs, vmap, ones, nocfl, p)
    for c in range(3):
        means = xyb[c].reshape(H // 8, 8, W // 8, 8).mean(axis=(1, 3))
        np.testing.assert_allclose(means, p.m_dc[c] * q[c], atol=1e-13)
    coeffs[:, :H // 8, :W // 8] = q[:, :1, :1]
    xyb = R.reconstruct_xyb(coeffs, vmap, ones, nocfl, p)
    for c in range(3):
        np.testing.assert_allclose(xyb[c], p.m_dc[c] * q[c, 0, 0], atol=1e-13)


def test_batched_inverse_equals_step_by_step():
    """The per-shape batched evaluation equals the one-varblock-at-a-time
    procedures of I.2.4 on a mixed tiling."""
    im = synth.make_image(96, 64, 7)
    # make every 8x8-class code appear
    codes = [12, 13, 14, 1, 2, 3]
    for i, c in enumerate(codes):
        im['vmap'][7, i] = c
    dq = R.dequantize(im['coeffs'], im['vmap'], im['acmul'], im['cfl'], R.Params())
    np.testing.assert_allclose(R.inverse_transform(dq, im['vmap']),
                               R.inverse_transform_literal(dq, im['vmap']),
                               atol=1e-12)


# --------------------------------------------------------------------------
# C.6.1: dequantisation matrices
# --------------------------------------------------------------------------
@pytest.mark.parametrize("code", sorted(T.SHAPE_WH))
def test_default_matrices_positive_finite(code):
    """C.6.1: a non-positive or infinite entry makes the codestream
    ill-formed, so every default matrix must be positive and finite."""
    W, H = T.SHAPE_WH[code]
    for c in range(3):
        m = T.dequant_matrix(code, c)
        assert m.shape == (H, W)
        ac = np.ones((H, W), bool)
        ac[:H // 8, :W // 8] = False      # LLF slots take no matrix entry
        assert np.all(np.isfinite(m[ac])) and np.all(m[ac] > 0)


@pytest.mark.parametrize("a,b", [(6, 7), (8, 9), (10, 11), (12, 13)])
def test_transposed_shapes_have_transposed_matrices(a, b):
    """Both orientations share one default encoding (C.6.1.1), and the
    weights depend only on (x/X, y/Y); so the matrices are transposes."""
    for c in range(3):
        np.testing.assert_allclose(T.dequant_matrix(a, c), T.dequant_matrix(b, c).T,
                                   rtol=1e-14)


def test_dct8_weight_closed_forms():
    """DCT8 channel X: with eccentricity bands all 0 the eccentricity factor
    is 1, and the first two distance bands are 5 and 5 * 1/(1-0) = 5, so the
    weight is 5 wherever the distance lies in the first band interval
    (distance < sqrt(2)/5)."""
    num = T.I(8, 1) * T.I(8, 0) / 64.0
    assert T.dequant_matrix(0, 0)[0, 1] == pytest.approx(num / 5.0, rel=1e-14)
    assert T.dequant_matrix(0, 0)[1, 1] == pytest.approx(T.I(8, 1) ** 2 / 64.0 / 5.0,
                                                         rel=1e-14)


def _c61_golden():
    """Entries of tests/golden/c61_weights.txt: (code, channel, x, y, value),
    each value a hand-specialised expression of C.6.1.1's printed numbers."""
    path = os.path.join(os.path.dirname(__file__), "golden", "c61_weights.txt")
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            code, c, x, y, expr = line.split(None, 4)
            val = eval(expr, {"__builtins__": {}}, {"sqrt": math.sqrt})
            rows.append((int(code), int(c), int(x), int(y), float(val), expr))
    return rows


def test_c61_weights_hand_derived_entries():
    """C.6.1 weight synthesis against entries derived by hand from the
    printed band arrays (distance on a band or at a known fraction between
    two, eccentricity 0 on the diagonal, 1 on the axes, or in between for
    the 32x8 shapes), covering every DCT-mode shape, the DCT4 and 4x8
    up-sampling with their multipliers, and the AFV cells."""
    rows = _c61_golden()
    codes = {r[0] for r in rows}
    assert codes == {0, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14}
    for code, c, x, y, want, expr in rows:
        got = T._weights(code, c)[y, x]
        assert got == pytest.approx(want, rel=1e-12), (code, c, x, y, expr)


def test_c61_golden_catches_band_slips():
    """The hand-derived entries fail for plausible misreadings: bands shifted
    by one index, the eccentricity bands dropped, DCT32x8 and DCT8x32
    exchanged, the 4x8 up-sampling on the wrong axis, and the AFV frequency
    table read transposed."""
    rows = _c61_golden()

    def fails(weights_fn):
        return any(abs(weights_fn(code, c)[y, x] - want) > 1e-9 * abs(want)
                   for code, c, x, y, want, _ in rows
                   if weights_fn(code, c).shape[0] > y and weights_fn(code, c).shape[1] > x)

    orig_db, orig_ecc = T.distance_bands, T.eccentricity_bands
    orig_freqs = T._AFV_FREQS
    try:
        T.distance_bands = lambda db: [db[0]] + [T._band_factor(db[i + 1 if i + 1 < len(db) else i])
                                                 * db[0] for i in range(1, len(db))]
        assert fails(T._weights)
        T.distance_bands = orig_db
        T.eccentricity_bands = lambda eb: [1.0] * (len(eb) + 1)
        assert fails(T._weights)
        T.eccentricity_bands = orig_ecc
        T._AFV_FREQS = tuple(orig_freqs[4 * (i % 4) + i // 4] for i in range(16))
        assert fails(T._weights)
        T._AFV_FREQS = orig_freqs
    finally:
        T.distance_bands, T.eccentricity_bands, T._AFV_FREQS = orig_db, orig_ecc, orig_freqs

    def swapped(code, c):
        # the orientation misread: DCT32x8 given DCT8x32's matrix and back
        return T._weights(17 - code if code in (8, 9) else code, c)
    assert fails(swapped)

    def up_wrong_axis(code, c):
        if code in (12, 13):
            w48 = T.dct_weights(4, 8, T._DB_DCT4X8[c], (0.0, 0.0))
            w = np.array([[w48[y, x // 2] for x in range(8)] for y in range(8)])
            return w if code == 12 else w.T
        return T._weights(code, c)
    assert fails(up_wrong_axis)


def test_dct2_identity_matrices_are_reciprocal_parameters():
    """Modes DCT2 and Identity have numerators 1, so the matrix holds
    1/parameter at the positions C.6.1 lists."""
    m = T.dequant_matrix(2, 1)
    assert m[0, 1] == 1 / 960.0 and m[1, 1] == 1 / 640.0
    assert m[0, 3] == 1 / 320.0 and m[3, 0] == 1 / 320.0 and m[3, 3] == 1 / 180.0
    assert m[1, 6] == 1 / 140.0 and m[7, 7] == 1 / 120.0
    m = T.dequant_matrix(1, 2)
    assert m[0, 1] == 1 / 23.982311358829531 and m[1, 1] == 1 / 11.201853748207084
    assert m[5, 5] == 1 / 9.2887405354132238


# --------------------------------------------------------------------------
# F.3 / G: dequantisation and chroma from luma
# --------------------------------------------------------------------------
def test_ac_bias_and_cfl():
    """F.3 bias (|q|<=1 scaled, else q - 0.145/q), AcMul and matrix factors,
    and G's X += kX Y, B += kB Y on AC coefficients."""
    vmap = np.zeros((1, 1), np.uint8)
    coeffs = np.zeros((3, 8, 8), np.int16)
    coeffs[:, 0, 1] = (1, -7, 3)
    coeffs[:, 2, 0] = (0, 1, -1)
    acm = np.full((1, 1), 2.5, np.float32)
    cfl = np.array([[[0.25, -0.375]]], np.float32)
    dq = R.dequantize(coeffs, vmap, acm, cfl, R.Params())
    m = [T.dequant_matrix(0, c) for c in range(3)]
    y01 = (-7 - 0.145 / -7) * 2.5 * m[1][0, 1]
    assert dq[1, 0, 1] == pytest.approx(y01, rel=1e-14)
    assert dq[0, 0, 1] == pytest.approx((1 - T.K_ONE_BIAS[0]) * 2.5 * m[0][0, 1]
                                        + 0.25 * y01, rel=1e-14)
    assert dq[2, 0, 1] == pytest.approx((3 - 0.145 / 3) * 2.5 * m[2][0, 1]
                                        - 0.375 * y01, rel=1e-14)
    y20 = (1 - T.K_ONE_BIAS[1]) * 2.5 * m[1][2, 0]
    assert dq[0, 2, 0] == pytest.approx(0.25 * y20, rel=1e-14)
    assert dq[2, 2, 0] == pytest.approx(-(1 - T.K_ONE_BIAS[2]) * 2.5 * m[2][2, 0]
                                        - 0.375 * y20, rel=1e-14)


def test_cfl_zero_is_identity_and_dc_cfl():
    im = synth.make_image(64, 64, 3, cfl=False)
    p0 = R.Params()
    a = R.dequantize(im['coeffs'], im['vmap'], im['acmul'], im['cfl'], p0)
    p1 = R.Params(kx_dc=0.5, kb_dc=-0.25)
    b = R.dequantize(im['coeffs'], im['vmap'], im['acmul'], im['cfl'], p1)
    np.testing.assert_array_equal(a[1], b[1])
    # DC CfL enters through the (linear) LLF map: X_b - X_a == 0.5 * Y
    xa = R.inverse_transform(a, im['vmap'])
    xb = R.inverse_transform(b, im['vmap'])
    # only the LLF part differs, and it differs by kX_dc * (LLF-only Y)
    ll = np.zeros_like(a)
    for c_, bx, by in R.varblocks(im['vmap']):
        W, H = T.SHAPE_WH[c_]
        ll[1, 8 * by:8 * by + H // 8, 8 * bx:8 * bx + W // 8] = \
            a[1, 8 * by:8 * by + H // 8, 8 * bx:8 * bx + W // 8]
    yl = R.inverse_transform(ll, im['vmap'])[1]
    np.testing.assert_allclose(xb[0] - xa[0], 0.5 * yl, atol=1e-12)
    np.testing.assert_allclose(xb[2] - xa[2], -0.25 * yl, atol=1e-12)


# --------------------------------------------------------------------------
# J.2: edge-preserving filter
# --------------------------------------------------------------------------
def test_mul_table_closed_form():
    """Weight(s, mul) > 0.5 iff floor(64 s mul / 65536) >= -127, i.e.
    mul >= ceil(-127 * 1024 / s); with the search of J.2.4 starting at
    -32768 and sad = sigma >> 2, mul_table[sigma] is that bound on the
    grid, interpolated linearly in between (kSigmaShift = 2)."""
    t4 = R.mul_table4()
    for sigma in range(16, 673, 4):
        s = sigma >> 2
        bound = max(-32768, -((127 * 1024) // s))   # ceil of a negative
        assert t4[sigma] == 4 * bound, sigma
    assert t4[16] == 4 * -32512
    for sigma in range(16, 672, 4):
        for i in range(1, 4):
            assert 4 * t4[sigma + i] == 4 * t4[sigma] + i * (t4[sigma + 4] - t4[sigma])
    assert np.all(np.diff(t4[16:]) >= 0)


def test_weight_properties():
    """Weight(0, mul) is exactly 1 (sad 27 of J.2.3 is the reference); the
    weight never increases with sad; it halves when sad * mul / 1024 drops
    by 128 (one binary32 exponent step)."""
    for m4 in (-131072, -80000, -4, 0):
        assert R.weight(0, m4) == 1.0
    sad = np.arange(0, 600)
    for m4 in (-131072, -50000, -1000):
        w = R.weight(sad, m4)
        assert np.all(np.diff(w) <= 0)
    # sad 4, mul -32768: high16 = -128 + 16256 -> exactly 0.5
    assert R.weight(4, -4 * 32768) == 0.5
    assert R.weight(8, -4 * 32768) == 0.25


def test_mirror_rule():
    """6.5 mirroring: -1 -> 0, size -> size-1, repeated for far coordinates."""
    assert list(R.mirror(np.array([-1, -2, 5, 6, 7, 12]), 5)) == [0, 1, 4, 3, 2, 2]
    assert list(R.mirror(np.array([-3, 3, 4]), 2)) == [1, 0, 0]


def _constant_inputs(xs, ys, val=(0.01, 0.4, 0.3)):
    img = np.stack([np.full((ys, xs), v) for v in val])
    vmap = synth.tiling((xs + 7) // 8, (ys + 7) // 8, np.random.default_rng(0))
    acm = np.ones(vmap.shape, np.float32)
    sharp = np.full(vmap.shape, 7, np.uint8)
    return img, vmap, acm, sharp


def test_epf_preserves_constant_and_gaborish_sums_to_one():
    img, vmap, acm, sharp = _constant_inputs(40, 24)
    p = R.Params(epf=True, gab=True)
    np.testing.assert_allclose(R.epf(img, vmap, acm, sharp, p), img, atol=1e-15)
    np.testing.assert_allclose(R.gaborish(img, p), img, atol=1e-15)
    delta = np.zeros((3, 9, 9))
    delta[:, 4, 4] = 1.0
    g = R.gaborish(delta, p)
    np.testing.assert_allclose(g.sum(axis=(1, 2)), 1.0, atol=1e-15)
    w1, w2 = T.GAB_W1[0], T.GAB_W2[0]
    n = 1 + 4 * w1 + 4 * w2
    assert g[0, 4, 4] == pytest.approx(1 / n) and g[0, 3, 4] == pytest.approx(w1 / n)
    assert g[0, 3, 3] == pytest.approx(w2 / n)


@pytest.mark.parametrize("ys,xs", [(13, 17), (1, 5), (2, 1), (1, 1)])
def test_gaborish_is_a_mirrored_3x3_correlation(ys, xs):
    """J.4: per channel, the 3x3 kernel (centre 1, edges w1, corners w2,
    scaled to sum 1) applied with the 6.5 mirroring, which at a distance of
    one sample is the edge-duplicating reflection of scipy.ndimage
    ('reflect'); distinct weights per channel."""
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(99)
    img = rng.normal(0.0, 1.0, (3, ys, xs))
    p = R.Params(gab=True)
    p.gab_w1 = [0.11, 0.09, 0.13]
    p.gab_w2 = [0.05, 0.07, 0.02]
    got = R.gaborish(img, p)
    for c in range(3):
        w1, w2 = p.gab_w1[c], p.gab_w2[c]
        k = np.array([[w2, w1, w2], [w1, 1.0, w1], [w2, w1, w2]]) / (1.0 + 4 * w1 + 4 * w2)
        np.testing.assert_allclose(got[c], ndi.correlate(img[c], k, mode="reflect"),
                                   rtol=0, atol=1e-14)


def test_epf_zero_sad_is_56_tap_mean():
    """With a guide that is constant (every scaled value clamps to 0) all
    SADs are 0, all weights 1, and J.2.5 is the plain mean of the 7x8
    window (mirrored at the borders)."""
    ys, xs = 20, 24
    rng = np.random.default_rng(5)
    img = np.stack([rng.uniform(-0.2, -0.1, (ys, xs)),      # X < -0.03: scaled < 0
                    rng.uniform(-0.5, -0.01, (ys, xs)),
                    rng.uniform(-0.5, -0.01, (ys, xs))])
    vmap = np.zeros(((ys + 7) // 8, (xs + 7) // 8), np.uint8)
    acm = np.full(vmap.shape, 0.5, np.float32)
    sharp = np.full(vmap.shape, 7, np.uint8)
    p = R.Params(epf=True)
    # ranges are from the unclamped scaled values, so sigma >= 16 here
    assert R.epf_sigma(img, vmap, acm, sharp, p).min() >= 16
    out = R.epf(img, vmap, acm, sharp, p)
    want = np.zeros_like(img)
    for y in range(ys):
        for x in range(xs):
            for cy in range(-3, 4):
                for cx in range(-3, 5):
                    want[:, y, x] += img[:, R.mirror(y + cy, ys), R.mirror(x + cx, xs)]
    np.testing.assert_allclose(out, want / 56.0, atol=1e-14)


def test_guide_closed_form():
    """J.2.2: g[c] = clamp(trunc((in[c] - min[c]) * epf_scale[c]), 0, 255)
    with min = -0.03 * intensity_multiplier3 for X and 0 for Y and B.  The
    inputs sit at scaled values away from integers, so binary32 rounding
    cannot move the result."""
    p = R.Params(epf=True)
    im3 = (p.target_nits_div50 * 50.0 / 250.0) ** (1.0 / 3.0)
    ks = np.array([-7.3, -0.4, 0.5, 1.75, 100.25, 254.4, 255.6, 1.0e4])
    want = np.array([0, 0, 0, 1, 100, 254, 255, 255])
    img = np.zeros((3, 2, len(ks)))
    for c in range(3):
        mn = (-0.03 if c == 0 else 0.0) * im3
        img[c, :, :] = mn + ks / float(p.epf_scale[c])
    g = R.guide(img, p)
    assert g.dtype.kind in "iu"
    assert (g == want[None, None, :]).all()
    # the X offset matters: X = 0 is above X's minimum, so its guide is positive
    zero = R.guide(np.zeros((3, 1, 1)), p)
    assert zero[0, 0, 0] == int(0.03 * im3 * float(p.epf_scale[0])) > 0
    assert zero[1, 0, 0] == 0 and zero[2, 0, 0] == 0


def test_epf_brute_force_per_pixel():
    """J.2.3 - J.2.5 pixel by pixel on a 16x16 image of EPF-active
    statistics: for every reference pixel, 56 offsets (cx -3..4, cy -3..3),
    each distance the sum over the 3 channels of the 3x4 patch (iy -1..1,
    ix -1..2) of guide differences, samples and guide mirrored at the image
    edge (6.5); weights by Weight() with the J.2.4 cut-off; the weighted mean
    of J.2.5.  Pixels of blocks with sigma < 16 pass through.  Only the
    guide, sigma and Weight() (each pinned in this file) are shared with the
    oracle."""
    img = synth.make_image(16, 16, 4242, coef_scale=2.0, acmul=0.5, dc='smooth')
    p = R.Params(epf=True)
    xyb = R.reconstruct_xyb(img['coeffs'], img['vmap'], img['acmul'], img['cfl'], p)[:, :16, :16]
    ys, xs = 16, 16
    g = R.guide(xyb, p)
    sig = R.epf_sigma(xyb, img['vmap'], img['acmul'], img['sharpness'], p)
    mt4 = R.mul_table4()
    want = np.array(xyb, dtype=np.float64)
    live = 0
    for y in range(ys):
        for x in range(xs):
            sg = int(sig[y // 8, x // 8])
            if sg < 16:
                continue
            num = np.zeros(3)
            den = 0.0
            for cy in range(-3, 4):
                for cx in range(-3, 5):
                    sad = 0
                    for c in range(3):
                        for iy in (-1, 0, 1):
                            for ix in (-1, 0, 1, 2):
                                a = g[c, R.mirror(y + iy, ys), R.mirror(x + ix, xs)]
                                b = g[c, R.mirror(y + cy + iy, ys), R.mirror(x + cx + ix, xs)]
                                sad += abs(int(a) - int(b))
                    w = float(R.weight(sad, mt4[sg]))
                    if w < p.epf_weight_min:
                        w = 0.0
                    if w > 0 and (cx, cy) != (0, 0):
                        live += 1
                    num += w * xyb[:, R.mirror(y + cy, ys), R.mirror(x + cx, xs)]
                    den += w
            want[:, y, x] = num / den
    assert live > 1000        # many offsets besides the reference's own keep a weight
    np.testing.assert_allclose(R.epf(xyb.astype(np.float64), img['vmap'], img['acmul'],
                                     img['sharpness'], p), want, rtol=0, atol=1e-12)


def test_epf_sigma_rule():
    """J.2.4: sigma = trunc(min(min(range,70)*12.6*lut, 20/AcMul, 170)),
    range = max over the varblock of the per-block channel-max range."""
    ys, xs = 16, 16
    img = np.zeros((3, ys, xs))
    img[1, 3, 3] = 0.05       # Y block (0,0): scaled range 0.05*111.965157
    vmap = np.full((2, 2), T.COVERED, np.uint8)
    vmap[0, 0] = T.DCT16
    acm = np.full((2, 2), 1.0, np.float32)
    sharp = np.array([[7, 3], [0, 7]], np.uint8)
    p = R.Params(epf=True)
    s = R.epf_sigma(img, vmap, acm, sharp, p)
    rng_ = np.float32(np.float32(0.05) * np.float32(111.965157))
    for (by, bx), sh in np.ndenumerate(sharp):
        want = min(min(float(rng_), 70.0) * 12.6 * sh / 7.0, 20.0, 170.0)
        assert s[by, bx] == math.trunc(want)
    assert s[1, 0] == 0   # sharpness 0: unfiltered


# --------------------------------------------------------------------------
# L.2 colour and the output encodings
# --------------------------------------------------------------------------
def test_decision_bounds_without_slack_are_the_decisions():
    """With no slack the smallest and largest reachable guide bytes and
    sigmas are the ones J.2.2 and J.2.4 give."""
    img = synth.make_image(72, 48, 61, coef_scale=2.0, acmul=0.5, dc='smooth')
    p = R.Params(epf=True)
    x = R.reconstruct_xyb(img['coeffs'], img['vmap'], img['acmul'], img['cfl'], p)[:, :48, :72]
    g_lo, g_hi, s_lo, s_hi = R.epf_decision_bounds(x, img['vmap'], img['acmul'],
                                                   img['sharpness'], p, 0.0)
    g = R.guide(x, p)
    s = R.epf_sigma(x, img['vmap'], img['acmul'], img['sharpness'], p)
    assert np.array_equal(g_lo, g) and np.array_equal(g_hi, g)
    assert np.array_equal(s_lo, s) and np.array_equal(s_hi, s)
    assert not R.epf_undetermined(x, img['vmap'], img['acmul'], img['sharpness'], p, 0.0).any()


def test_undetermined_pixels_are_the_only_ones_a_perturbation_changes():
    """Decisions taken from inputs whose scaled guide samples move by up to
    +-slack (each sample and channel at random, clamped to the slack) leave
    every pixel that epf_undetermined does not report bit for bit unchanged;
    the reported pixels do change under some of the perturbations."""
    img = synth.make_image(64, 48, 62, coef_scale=2.0, acmul=0.5, dc='smooth')
    p = R.Params(epf=True)
    x = R.reconstruct_xyb(img['coeffs'], img['vmap'], img['acmul'], img['cfl'], p)[:, :48, :64]
    args = (img['vmap'], img['acmul'], img['sharpness'], p)
    slack = 0.05
    und = R.epf_undetermined(x, *args, slack)
    assert 0.01 < und.mean() < 0.9
    base = R.epf(x, *args)
    rng = np.random.default_rng(5)
    changed = np.zeros_like(und)
    scale = np.asarray(p.epf_scale)[:, None, None]
    for _ in range(6):
        d = x + rng.uniform(-slack, slack, size=x.shape) / scale
        got = R.epf(x, *args, decide=d)
        diff = np.any(got != base, axis=0)
        assert not (diff & ~und).any()
        changed |= diff
    assert changed.any()
    # another evaluation's decisions widen exactly the decisions it takes
    # differently (one below the real sigma on some blocks, one guide byte up)
    s_real = R.epf_sigma(x, *args)
    low = np.zeros_like(s_real, bool)
    low[::2, ::3] = True
    g = R.guide(x, p)
    g_alt = g.copy()
    g_alt[1, 5, 7] += 1
    g_lo, g_hi, lo, hi = R.epf_decision_bounds(x, *args, 0.0, guide_alt=g_alt,
                                               sigma_alt=np.where(low, s_real - 1, s_real))
    assert np.array_equal(lo != hi, low) and np.array_equal(hi, s_real)
    assert np.array_equal(lo[low], s_real[low] - 1)
    assert (g_lo != g_hi).sum() == 1 and g_hi[1, 5, 7] == g[1, 5, 7] + 1


def test_dc_smooth_margin():
    """The margin is the distance of wa to the nearer window end: zero for a
    sample whose neighbourhood puts wa exactly on an end, and a perturbation
    of every sample smaller than margin / 3 (the weights sum to 1, and the
    centre also moves the window) keeps every decision."""
    p = R.Params(dc_smooth=True)
    w0, w1, w2 = R.DC_SMOOTH_W
    half = 0.5 * p.m_dc[1]
    # centre 0, every neighbour t: wa = (1 - w0) t, on the upper end when
    # (1 - w0) t = half
    t = half / (1.0 - w0)
    dc = np.zeros((3, 3, 3))
    dc[1] = t
    dc[1, 1, 1] = 0.0
    assert R.dc_smooth_margin(dc, p)[1, 1, 1] == pytest.approx(0.0, abs=1e-18)
    im = synth.make_image(160, 120, 63, mix='dct8', dc='smooth')
    raw = R.dc_image(im['coeffs'], im['vmap'], p)
    m = R.dc_smooth_margin(raw, p)
    def decisions(d):
        wa, s_, hf = R._dc_window(d, p)
        return (s_ - hf <= wa) & (wa <= s_ + hf)

    rng = np.random.default_rng(3)
    eps = 1e-3 * np.asarray(p.m_dc)[:, None, None]
    pert = raw + rng.uniform(-1, 1, raw.shape) * eps
    moved = decisions(pert) != decisions(raw)
    assert not (moved & (m[:, 1:-1, 1:-1] > 3 * eps)).any()
    assert 0.2 < decisions(raw).mean() < 0.8
    assert np.isinf(m[:, 0, :]).all() and np.isinf(m[:, :, -1]).all()


def test_xyb_round_trip_through_opsin_inverse():
    """L.2 applies the inverse opsin matrix; inverting that matrix and the
    cube by hand from linear RGB and going back must return the RGB."""
    p = R.Params()
    rgb = np.random.default_rng(2).uniform(0.0, 1.0, (5, 7, 3))
    M = np.array(p.inv_opsin).reshape(3, 3)
    div = p.target_nits_div50 * 50 / 250
    mix = np.einsum('ij,hwj->hwi', np.linalg.inv(M), rgb * 255.0 * div)
    gam = np.cbrt(mix - np.array(p.opsin_bias))
    X = (gam[..., 0] - gam[..., 1]) / 2
    Y = (gam[..., 0] + gam[..., 1]) / 2
    B = gam[..., 2]
    back = R.xyb_to_linear01(np.stack([X, Y, B]), p)
    np.testing.assert_allclose(back, rgb, atol=1e-12)


def test_srgb_encoding_values():
    """IEC 61966-2-1: 0 -> 0, 1 -> 255, 0.5 -> 0.7354 -> 188, linear segment
    below 0.0031308 (slope 12.92)."""
    v = R.srgb_u8(np.array([0.0, 1.0, 0.5, 0.002, -1.0, 2.0]))
    assert list(v) == [0, 255, 188, 7, 0, 255]



# --------------------------------------------------------------------------
# F.2 adaptive DC smoothing
# --------------------------------------------------------------------------
def test_dc_smoothing_weights_and_invariants():
    """The nine weights of F.2 sum to one, so constant and linear DC images
    are fixed points; borders are untouched; a lone spike is smoothed only
    when the average stays within half a quantisation step."""
    w0, w1, w2 = R.DC_SMOOTH_W
    assert w0 + 4 * w1 + 4 * w2 == pytest.approx(1.0, abs=1e-15)
    p = R.Params(m_dc=(0.1, 0.1, 0.1))
    yy, xx = np.mgrid[0:9, 0:11]
    ramp = np.stack([0.01 * xx + 0.02 * yy, np.full((9, 11), 0.3), -0.01 * yy]).astype(np.float32)
    np.testing.assert_allclose(R.dc_smooth(ramp, p), ramp, atol=1e-6)
    spike = np.zeros((3, 5, 5), np.float32)
    spike[:, 2, 2] = 0.04          # wa = w0 * 0.04, deviation 0.038 < 0.05: smoothed
    out = R.dc_smooth(spike, p)
    assert out[0, 2, 2] == pytest.approx(w0 * 0.04, rel=1e-6)
    assert out[0, 1, 2] == pytest.approx(w1 * 0.04, rel=1e-6)
    assert out[0, 1, 1] == pytest.approx(w2 * 0.04, rel=1e-6)
    spike[:, 2, 2] = 0.2           # deviation 0.19 > 0.05: kept
    out = R.dc_smooth(spike, p)
    assert out[0, 2, 2] == pytest.approx(0.2)
    assert out[0, 0, 2] == 0.0 and out[0, 4, 4] == 0.0   # border samples untouched


def test_dc_smoothing_reaches_the_pixels():
    """With smoothing the DC samples of the varblocks change as F.2 says, and
    the box means of the reconstruction follow them (I.2.6/I.2.7)."""
    im = synth.make_image(64, 48, 11, dc='smooth')
    p = R.Params(dc_smooth=True)
    raw = R.dc_image(im['coeffs'], im['vmap'], p)
    dci = R.dc_smooth(raw, p)
    assert 0.2 < np.mean(dci != raw) < 0.8      # the workload exercises both outcomes
    x = R.reconstruct_xyb(im['coeffs'], im['vmap'], im['acmul'], np.zeros_like(im['cfl']), p)
    # AC contributes zero mean to every 8x8 block of a DCT8 varblock
    for by, bx in zip(*np.nonzero(im['vmap'] == 0)):
        mean = x[:, 8 * by:8 * by + 8, 8 * bx:8 * bx + 8].mean(axis=(1, 2))
        np.testing.assert_allclose(mean, dci[:, by, bx], atol=1e-9)


# --------------------------------------------------------------------------
# Annex H AC prediction; I.2.6 / I.2.7 at N = 4
# --------------------------------------------------------------------------
def _inverse_any(code, coef):
    return TR.idct_2d(coef) if code in R._DCT_SHAPES else TR.idct_8x8_class(code, coef)


@pytest.mark.parametrize('code', range(15))
def test_lf_from_image4_inverts_the_4x4_means(code):
    """I.2.7.1: the N = 4 coefficients reproduce the given 4x4 means when
    reconstructed by the shape's own inverse transform (I.2.4), for every
    DctSelect code, the printed 8x4 / 4x8 / AFV forms included."""
    W, H = T.SHAPE_WH[code]
    img = np.random.default_rng(code).normal(size=(H // 4, W // 4))
    c = R.lf_from_image4(code, img)
    coef = np.zeros((H, W))
    coef[:H // 4, :W // 4] = c
    means = _inverse_any(code, coef).reshape(H // 4, 4, W // 4, 4).mean(axis=(1, 3))
    np.testing.assert_allclose(means, img, atol=1e-12)


def test_half_mean_scale_is_the_printed_scalef():
    """The 8x4 / 4x8 factor read as an exact inverse equals the printed
    ScaleF(2, 8, 1) of I.2.7.3."""
    assert R.half_mean_scale() == pytest.approx(T.ScaleF(2, 8, 1), rel=1e-14)


@pytest.mark.parametrize('code', R._DCT_SHAPES)
def test_downsample4_matches_printed_scalef(code):
    """I.2.6.2 as printed with N = 4 (ScaleF, then an IDCT of the LF size)
    equals the 4x4 box means of the LLF-only reconstruction; and the 2x2
    means of the 4x image are the 8x DC samples (I.2.7 at N = 8)."""
    W, H = T.SHAPE_WH[code]
    rng = np.random.default_rng(100 + code)
    dc = rng.normal(size=(H // 8, W // 8))
    llf = TR.llf_from_dc(dc)
    d4 = R.downsample4(code, llf)
    coef = np.zeros((H, W))
    coef[:H // 8, :W // 8] = llf
    np.testing.assert_allclose(TR.downsample_scalef(coef, N=4), d4, atol=1e-13)
    np.testing.assert_allclose(d4.reshape(H // 8, 2, W // 8, 2).mean(axis=(1, 3)), dc, atol=1e-13)


def test_lf_smoothing_weights_and_threshold():
    """Annex H smoothing: weights sum to one (constant and linear images are
    fixed points); a spike is averaged with 0.12 / 0.2 / 0.02 only within
    1.7 dcq; the 2-sample ring is never changed."""
    wc, we, wd = R.LF_SMOOTH_W
    assert wc + 4 * we + 4 * wd == pytest.approx(1.0, abs=1e-15)
    yy, xx = np.mgrid[0:10, 0:12]
    ramp = 0.3 + 0.01 * xx - 0.02 * yy
    sm, _ = R.lf_smooth(ramp, 0.1)
    np.testing.assert_allclose(sm, ramp[2:-2, 2:-2], atol=1e-15)
    img = np.zeros((7, 7))
    img[3, 3] = 0.1                          # |wa - s| = 0.088 <= 0.17: averaged
    sm, _ = R.lf_smooth(img, 0.1)
    assert sm[1, 1] == pytest.approx(0.012)
    assert sm[0, 1] == pytest.approx(0.02) and sm[0, 0] == pytest.approx(0.002)
    img[3, 3] = 1.0                          # |wa - s| = 0.88 > 0.17: kept
    sm, _ = R.lf_smooth(img, 0.1)
    assert sm[1, 1] == 1.0
    assert sm.shape == (3, 3)


@pytest.mark.parametrize('mix', ['mixed', 3, 12, 13, 14, 1, 2])
def test_ac_prediction_closes_the_loop(mix):
    """With only DC transmitted, the W/4 x H/4 coefficients that the
    reconstruction's own 4x4 means imply (I.2.7 at N = 4) are the LLF
    coefficients from the DC samples in the LLF corner and those of the
    smoothed DC2x2 image outside it (Annex H + I.2.4); a constant DC image
    yields no prediction at all."""
    im = synth.make_image(72, 56, 5, mix=mix, dc='smooth', ac=False)
    p = R.Params(dc_smooth=True, lf_predict=True)
    diag = {}
    x = R.reconstruct_xyb(im['coeffs'], im['vmap'], im['acmul'], im['cfl'], p, diag)
    base = R.dequantize(im['coeffs'], im['vmap'], im['acmul'], im['cfl'], R.Params(dc_smooth=True))
    _, Hp, Wp = x.shape
    means = x.reshape(3, Hp // 4, 4, Wp // 4, 4).mean(axis=(2, 4))
    us = diag['lf_image']
    assert np.abs(us - means).max() > 1e-4          # the prediction did something
    for code, bx, by in R.varblocks(im['vmap']):
        W, H = T.SHAPE_WH[code]
        llf = np.zeros((H // 4, W // 4), dtype=bool)
        llf[:H // 8, :W // 8] = True
        for c in range(3):
            area = (slice(2 * by, 2 * by + H // 4), slice(2 * bx, 2 * bx + W // 4))
            got = R.lf_from_image4(code, means[c][area])
            want = np.where(llf, base[c, 8 * by:8 * by + H // 4, 8 * bx:8 * bx + W // 4],
                            R.lf_from_image4(code, us[c][area]))
            np.testing.assert_allclose(got, want, atol=1e-12)
    u, v, ox, oy = synth.coefficient_positions(im['vmap'])
    slots = synth.llf_slots(im['vmap'], u, v, ox, oy)
    q = np.broadcast_to(np.where(slots, 7, 0), im['coeffs'].shape).astype(np.int16)
    a = R.dequantize(q, im['vmap'], im['acmul'], np.zeros_like(im['cfl']), R.Params())
    b = R.dequantize(q, im['vmap'], im['acmul'], np.zeros_like(im['cfl']),
                     R.Params(lf_predict=True))
    np.testing.assert_allclose(a, b, atol=1e-15)


def test_ac_prediction_ring_reads_only_the_border_dc():
    """A group's prediction depends on its own varblocks and the 1-block ring
    of DC samples around it, not on anything further out: two images that
    agree on group 0 (256 x 256) and its ring agree there; a change inside
    the ring does reach group 0."""
    im = synth.make_image(280, 64, 9, mix='dct8', dc='smooth')
    p = R.Params(lf_predict=True)
    base = R.dequantize(im['coeffs'], im['vmap'], im['acmul'], im['cfl'], p)
    far = im['coeffs'].copy()
    far[:, :, 8 * 34:] += 5                   # blocks 34.. (beyond the ring at 32)
    other = R.dequantize(far, im['vmap'], im['acmul'], im['cfl'], p)
    np.testing.assert_array_equal(other[:, :, :256], base[:, :, :256])
    near = im['coeffs'].copy()
    near[:, ::8, 8 * 32] += 5                 # DC of the ring column (block 32)
    other = R.dequantize(near, im['vmap'], im['acmul'], im['cfl'], p)
    assert np.abs(other[:, :, 248:256] - base[:, :, 248:256]).max() > 0


# --------------------------------------------------------------------------
# J.3 quantization constraint
# --------------------------------------------------------------------------
def _qco_case(mix, seed=3, xs=72, ys=56):
    im = synth.make_image(xs, ys, seed, mix=mix)
    p = R.Params()
    orig = R.reconstruct_xyb(im['coeffs'], im['vmap'], im['acmul'], im['cfl'], p)
    rng = np.random.default_rng(seed + 1)
    filt = orig[:, :ys, :xs] + rng.normal(0, 0.02, size=(3, ys, xs)) * \
        np.abs(orig[:, :ys, :xs]).mean(axis=(1, 2), keepdims=True)
    return im, orig, filt


@pytest.mark.parametrize('code', range(15))
def test_forward_transform_inverts_every_shape(code):
    """I.2.3 against I.2.4: the forward transform of every shape is the exact
    inverse of its reconstruction procedure."""
    W, H = T.SHAPE_WH[code]
    x = np.random.default_rng(code).normal(size=(H, W))
    np.testing.assert_allclose(R.inverse_any(code, R.forward_transform(code, x)), x, atol=1e-12)


@pytest.mark.parametrize('mix', ['mixed', 1, 2, 3, 12, 13, 14])
def test_qco_limits_and_invariants(mix):
    """J.3: with an unbounded interval the filter output passes unchanged;
    with a zero interval the filter input comes back; the output residual's
    coefficients lie inside the intervals (DC samples within the DC
    interval); applying the constraint twice changes nothing."""
    im, orig, filt = _qco_case(mix)
    ys, xs = filt.shape[1:]
    big = R.Params(qco_interval_mul=1e12)
    np.testing.assert_allclose(R.qco(filt, orig, im['vmap'], im['acmul'], big), filt, atol=1e-9)
    zero = R.Params(qco_interval_mul=0.0)
    np.testing.assert_allclose(R.qco(filt, orig, im['vmap'], im['acmul'], zero),
                               orig[:, :ys, :xs], atol=1e-12)
    p = R.Params()
    out = R.qco(filt, orig, im['vmap'], im['acmul'], p)
    assert np.abs(out - filt).max() > 1e-6          # something was clamped
    np.testing.assert_allclose(R.qco(out, orig, im['vmap'], im['acmul'], p), out, atol=1e-10)
    res = np.zeros_like(orig)
    res[:, :ys, :xs] = out - orig[:, :ys, :xs]
    for code, bx, by in R.varblocks(im['vmap']):
        W, H = T.SHAPE_WH[code]
        cx, cy = W // 8, H // 8
        for c in range(3):
            coef = R.forward_transform(code, res[c, 8 * by:8 * by + H, 8 * bx:8 * bx + W])
            lim = 0.5 * im['acmul'][by, bx] * T.dequant_matrix(code, c)
            hf = np.ones((H, W), bool)
            hf[:cy, :cx] = False
            assert np.all(np.abs(coef[hf]) <= lim[hf] * (1 + 1e-9) + 1e-12)
            if code in R._DCT_SHAPES:
                dc = TR.box_mean_map(W, H) @ coef[:cy, :cx].reshape(-1)
            else:
                dc = coef[:1, :1].reshape(-1)
            assert np.all(np.abs(dc) <= 0.5 * p.m_dc[c] * (1 + 1e-9) + 1e-15)


def test_qco_dc_interval_is_the_block_mean():
    """A residual that is constant over an 8x8 DCT8 block is pure DC: it is
    clamped to +-mul x m_DC of the channel, whatever its AC intervals."""
    im = synth.make_image(16, 16, 1, mix='dct8', acmul=1.0)
    p = R.Params()
    orig = np.zeros((3, 16, 16))
    filt = np.zeros((3, 16, 16))
    filt[:, :8, :8] = 1.0
    out = R.qco(filt, orig, im['vmap'], im['acmul'], p)
    for c in range(3):
        np.testing.assert_allclose(out[c, :8, :8], 0.5 * p.m_dc[c], rtol=1e-9)
    np.testing.assert_allclose(out[:, 8:, :], 0.0, atol=1e-15)
    np.testing.assert_allclose(out[:, :, 8:], 0.0, atol=1e-15)
