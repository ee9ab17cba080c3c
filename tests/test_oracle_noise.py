"""Pins of the K.5 noise oracle against what the draft, the published
generators and the mathematics fix."""
import numpy as np
import pytest

from oracle import noise as N


def test_splitmix64_published_outputs():
    """SplitMix64 as defined in K.5.2 (the mixing step; the seeding adds the
    golden gamma first): from state 0 the published generator's first two
    outputs."""
    assert N.splitmix64(0 + N.GOLDEN_GAMMA) == 0xE220A8397B1DCDAF
    assert N.splitmix64(2 * N.GOLDEN_GAMMA) == 0x6E789E6AA1B965F4


def test_generator_state_rotation_and_linearity():
    """The state update rotates the words (the new s0 is the old s1) and is
    linear over GF(2), as every xorshift update is."""
    rng = np.random.default_rng(0)
    a0, a1 = (rng.integers(0, 2**63, size=8, dtype=np.uint64) for _ in range(2))
    b0, b1 = (rng.integers(0, 2**63, size=8, dtype=np.uint64) for _ in range(2))
    n0, n1, _ = N.step(a0, a1)
    np.testing.assert_array_equal(n0, a1)
    m0, m1, _ = N.step(b0, b1)
    x0, x1, _ = N.step(a0 ^ b0, a1 ^ b1)
    np.testing.assert_array_equal(x0, n0 ^ m0)
    np.testing.assert_array_equal(x1, n1 ^ m1)
    assert np.all(n1 != 0)


def test_random_channels_statistics_and_determinism():
    r = N.random_channels(0, 0, 256, 64)
    assert r.dtype == np.float32 and r.min() >= 0.0 and r.max() < 1.0
    assert np.all((r * 2**23) == np.floor(r * 2**23))            # 23-bit mantissas
    assert abs(r.mean() - 0.5) < 0.01 and abs(r.var() - 1 / 12) < 0.005
    np.testing.assert_array_equal(r, N.random_channels(0, 0, 256, 64))
    other = N.random_channels(256, 0, 256, 64)
    assert np.mean(other == r) < 0.01
    # a narrower group consumes one step of all generators per 16 samples:
    # its first 16 columns equal those of a full-width group at the same origin
    np.testing.assert_array_equal(N.random_channels(0, 0, 20, 3)[0, 0, :16], r[0, 0, :16])


def test_laplacian_kernel():
    """Constants map to 0; a spike gives -4 at the centre and 1 at distance 2
    on the axes; at the bounds index -1 reads 0 and -2 reads 1 (6.5)."""
    np.testing.assert_allclose(N.laplacian(np.full((9, 7), 3.0)), 0.0, atol=1e-12)
    x = np.zeros((9, 9))
    x[4, 4] = 1.0
    l = N.laplacian(x)
    assert l[4, 4] == -4.0 and l[2, 4] == 1.0 and l[6, 4] == 1.0 and l[4, 2] == 1.0 and l[4, 6] == 1.0
    assert np.count_nonzero(l) == 5
    row = np.arange(6, dtype=np.float64)[None, :].repeat(5, 0)
    l = N.laplacian(row)
    # x = 0: x[-2] = x[1] = 1, x[2] = 2 -> 1 + 2 - 0 = 3 (the vertical taps cancel)
    assert l[2, 0] == pytest.approx(3.0)
    assert l[2, 3] == pytest.approx(0.0)                        # interior of a ramp


def test_strength_interpolation():
    """K.5.3: with LUT[i] = i / 15 the strength is In x 14 / 15 on [0, 1),
    clamped to [0, 1]; a zero LUT gives no noise."""
    lut = np.arange(16) / 15.0
    v = np.linspace(0.0, 0.99, 50)
    np.testing.assert_allclose(N.strength(v, lut), v * 14 / 15, atol=1e-12)
    assert np.all(N.strength(np.array([-3.0, 5.0]), np.full(16, 2.0)) == 1.0)
    xyb = np.random.default_rng(1).normal(0, 0.1, size=(3, 40, 300))
    np.testing.assert_array_equal(N.add_noise(xyb, np.zeros(16)), xyb)


def test_additive_update_couples_y_and_b():
    """The B update is 0.935669 times the Y update at every pixel, and the
    noise crosses group boundaries (two groups along x)."""
    xyb = np.zeros((3, 20, 300))
    xyb[1] = 0.5
    out = N.add_noise(xyb, np.full(16, 0.5))
    dy, db = out[1] - xyb[1], out[2] - xyb[2]
    assert np.abs(dy).max() > 1e-3
    np.testing.assert_allclose(db, 0.935669 * dy, atol=1e-15)
