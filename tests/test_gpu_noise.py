"""Parity of K.5 noise synthesis (through the C ABI) with the FP64 oracle.

The generator is integer arithmetic on both sides (the library jumps each
generator to its 32-row chunk with GF(2) matrices; the oracle steps through
the group sequentially), so with a constant strength LUT the output depends
only on the random channels and is compared within binary32 rounding.  With
a varying LUT the strength is discontinuous where In x 14 crosses an integer
outside [0, 15) (the printed clamp of the integer part only); pixels within
1e-4 of such a point are excluded and counted.
"""
import numpy as np
import pytest

from oracle import noise as N
from oracle import recon as R
from paper_1908_03565_gb300 import synth
from test_gpu_parity import B, ctx, XYB, F32, params_pair, run  # noqa: F401

pytestmark = pytest.mark.gpu


def _staged(B, ctx, xyb, lp, dtype=XYB, img=None):
    """Filters + noise + colour of the library on caller XYB (3, ys, xs)."""
    import torch
    _, ys, xs = xyb.shape
    if img is None:
        img = synth.make_image(xs, ys, 1)
    dx = torch.from_numpy(np.ascontiguousarray(xyb, dtype=np.float32)).cuda()
    tdt = torch.float32 if dtype in (XYB, F32) else torch.uint8
    out = torch.empty((ys, xs, 3), dtype=tdt, device="cuda")
    dimg = B.to_device(img, torch)
    t = ctx.submit_xyb(dx, xs, ys, dimg['vmap'], dimg['acmul'], dimg['sharpness'], lp, out, dtype)
    ctx.poll(t)
    return out.cpu().numpy().transpose(2, 0, 1)


@pytest.mark.parametrize("xs,ys", [(600, 300), (256, 256), (5, 3), (17, 260)])
def test_noise_channels(B, ctx, xs, ys):
    """Zero input and a constant LUT of 1: X = 0.01 (A_R - A_G), Y = 0.01
    (A_R + A_G) + 1.98 A_B, B = 0.935669 Y from the generator alone; groups
    with ragged edges."""
    lp = B.filter_defaults(noise=1, noise_lut=[1.0] * 16)
    xyb = np.zeros((3, ys, xs), np.float32)
    got = _staged(B, ctx, xyb, lp)
    want = N.add_noise(xyb.astype(np.float64), np.ones(16))
    assert np.abs(want).max() > 0.1
    np.testing.assert_allclose(got, want, atol=2e-6, rtol=0)


def test_noise_strength(B, ctx):
    """Smooth XYB spanning the LUT's range, LUT[i] = i / 15."""
    ys, xs = 280, 520
    yy, xx = np.mgrid[0:ys, 0:xs]
    xyb = np.stack([0.05 * np.sin(xx / 37.0), 0.6 + 0.6 * np.sin(yy / 53.0) * np.cos(xx / 71.0),
                    0.3 * np.cos(yy / 29.0)]).astype(np.float32)
    lut = np.arange(16) / 15.0
    lp = B.filter_defaults(noise=1, noise_lut=list(lut))
    got = _staged(B, ctx, xyb, lp)
    want = N.add_noise(xyb.astype(np.float64), lut)
    near = N.margins(xyb) < 1e-4
    assert near.mean() < 0.01
    keep = ~near[None]
    assert np.abs(want - xyb).max() > 1e-3
    np.testing.assert_allclose(np.where(keep, got, want), want, atol=2e-6, rtol=0)


def test_noise_after_filters_full_path(B, ctx):
    """Submit with EPF + Gaborish + noise == reconstruction to XYB, then the
    filter entry point (bitwise); noise alone forces the filter stage."""
    img = synth.make_image(300, 264, 3, y_dc_offset_q=200)
    lp = B.filter_defaults(epf=1, gab=1, noise=1, noise_lut=list(np.linspace(0.2, 0.9, 16)))
    xyb = run(B, ctx, img, params_pair(B)[1], XYB).transpose(2, 0, 1).copy()
    staged = _staged(B, ctx, xyb, lp, F32, img).transpose(1, 2, 0)
    full = run(B, ctx, img, lp, F32)
    np.testing.assert_array_equal(full, staged)
    lp_n = B.filter_defaults(noise=1, noise_lut=[0.5] * 16)
    got = run(B, ctx, img, lp_n, XYB).transpose(2, 0, 1)
    want = N.add_noise(xyb.astype(np.float64), np.full(16, 0.5))
    np.testing.assert_allclose(got, want, atol=2e-6, rtol=1e-6)


def test_noise_only_on_submit_path(B, ctx):
    import torch
    img = synth.make_image(64, 64, 5)
    lp = B.filter_defaults(noise=1)
    dimg = B.to_device(img, torch)
    out = torch.empty((64, 64, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(B.JxlrError) as e:
        ctx.batch([(dimg, lp, out, F32)], autotune=False)
    assert e.value.status == B.JXLR_EINVAL
    with pytest.raises(B.JxlrError) as e:
        B.run_noalloc(dimg, lp, out, F32)
    assert e.value.status == B.JXLR_EINVAL
