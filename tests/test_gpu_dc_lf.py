"""Parity of F.2 adaptive DC smoothing and Annex H AC prediction (through the
C ABI) with the FP64 oracle.

* F.2: the oracle decides in real arithmetic, the kernel in binary32.  A
  sample whose weighted average lies within the binary32 evaluation bound
  (F2_REL of the window's largest |sample|) of a window edge may go either
  way; such samples are counted (at most 1e-3 of them) and excluded.  With
  DC-only DCT8 input every other XYB sample equals the oracle's smoothed DC
  within binary32 rounding, so every decision outside that bound agrees.
* Annex H smooths real-valued DC2x2 samples that the two sides compute in
  different precisions; a sample whose weighted average lies within
  LF_AMBIG of a window edge may go either way, so the varblock holding it is
  excluded (and counted: the test fails if more than 1% of the DC2x2
  samples are near-ties or more than 10% of the area is excluded).
  Everything else is compared with the XYB tolerance of the main parity
  tests.
"""
import numpy as np
import pytest

from oracle import recon as R
from paper_1908_03565_gb300 import synth
from test_gpu_parity import (B, ctx, XYB, F32, assert_xyb_close, local_mag,  # noqa: F401
                             rgb_tolerance, run)

pytestmark = pytest.mark.gpu

LF_AMBIG = 1e-6


def _params(B, smooth, predict, gab=False, kx_dc=0.0, kb_dc=0.0):
    p = R.Params(dc_smooth=smooth, lf_predict=predict, gab=gab, kx_dc=kx_dc, kb_dc=kb_dc)
    lp = B.filter_defaults(dc_smooth=int(smooth), lf_predict=int(predict), gab=int(gab))
    return p, lp


def _ambiguous_varblocks(img, diag):
    """Per-sample mask (padded image) of the varblocks with a near-tie
    smoothing decision; asserts that near-ties are rare."""
    vmap = img['vmap']
    bh, bw = vmap.shape
    near = (diag['lf_margin'] < LF_AMBIG).any(axis=0)           # (2bh, 2bw)
    assert near.mean() < 1e-2
    mask = np.zeros((8 * bh, 8 * bw), dtype=bool)
    vbs = R.varblocks(vmap)
    for code, bx, by in vbs:
        W, H = synth.SHAPE_WH[code]
        if near[2 * by:2 * by + H // 4, 2 * bx:2 * bx + W // 4].any():
            mask[8 * by:8 * by + H, 8 * bx:8 * bx + W] = True
    assert mask.mean() < 0.1
    return mask


F2_REL = 2.0 ** -19   # binary32 DC rounding, 9-term average and window ends


def test_dc_smoothing_decisions(B, ctx):
    """DC-only DCT8 input: every XYB sample of a block is its DC after F.2;
    the kernel's binary32 decisions agree with the real-number ones
    wherever the margin exceeds the binary32 bound; both outcomes occur."""
    from scipy.ndimage import maximum_filter
    img = synth.make_image(200, 136, 21, mix='dct8', dc='smooth', ac=False, cfl=False)
    p, lp = _params(B, True, False)
    raw = R.dc_image(img['coeffs'], img['vmap'], p)
    want = R.dc_smooth(raw, p)
    assert 0.2 < np.mean(want != raw) < 0.8
    mag = maximum_filter(np.abs(raw), size=(1, 3, 3), mode='nearest')
    near = R.dc_smooth_margin(raw, p) < F2_REL * (mag + np.asarray(p.m_dc)[:, None, None])
    assert near.mean() <= 1e-3, near.mean()
    got = run(B, ctx, img, lp, XYB).transpose(2, 0, 1)
    ys, xs = img['ysize'], img['xsize']

    def px(a):
        return np.repeat(np.repeat(a, 8, 1), 8, 2)[:, :ys, :xs]

    err = np.abs(got - px(want))
    tol = 2.0 ** -20 * px(mag)
    bad = (err > tol) & ~px(near)
    assert not bad.any(), f"{bad.sum()} samples, worst {np.where(bad, err, 0).max():.3g}"
    print(f"F.2 near-ties excluded: {int(near.sum())} of {near.size} DC samples")


@pytest.mark.parametrize("xs,ys,seed", [(72, 56, 1), (33, 17, 2), (200, 136, 3), (300, 264, 4)])
def test_dc_smoothing_parity(B, ctx, xs, ys, seed):
    """Mixed varblocks with AC, smooth DC field, CfL for DC and AC."""
    img = synth.make_image(xs, ys, seed, dc='smooth')
    p, lp = _params(B, True, False, kx_dc=0.25, kb_dc=-0.5)
    want = R.reconstruct_xyb(img['coeffs'], img['vmap'], img['acmul'], img['cfl'], p)
    got = run(B, ctx, img, lp, XYB, kx_dc=0.25, kb_dc=-0.5).transpose(2, 0, 1)
    assert_xyb_close(got, want[:, :ys, :xs])


@pytest.mark.parametrize("mix", ['mixed', 'dct8', 1, 2, 3, 12, 13, 14, 5, 10, 11])
@pytest.mark.parametrize("smooth", [True, False])
def test_lf_prediction_parity(B, ctx, mix, smooth):
    """Annex H with and without F.2, per shape family, DC-only input (the
    prediction is then the whole LF content) on 2 x 2 groups with a ragged
    edge."""
    img = synth.make_image(296, 280, 7, mix=mix, dc='smooth', ac=False)
    p, lp = _params(B, smooth, True)
    diag = {}
    want = R.reconstruct_xyb(img['coeffs'], img['vmap'], img['acmul'], img['cfl'], p, diag)
    got = run(B, ctx, img, lp, XYB).transpose(2, 0, 1)
    mask = _ambiguous_varblocks(img, diag)
    ys, xs = img['ysize'], img['xsize']
    keep = ~mask[:ys, :xs]
    err = np.where(keep[None], got, want[:, :ys, :xs])
    assert_xyb_close(err, want[:, :ys, :xs])
    # the prediction changed the image
    base = R.reconstruct_xyb(img['coeffs'], img['vmap'], img['acmul'], img['cfl'],
                             R.Params(dc_smooth=smooth))
    assert np.abs(want - base).max() > 1e-3


@pytest.mark.parametrize("xs,ys,seed", [(520, 264, 11), (95, 64, 12)])
def test_dc_and_lf_full_path(B, ctx, xs, ys, seed):
    """Both steps with AC, CfL and Gaborish, linear RGB output (the RGB bound
    of the main parity tests: 1e-4 plus the XYB bound through L.2); host and
    device inputs give identical bytes."""
    img = synth.make_image(xs, ys, seed, dc='smooth')
    p, lp = _params(B, True, True, gab=True)
    diag = {}
    out = R.reconstruct(img, p, diag)
    mask = _ambiguous_varblocks(img, diag)
    # XYB before the filters
    want = out['xyb_padded'][:, :ys, :xs]
    got_xyb = run(B, ctx, img, _params(B, True, True)[1], XYB).transpose(2, 0, 1)
    assert_xyb_close(np.where(mask[None, :ys, :xs], want, got_xyb), want)
    got = run(B, ctx, img, lp, F32)
    # Gaborish spreads an excluded varblock by one sample
    from scipy.ndimage import binary_dilation
    keep = ~binary_dilation(mask, iterations=1)[:ys, :xs]
    tol = rgb_tolerance(out['xyb'], local_mag(out['xyb'], out['xyb_padded'][:, :ys, :xs]), p)
    err = np.abs(np.clip(got, 0, 1) - np.clip(out['rgb01'], 0, 1))
    bad = (err > tol) & keep[..., None]
    if bad.any():
        i = np.unravel_index(np.where(bad, err - tol, -1).argmax(), err.shape)
        raise AssertionError(f"{bad.sum()} samples out of tolerance; worst at {i}: err {err[i]:.3g} "
                             f"tol {tol[i]:.3g} rgb {out['rgb01'][i[0], i[1]]} "
                             f"xyb {out['xyb'][:, i[0], i[1]]} masked-near {mask[i[0], i[1]]}")
    host = run(B, ctx, img, lp, F32, device_io=False)
    np.testing.assert_array_equal(host, got)


def test_dc_steps_with_invalid_maps(B, ctx):
    """The DC-domain kernels stay inside their buffers for a map the device
    validation rejects; the context keeps working."""
    import torch
    img = synth.make_image(64, 64, 3, dc='smooth')
    _, lp = _params(B, True, True)
    bad = dict(img)
    vm = img['vmap'].copy()
    vm[0, 0] = 5
    vm[1, 1] = 0
    vm[3, 3] = 16
    vm[7, 7] = 5          # a DCT32 that would reach past the image
    bad['vmap'] = vm
    dimg = B.to_device(bad, torch)
    dout = torch.empty((64, 64, 3), dtype=torch.float32, device="cuda")
    t = ctx.submit(dimg, lp, dout, F32, on_device=True)
    with pytest.raises(B.JxlrError) as e:
        ctx.poll(t)
    assert e.value.status == B.JXLR_EINVAL
    assert np.isfinite(run(B, ctx, img, lp, F32)).all()


def test_dc_steps_only_on_submit_path(B, ctx):
    """Batches and the no-allocation entry point reject the two steps."""
    import torch
    img = synth.make_image(64, 64, 5)
    _, lp = _params(B, True, False)
    dimg = B.to_device(img, torch)
    out = torch.empty((64, 64, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(B.JxlrError) as e:
        ctx.batch([(dimg, lp, out, F32)], autotune=False)
    assert e.value.status == B.JXLR_EINVAL
    with pytest.raises(B.JxlrError) as e:
        B.run_noalloc(dimg, lp, out, F32)
    assert e.value.status == B.JXLR_EINVAL
