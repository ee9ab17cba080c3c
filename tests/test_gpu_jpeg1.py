"""Parity of JPEG1 direct rasterisation (M.6, through the C ABI) with the FP64
oracle.

Bounds: f32 output (sample / 255) within 1e-5 of the oracle (binary32 IDCT
and colour arithmetic on samples of magnitude <= ~2); u8 within +-1 (the
rounding of a sample at a .5 boundary may go either way); f16 within half
an f16 ulp + 1e-5.  The block-conditional Gaborish of M.6.3 decides per
block from |sample - smoothed| > threshold: blocks with an inner sample
within 1e-3 of the threshold may go either way, so their output footprint
is excluded (and counted: the test fails if more than 5% of the blocks are).
"""
import numpy as np
import pytest

from oracle import jpeg1 as J
from paper_1908_03565_gb300 import synth
from test_gpu_parity import B  # noqa: F401

pytestmark = pytest.mark.gpu

F32, F16, U8, XYB = 0, 1, 2, 3
GAB_AMBIG = 1e-3


@pytest.fixture(scope="module")
def ctx(B):
    c = B.Context(max_slots=2)
    yield c
    c.close()


def _run(B, ctx, stream, dtype, device_io=True):
    import torch
    xs, ys = stream['xsize'], stream['ysize']
    npd = {F32: np.float32, F16: np.float16, U8: np.uint8}[dtype]
    if device_io:
        ds = B.jpeg_to_device(stream, torch)
        tdt = {np.float32: torch.float32, np.float16: torch.float16, np.uint8: torch.uint8}[npd]
        out = torch.full((ys, xs, 3), 7, dtype=tdt, device="cuda")
        ctx.poll(ctx.submit_jpeg(ds, out, dtype, on_device=True))
        return out.cpu().numpy()
    out = np.full((ys, xs, 3), 7, dtype=npd)
    ctx.poll(ctx.submit_jpeg(stream, out, dtype, on_device=False, out_on_device=False))
    return out


def _gab_mask(stream):
    """Output pixels whose value may depend on a near-tie M.6.3 decision."""
    xs, ys = stream['xsize'], stream['ysize']
    comps = stream['components']
    hmax = max(c['h_samp'] for c in comps)
    vmax = max(c['v_samp'] for c in comps)
    mask = np.zeros((ys, xs), bool)
    nblk = amb = 0
    for c in comps:
        if c.get('gab') is None:
            continue
        w1, w2, thr, _ = c['gab']
        p = J.component_pixels(c['coeffs'], c['quant'])
        s = J.gaborish_plane(p, w1, w2)
        near = np.abs(np.abs(p - s) - thr) < GAB_AMBIG
        bh, bw = c['coeffs'].shape[:2]
        sx, sy = hmax // c['h_samp'], vmax // c['v_samp']
        for by in range(bh):
            for bx in range(bw):
                nblk += 1
                if near[8 * by + 1:8 * by + 7, 8 * bx + 1:8 * bx + 7].any():
                    amb += 1
                    x0, y0 = max(0, 8 * bx * sx - 1), max(0, 8 * by * sy - 1)
                    mask[y0:8 * (by + 1) * sy + 1, x0:8 * (bx + 1) * sx + 1] = True
    assert amb <= 0.05 * max(nblk, 1), (amb, nblk)
    return mask


@pytest.mark.parametrize("sampling,xs,ys", [('420', 64, 48), ('420', 131, 77), ('444', 40, 24),
                                            ('grey', 33, 19), ('420', 9, 7), ('420', 512, 264)])
def test_jpeg1_outputs(B, ctx, sampling, xs, ys):
    """M.6.1-M.6.6 without the side channel: f32, f16 and u8 outputs."""
    st = synth.make_jpeg(xs, ys, 1000 + xs + ys, sampling=sampling)
    want = J.rasterize(st)
    got = _run(B, ctx, st, F32)
    np.testing.assert_allclose(got, want / 255.0, atol=1e-5, rtol=0)
    h = _run(B, ctx, st, F16).astype(np.float64)
    w01 = want / 255.0
    ulp = np.spacing(np.abs(w01).astype(np.float16)).astype(np.float64)
    assert np.all(np.abs(h - w01) <= 0.5 * ulp + 1e-5)
    d8 = np.abs(_run(B, ctx, st, U8).astype(np.int64) - J.to_u8(want).astype(np.int64))
    assert d8.max() <= 1


@pytest.mark.parametrize("sampling,xs,ys", [('420', 136, 104), ('444', 72, 56), ('grey', 64, 40)])
def test_jpeg1_conditional_gaborish(B, ctx, sampling, xs, ys):
    """M.6.3 on every component, then upsampling and colour."""
    # AC scale 3: about 40% of the blocks take the smoothed samples
    st = synth.make_jpeg(xs, ys, 2000 + xs, sampling=sampling, gab=True, ac_scale=3.0)
    want = J.rasterize(st)
    plain = J.rasterize(synth.make_jpeg(xs, ys, 2000 + xs, sampling=sampling, ac_scale=3.0))
    assert np.abs(want - plain).max() > 0.1           # the side channel changed blocks
    mask = _gab_mask(st)
    got = _run(B, ctx, st, F32)
    keep = ~mask[..., None]
    np.testing.assert_allclose(np.where(keep, got, want / 255.0), want / 255.0, atol=1e-5, rtol=0)


def test_jpeg1_host_and_device_inputs_agree(B, ctx):
    st = synth.make_jpeg(200, 136, 5, sampling='420', gab=True)
    np.testing.assert_array_equal(_run(B, ctx, st, U8), _run(B, ctx, st, U8, device_io=False))


def test_jpeg1_rejects_ill_formed_streams(B, ctx):
    import torch
    st = synth.make_jpeg(64, 64, 6, sampling='420')
    out = torch.empty((64, 64, 3), dtype=torch.uint8, device="cuda")
    bad = dict(st)
    bad['components'] = st['components'][:2]             # 2 components
    with pytest.raises(B.JxlrError) as e:
        ctx.submit_jpeg(B.jpeg_to_device(bad, torch), out, U8)
    assert e.value.status == B.JXLR_EINVAL
    bad = dict(st)
    bad['components'] = [dict(c) for c in st['components']]
    bad['components'][1]['h_samp'] = 3                  # unsupported factor
    with pytest.raises(B.JxlrError):
        ctx.submit_jpeg(B.jpeg_to_device(bad, torch), out, U8)
    bad = dict(st)
    bad['xsize'] = 80                                  # grid does not cover the image
    with pytest.raises(B.JxlrError):
        ctx.submit_jpeg(B.jpeg_to_device(bad, torch), torch.empty((64, 80, 3), dtype=torch.uint8,
                                                                  device="cuda"), U8)
    with pytest.raises(B.JxlrError):                    # XYB output is not defined here
        ctx.submit_jpeg(B.jpeg_to_device(st, torch),
                        torch.empty((64, 64, 3), dtype=torch.float32, device="cuda"), XYB)
    # the context still works
    assert _run(B, ctx, st, U8).shape == (64, 64, 3)


@pytest.mark.parametrize("sampling,xs,ys", [('420', 200, 136), ('444', 72, 56), ('grey', 131, 77)])
def test_jpeg1_conditioning(B, ctx, sampling, xs, ys):
    """M.6.1.1 on staircase DC with mostly zero first AC coefficients: the
    plateau decisions are binary32 on both sides, so the outputs agree
    within float rounding everywhere."""
    st = synth.make_jpeg(xs, ys, 3000 + xs, sampling=sampling, plateaus=True, cond=(0.5, 0.5))
    want = J.rasterize(st)
    plain = dict(st)
    plain['components'] = [dict(c, cond=None) for c in st['components']]
    assert np.abs(want - J.rasterize(plain)).max() > 0.1       # conditioning changed samples
    got = _run(B, ctx, st, F32)
    np.testing.assert_allclose(got, want / 255.0, atol=1e-5, rtol=0)
    np.testing.assert_array_equal(_run(B, ctx, st, U8), _run(B, ctx, st, U8, device_io=False))
