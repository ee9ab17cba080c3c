"""Parity of the J.3 quantization constraint (through the C ABI) with the FP64
oracle.

The constraint runs on the EPF output.  As in the filter-stage tests, both
sides start from the same binary32 XYB samples (the GPU's own
reconstruction); the oracle takes the EPF's decisions in real arithmetic,
and the EPF pixels those decisions do not fix within the binary32 rounding
(counted, rare) exclude their whole varblock, since J.3 spreads a residual
over its varblock.  The clamp itself is continuous, so the result is
compared with the XYB bound of the main parity tests over a varblock-sized
neighbourhood.
"""
import numpy as np
import pytest

from oracle import recon as R
from paper_1908_03565_gb300 import synth
from test_gpu_parity import (B, ctx, XYB, F32, assert_rare, assert_xyb_close,  # noqa: F401
                             params_pair, run, undetermined)

pytestmark = pytest.mark.gpu

# Inputs on which the EPF and the constraint act on most samples (with the
# workload's coefficient statistics every EPF weight but the centre's falls
# below the cut-off): small AC, a smooth DC field, AcMul 0.5.
ACTIVE = dict(coef_scale=2.0, acmul=0.5, dc='smooth')


def _params(B, mul=0.5, gab=False):
    p = R.Params(epf=True, gab=gab, qco=True, qco_interval_mul=mul)
    lp = B.filter_defaults(epf=1, gab=int(gab), qco=1, qco_interval_mul=mul)
    return p, lp


def _gpu_xyb(B, ctx, img):
    return run(B, ctx, img, params_pair(B)[1], XYB).transpose(2, 0, 1).copy()


def _staged(B, ctx, img, xyb, lp, dtype):
    """EPF (+ QCO, + Gaborish) and colour of the library on caller XYB."""
    import torch
    xs, ys = img['xsize'], img['ysize']
    dx = torch.from_numpy(xyb).cuda()
    shape, npd = B.out_shape(img, dtype)
    tdt = {np.float32: torch.float32, np.uint8: torch.uint8, np.float16: torch.float16}[npd]
    out = torch.empty(shape, dtype=tdt, device="cuda")
    dimg = B.to_device(img, torch)
    t = ctx.submit_xyb(dx, xs, ys, dimg['vmap'], dimg['acmul'], dimg['sharpness'], lp, out, dtype)
    ctx.poll(t)
    return out.cpu().numpy()


def _oracle(img, xyb, p):
    """EPF then J.3 (then Gaborish) on the binary32 samples xyb (3, ys, xs)."""
    x = xyb.astype(np.float64)
    bh, bw = img['vmap'].shape
    padded = np.zeros((3, 8 * bh, 8 * bw))
    padded[:, :x.shape[1], :x.shape[2]] = x
    f = R.epf(x, img['vmap'], img['acmul'], img['sharpness'], p)
    out = R.qco(f, padded, img['vmap'], img['acmul'], p)
    if p.gab:
        out = R.gaborish(out, p)
    return f, out


def _excluded(img, xyb, p, gab):
    """Samples of the varblocks holding an EPF pixel that the decisions do
    not fix on the samples xyb (grown by one sample with Gaborish)."""
    from scipy.ndimage import binary_dilation
    amb, nd = undetermined(img, xyb.astype(np.float64), xyb, p, False)
    assert_rare(amb, nd, "J.3")
    m = np.zeros_like(amb)
    for code, bx, by in R.varblocks(img['vmap']):
        W, H = synth.SHAPE_WH[code]
        sl = (slice(8 * by, 8 * by + H), slice(8 * bx, 8 * bx + W))
        if amb[sl].any():
            m[sl] = True
    if gab:
        m = binary_dilation(m, structure=np.ones((3, 3), bool))
    assert m.mean() <= 0.02 or nd <= 2
    return m


@pytest.mark.parametrize("mix", ['mixed', 'dct8', 1, 2, 3, 12, 13, 14, 4, 5, 6, 9, 10, 11])
def test_qco_every_shape(B, ctx, mix):
    """J.3 after the EPF on identical input samples, per shape family."""
    img = synth.make_image(136, 104, 50 + (mix if isinstance(mix, int) else 99), mix=mix,
                           **ACTIVE)
    p, lp = _params(B)
    xyb = _gpu_xyb(B, ctx, img)
    f, want = _oracle(img, xyb, p)
    assert np.mean(np.abs(want - f) > 1e-7) > 0.05  # the constraint changed samples
    got = _staged(B, ctx, img, xyb, lp, XYB).transpose(2, 0, 1)
    m = _excluded(img, xyb, p, False)
    assert_xyb_close(np.where(m[None], want, got), want, abs_tol=5e-6, radius=32)


@pytest.mark.parametrize("xs,ys", [(9, 13), (131, 77), (300, 264)])
def test_qco_ragged_with_gaborish(B, ctx, xs, ys):
    """Ragged sizes (varblocks reaching past the image), then Gaborish."""
    img = synth.make_image(xs, ys, 7 * xs + ys, **ACTIVE)
    p, lp = _params(B, gab=True)
    xyb = _gpu_xyb(B, ctx, img)
    _, want = _oracle(img, xyb, p)
    got = _staged(B, ctx, img, xyb, lp, XYB).transpose(2, 0, 1)
    m = _excluded(img, xyb, p, True)
    assert_xyb_close(np.where(m[None], want, got), want, abs_tol=5e-6, radius=32)


def test_qco_limits(B, ctx):
    """A zero interval returns the EPF input bit for bit; an unbounded one
    returns the EPF output within the round trip of the transforms."""
    img = synth.make_image(200, 136, 77, **ACTIVE)
    xyb = _gpu_xyb(B, ctx, img)
    got0 = _staged(B, ctx, img, xyb, _params(B, mul=0.0)[1], XYB).transpose(2, 0, 1)
    np.testing.assert_array_equal(got0, xyb)
    p_inf, lp_inf = _params(B, mul=1e30)
    got_inf = _staged(B, ctx, img, xyb, lp_inf, XYB).transpose(2, 0, 1)
    epf_only = _staged(B, ctx, img, xyb, B.filter_defaults(epf=1), XYB).transpose(2, 0, 1)
    assert_xyb_close(got_inf, epf_only.astype(np.float64), abs_tol=5e-6, radius=32)


def test_qco_full_path_equals_staged(B, ctx):
    """Submit with EPF + J.3 + Gaborish == reconstruction to XYB, then the
    filter entry point; off when the EPF is off."""
    img = synth.make_image(264, 200, 21, **ACTIVE)
    _, lp = _params(B, gab=True)
    xyb = _gpu_xyb(B, ctx, img)
    staged = _staged(B, ctx, img, xyb, lp, F32)
    full = run(B, ctx, img, lp, F32)
    np.testing.assert_array_equal(full, staged)
    lp_off = B.filter_defaults(gab=1, qco=1)
    np.testing.assert_array_equal(run(B, ctx, img, lp_off, F32),
                                  run(B, ctx, img, B.filter_defaults(gab=1), F32))


def test_qco_only_on_submit_path(B, ctx):
    """Batches and the no-allocation entry point reject the constraint."""
    import torch
    img = synth.make_image(64, 64, 5)
    _, lp = _params(B)
    dimg = B.to_device(img, torch)
    out = torch.empty((64, 64, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(B.JxlrError) as e:
        ctx.batch([(dimg, lp, out, F32)], autotune=False)
    assert e.value.status == B.JXLR_EINVAL
    with pytest.raises(B.JxlrError) as e:
        B.run_noalloc(dimg, lp, out, F32)
    assert e.value.status == B.JXLR_EINVAL
