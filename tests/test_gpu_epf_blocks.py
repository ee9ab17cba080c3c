"""The block-list J.2 kernel of the submit and batch paths against the
single-launch EPF kernel of the no-allocation entry point, and its block
count.

Both kernels form every weight and every weighted sum in the same order, so
their results must agree bit for bit; the block-sparse one only skips the
patch sums of the 8x8 blocks whose sigma is below 16 (J.2.4: their samples
pass through) and copies those blocks instead.
"""
import numpy as np
import pytest

from oracle import recon as R
from paper_1908_03565_gb300 import synth
from test_gpu_parity import (B, XYB, F32, U8, params_pair, run,  # noqa: F401
                             _filters_on_gpu_xyb, assert_filter_stage, decisions_binary32)

pytestmark = pytest.mark.gpu

# Statistics under which the EPF changes most blocks (small AC, smooth DC,
# AcMul 0.5) and those of the throughput workload (most weights cut off).
ACTIVE = dict(coef_scale=2.0, acmul=0.5, dc='smooth')


@pytest.fixture(scope="module")
def tctx(B):
    c = B.Context(max_slots=2, timing=True)
    yield c
    c.close()


def _fused(B, ctx, img, lp, dtype):
    """The same request through the no-allocation entry point (the
    single-launch EPF)."""
    import torch
    dimg = B.to_device(img, torch)
    shape, npd = B.out_shape(img, dtype)
    tdt = {np.float32: torch.float32, np.float16: torch.float16, np.uint8: torch.uint8}[npd]
    out = torch.full(shape, 7, dtype=tdt, device="cuda")
    torch.cuda.synchronize()
    B.run_noalloc(dimg, lp, out, dtype)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _batch(B, ctx, img, lp, dtype):
    """The same request through a one-image batch."""
    import torch
    dimg = B.to_device(img, torch)
    shape, npd = B.out_shape(img, dtype)
    tdt = {np.float32: torch.float32, np.float16: torch.float16, np.uint8: torch.uint8}[npd]
    out = torch.full(shape, 7, dtype=tdt, device="cuda")
    b = ctx.batch([(dimg, lp, out, dtype)], autotune=False)
    stream = torch.cuda.Stream()
    for _ in range(2):   # replays restart the block lists
        b.launch(stream.cuda_stream)
    stream.synchronize()
    b.close()
    return out.cpu().numpy()


@pytest.mark.parametrize("xs,ys,stats", [(9, 13, 'active'), (33, 17, 'active'),
                                         (97, 61, 'active'), (300, 264, 'active'),
                                         (520, 264, 'workload'), (131, 77, 'workload')])
@pytest.mark.parametrize("gab", [False, True])
def test_block_kernel_equals_single_launch(B, tctx, xs, ys, stats, gab):
    kw = ACTIVE if stats == 'active' else {}
    img = synth.make_image(xs, ys, 5 * xs + ys, **kw)
    _, lp = params_pair(B, epf=True, gab=gab)
    for dtype in (XYB, F32, U8):
        want = _fused(B, tctx, img, lp, dtype)
        np.testing.assert_array_equal(run(B, tctx, img, lp, dtype), want)
        np.testing.assert_array_equal(_batch(B, tctx, img, lp, dtype), want)


def test_block_kernel_many_groups_per_warp(B, tctx):
    """A size where every persistent warp of k_epf_work takes several groups
    of listed blocks (about 21,000 blocks filtered, 2 per group)."""
    img = synth.make_image(2048, 1088, 77, **ACTIVE)
    _, lp = params_pair(B, epf=True, gab=True)
    want = _fused(B, tctx, img, lp, F32)
    np.testing.assert_array_equal(run(B, tctx, img, lp, F32), want)
    np.testing.assert_array_equal(_batch(B, tctx, img, lp, F32), want)


def _count_and_sigma(B, ctx, img, lp):
    import torch
    dimg = B.to_device(img, torch)
    shape, _ = B.out_shape(img, F32)
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    t = ctx.submit(dimg, lp, out, F32, on_device=True)
    ctx.poll(t)
    return ctx.epf_stats(t)


@pytest.mark.parametrize("xs,ys,stats", [(300, 264, 'active'), (520, 264, 'workload'),
                                         (33, 17, 'active')])
def test_block_count(B, tctx, xs, ys, stats):
    """The filtered blocks are those with sigma >= 16: on the GPU's own XYB
    samples the count equals that of the binary32 evaluation of J.2.4 and
    lies between those of the real-number and binary32 sigmas (equal unless
    a block's sigma sits at 16 within binary32 rounding)."""
    kw = ACTIVE if stats == 'active' else {}
    img = synth.make_image(xs, ys, 7 * xs + ys, **kw)
    p, lp = params_pair(B, epf=True, gab=True)
    xyb = run(B, tctx, img, params_pair(B)[1], XYB).transpose(2, 0, 1)
    _, s32 = decisions_binary32(img, xyb, p)
    _, _, s_lo, s_hi = R.epf_decision_bounds(xyb.astype(np.float64), img['vmap'], img['acmul'],
                                             img['sharpness'], p, sigma_alt=s32)
    ms, n = _count_and_sigma(B, tctx, img, lp)
    assert n == int(np.sum(s32 >= 16))
    assert int(np.sum(s_lo >= 16)) <= n <= int(np.sum(s_hi >= 16))
    assert int(np.sum(s_hi >= 16)) - int(np.sum(s_lo >= 16)) <= max(1, s_lo.size // 1000)
    assert 0 < n < s_lo.size
    assert ms > 0


def test_all_blocks_pass(B, tctx):
    """sigma_max below 16: no block is filtered, and the output is that of
    Gaborish alone."""
    img = synth.make_image(200, 136, 91, **ACTIVE)
    lp = B.filter_defaults(epf=1, gab=1, epf_sigma_max=15)
    ms, n = _count_and_sigma(B, tctx, img, lp)
    assert n == 0
    np.testing.assert_array_equal(run(B, tctx, img, lp, F32),
                                  run(B, tctx, img, B.filter_defaults(gab=1), F32))
    np.testing.assert_array_equal(run(B, tctx, img, lp, F32), _fused(B, tctx, img, lp, F32))


def test_no_epf_stats_without_the_filter(B, tctx):
    ms, n = _count_and_sigma(B, tctx, synth.make_image(64, 64, 3), B.filter_defaults(gab=1))
    assert (ms, n) == (0.0, 0)


def test_exact_clamp_variant(B, tctx):
    """Parameters under which Weight()'s clamp of sad at 507 can keep a weight
    above the cut-off (cut-off 0.001, sigma up to 672): the kernels' exact-clamp
    variant, block-list == single launch == batch, and the filter stage
    against the oracle on the same binary32 XYB."""
    kw = dict(epf_weight_min=0.001, epf_sigma_max=672, epf_quant_mul=1000.0)
    img = synth.make_image(264, 200, 95, **ACTIVE)
    lp = B.filter_defaults(epf=1, gab=1, **kw)
    for dtype in (XYB, F32):
        want = _fused(B, tctx, img, lp, dtype)
        np.testing.assert_array_equal(run(B, tctx, img, lp, dtype), want)
        np.testing.assert_array_equal(_batch(B, tctx, img, lp, dtype), want)
    p = R.Params(epf=True, **kw)
    lp1 = B.filter_defaults(epf=1, **kw)
    xyb, got = _filters_on_gpu_xyb(B, tctx, img, lp1, True, False, XYB)
    sig = R.epf_sigma(xyb.astype(np.float64), img['vmap'], img['acmul'], img['sharpness'], p)
    assert (sig >= 202).any()          # the clamp variant's sigma range is reached
    assert_filter_stage(img, xyb, got, p, False, "exact-clamp variant")
