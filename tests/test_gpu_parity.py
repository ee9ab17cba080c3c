"""Parity of the CUDA library (through its C ABI) with the FP64 oracle.

Tolerances (written here; derived from binary32 arithmetic):
  * linear RGB in [0, 1]: max |gpu - oracle| <= 1e-4 on clamp(., 0, 1);
  * 8-bit sRGB: every sample within +-1 of the oracle's;
  * f16 output: <= half an f16 ulp of the value + 1e-4;
  * XYB samples (before or after the filters): <= XYB_TOL + LOCAL_REL * m,
    m the largest |sample| of that channel within LOCAL_R samples.  Binary32
    sums of products err in proportion to the magnitude of their terms; the
    draft's default 32x8 / 8x32 matrices make some samples reach ~1e4, so an
    absolute bound alone does not describe FP32 arithmetic there.
The EPF decides integers (guide bytes, sigma) from real numbers; the oracle
takes those decisions in binary32 like the kernels, so the filter stage is
compared on identical input samples (the GPU's own XYB).  From-scratch
comparisons exclude, and count, only pixels whose EPF window saw a guide
byte or sigma that differs between the two XYB images.
"""
import numpy as np
import pytest

from oracle import recon as R
from paper_1908_03565_gb300 import synth

pytestmark = pytest.mark.gpu

TOL01 = 1e-4
XYB_TOL = 2e-5
LOCAL_REL = 4e-6
LOCAL_R = 16


def assert_xyb_close(got, want, abs_tol=XYB_TOL, rel=LOCAL_REL, radius=LOCAL_R):
    """got, want: (3, h, w).  Element-wise |got - want| <= abs_tol + rel * m."""
    from scipy.ndimage import maximum_filter
    got = np.asarray(got, np.float64)
    m = maximum_filter(np.abs(want), size=(1, 2 * radius + 1, 2 * radius + 1), mode='nearest')
    tol = abs_tol + rel * m
    err = np.abs(got - want)
    bad = err > tol
    assert not bad.any(), (f"{bad.sum()} samples out of tolerance; worst excess at "
                           f"{np.unravel_index((err - tol).argmax(), err.shape)}: "
                           f"err {err.flat[(err - tol).argmax()]:.3g} tol {tol.flat[(err - tol).argmax()]:.3g}")
    return float(err.max())

F32, F16, U8, XYB = 0, 1, 2, 3


def params_pair(B, epf=False, gab=False, kx_dc=0.0, kb_dc=0.0):
    """Matching oracle and library parameter sets (draft defaults)."""
    p = R.Params(epf=epf, gab=gab, kx_dc=kx_dc, kb_dc=kb_dc)
    lp = B.filter_defaults(epf=int(epf), gab=int(gab))
    return p, lp


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test without CUDA")
    from paper_1908_03565_gb300 import binding
    binding.load()
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.Context(max_slots=2)
    yield c
    c.close()


def run(B, ctx, img, lp, dtype, device_io=True, kx_dc=0.0, kb_dc=0.0):
    import torch
    shape, npd = B.out_shape(img, dtype)
    if device_io:
        dimg = B.to_device(img, torch)
        tdt = {np.float32: torch.float32, np.float16: torch.float16, np.uint8: torch.uint8}[npd]
        out = torch.full(shape, 7, dtype=tdt, device="cuda")
        t = ctx.submit(dimg, lp, out, dtype, on_device=True, kx_dc=kx_dc, kb_dc=kb_dc)
        ctx.poll(t)
        return out.cpu().numpy()
    out = np.full(shape, 7, dtype=npd)
    t = ctx.submit(img, lp, out, dtype, on_device=False, out_on_device=False,
                   kx_dc=kx_dc, kb_dc=kb_dc)
    ctx.poll(t)
    return out


def oracle_xyb(img, p):
    xyb = R.reconstruct_xyb(img['coeffs'], img['vmap'], img['acmul'], img['cfl'], p)
    return xyb[:, :img['ysize'], :img['xsize']]


def check_rgb01(got, want, tol=TOL01):
    err = np.abs(np.clip(got.astype(np.float64), 0, 1) - np.clip(want, 0, 1))
    assert err.max() <= tol, f"max err {err.max():.3g} at {np.unravel_index(err.argmax(), err.shape)}"
    return err.max()


def check_u8(got, want01):
    want = R.srgb_u8(want01).astype(np.int64)
    d = np.abs(got.astype(np.int64) - want)
    assert d.max() <= 1, f"u8 off by {d.max()} at {np.unravel_index(d.argmax(), d.shape)}"


# ---------------------------------------------------------------------------
# linear path: dequantisation, CfL, LLF, transforms, colour
# ---------------------------------------------------------------------------
def test_dct8_256_no_filters(B, ctx):
    """256x256, all DCT8, AcMul 1, no CfL, no filters, f32 output."""
    img = synth.make_image(256, 256, 0, mix='dct8', acmul=1.0, cfl=False)
    p, lp = params_pair(B)
    want_xyb = oracle_xyb(img, p)
    got_xyb = run(B, ctx, img, lp, XYB)
    assert_xyb_close(got_xyb.transpose(2, 0, 1), want_xyb)
    want = R.xyb_to_linear01(want_xyb, p)
    check_rgb01(run(B, ctx, img, lp, F32), want)
    check_u8(run(B, ctx, img, lp, U8), want)


@pytest.mark.parametrize("code", list(range(15)))
def test_every_shape(B, ctx, code):
    """An image tiled with one varblock shape (DCT8 where it does not fit),
    with quant field and CfL drawn as in the mixed workload."""
    img = synth.make_image(72, 80, 100 + code, mix=code, y_dc_offset_q=200)
    p, lp = params_pair(B)
    want_xyb = oracle_xyb(img, p)
    got = run(B, ctx, img, lp, XYB).transpose(2, 0, 1)
    assert_xyb_close(got, want_xyb)


@pytest.mark.parametrize("xs,ys", [(1, 1), (7, 9), (8, 8), (33, 17), (95, 64), (200, 136)])
def test_ragged_sizes_all_outputs(B, ctx, xs, ys):
    img = synth.make_image(xs, ys, xs * 1000 + ys, y_dc_offset_q=200)
    p, lp = params_pair(B)
    want_xyb = oracle_xyb(img, p)
    assert_xyb_close(run(B, ctx, img, lp, XYB).transpose(2, 0, 1), want_xyb)
    want = R.xyb_to_linear01(want_xyb, p)
    check_rgb01(run(B, ctx, img, lp, F32), want)
    check_u8(run(B, ctx, img, lp, U8), want)
    h = np.clip(run(B, ctx, img, lp, F16).astype(np.float64), 0, 1)
    w01 = np.clip(want, 0, 1)
    tol = w01 * 2.0 ** -11 + TOL01        # half an f16 ulp on [0, 1] + 1e-4
    assert np.all(np.abs(h - w01) <= tol)


def test_dc_cfl_factors(B, ctx):
    img = synth.make_image(64, 48, 77, y_dc_offset_q=200)
    p, lp = params_pair(B, kx_dc=0.25, kb_dc=0.9)
    want = oracle_xyb(img, p)
    got = run(B, ctx, img, lp, XYB, kx_dc=0.25, kb_dc=0.9).transpose(2, 0, 1)
    assert_xyb_close(got, want)


def test_host_io_equals_device_io(B, ctx):
    img = synth.make_image(150, 70, 5, y_dc_offset_q=200)
    for epf, gab in ((False, False), (True, True)):
        _, lp = params_pair(B, epf=epf, gab=gab)
        a = run(B, ctx, img, lp, F32, device_io=True)
        b = run(B, ctx, img, lp, F32, device_io=False)
        np.testing.assert_array_equal(a, b)


# ---------------------------------------------------------------------------
# filters: EPF and Gaborish
# ---------------------------------------------------------------------------
def _filters_on_gpu_xyb(B, ctx, img, lp, epf, gab, dtype=F32):
    """Runs the filter + colour stage of the library on the GPU's own XYB."""
    import torch
    xs, ys = img['xsize'], img['ysize']
    _, lp0 = params_pair(B)
    xyb = run(B, ctx, img, lp0, XYB).transpose(2, 0, 1).copy()      # (3, ys, xs) f32
    dx = torch.from_numpy(xyb).cuda()
    shape, npd = B.out_shape(img, dtype)
    tdt = {np.float32: torch.float32, np.float16: torch.float16, np.uint8: torch.uint8}[npd]
    out = torch.empty(shape, dtype=tdt, device="cuda")
    dimg = B.to_device(img, torch)
    t = ctx.submit_xyb(dx, xs, ys, dimg['vmap'], dimg['acmul'], dimg['sharpness'], lp, out, dtype)
    ctx.poll(t)
    return xyb, out.cpu().numpy()


def _oracle_filters(img, xyb, p, region=None):
    x = xyb.astype(np.float64)
    if p.epf:
        x = R.epf(x, img['vmap'], img['acmul'], img['sharpness'], p)
    if p.gab:
        x = R.gaborish(x, p)
    return x


@pytest.mark.parametrize("epf,gab", [(True, False), (False, True), (True, True)])
@pytest.mark.parametrize("xs,ys", [(64, 64), (131, 77), (9, 13)])
def test_filter_stage_on_identical_samples(B, ctx, epf, gab, xs, ys):
    """J.2 + J.4 + L.2 on the same binary32 XYB on both sides: every integer
    decision agrees, so the result is within float rounding."""
    img = synth.make_image(xs, ys, 31 * xs + ys, y_dc_offset_q=200)
    p, lp = params_pair(B, epf=epf, gab=gab)
    xyb, got = _filters_on_gpu_xyb(B, ctx, img, lp, epf, gab, XYB)
    want = _oracle_filters(img, xyb, p)
    assert_xyb_close(got.transpose(2, 0, 1), want, abs_tol=5e-6, radius=8)


@pytest.mark.parametrize("epf,gab", [(True, False), (True, True)])
@pytest.mark.parametrize("xs,ys,mix", [(136, 104, 'mixed'), (97, 61, 3), (64, 64, 14)])
def test_filter_stage_where_the_epf_acts(B, ctx, epf, gab, xs, ys, mix):
    """As above on inputs where most EPF weights survive the cut-off (small
    AC, smooth DC, AcMul 0.5): with the workload's coefficient statistics
    the EPF leaves almost every sample unchanged."""
    img = synth.make_image(xs, ys, 13 * xs + ys, mix=mix, coef_scale=2.0, acmul=0.5, dc='smooth')
    p, lp = params_pair(B, epf=epf, gab=gab)
    xyb, got = _filters_on_gpu_xyb(B, ctx, img, lp, epf, gab, XYB)
    want = _oracle_filters(img, xyb, p)
    assert np.mean(np.abs(R.epf(xyb.astype(np.float64), img['vmap'], img['acmul'],
                                img["sharpness"], p) - xyb) > 1e-7) > 0.03
    assert_xyb_close(got.transpose(2, 0, 1), want, abs_tol=5e-6, radius=8)


def test_full_path_equals_staged_path(B, ctx):
    """Submit with filters == recon to XYB then the filter entry point."""
    img = synth.make_image(200, 136, 9, y_dc_offset_q=200)
    p, lp = params_pair(B, epf=True, gab=True)
    _, staged = _filters_on_gpu_xyb(B, ctx, img, lp, True, True, F32)
    full = run(B, ctx, img, lp, F32)
    np.testing.assert_array_equal(full, staged)


def _ambiguous_mask(img, xyb_a, xyb_b, p):
    """Pixels whose EPF+Gaborish window (x -5..+6, y -5..+5) contains a guide
    byte or a block sigma that differs between two XYB images."""
    ga, gb = R.guide(xyb_a, p), R.guide(xyb_b, p)
    diff = np.any(ga != gb, axis=0)
    sa = R.epf_sigma(xyb_a, img['vmap'], img['acmul'], img['sharpness'], p)
    sb = R.epf_sigma(xyb_b, img['vmap'], img['acmul'], img['sharpness'], p)
    sd = np.repeat(np.repeat(sa != sb, 8, 0), 8, 1)[:diff.shape[0], :diff.shape[1]]
    bad = diff | sd
    out = np.zeros_like(bad)
    ys, xs = bad.shape
    for dy in range(-5, 6):
        for dx in range(-5, 7):
            out |= bad[R.mirror(np.arange(ys)[:, None] - dy, ys), R.mirror(np.arange(xs)[None, :] - dx, xs)]
    return out


def local_mag(*views, radius=8):
    """Largest |XYB| per channel within `radius` samples (the filter window)."""
    from scipy.ndimage import maximum_filter
    mag = np.max([np.abs(v) for v in views], axis=0)
    return maximum_filter(mag, size=(1, 2 * radius + 1, 2 * radius + 1), mode='nearest')


def rgb_tolerance(x, m, p):
    """Per-pixel bound for linear RGB in [0, 1] at XYB samples x (3, h, w):
    TOL01 plus the XYB bound XYB_TOL + LOCAL_REL * m (m from local_mag)
    carried through L.2 by its Jacobian (central differences).  Where the
    XYB samples are O(1) the added term is below 1e-5; it grows only where
    the synthetic coefficients meet large default matrix entries and samples
    reach 1e2..1e4, as binary32 arithmetic does."""
    dx = XYB_TOL + LOCAL_REL * m
    tol = np.full(x.shape[1:] + (3,), TOL01)
    for c in range(3):
        d = np.zeros_like(x)
        d[c] = 1e-6 * np.maximum(1.0, np.abs(x[c]))
        jac = (R.xyb_to_linear01(x + d, p) - R.xyb_to_linear01(x - d, p)) / (2 * d[c][..., None])
        tol += np.abs(jac) * dx[c][..., None]
    return tol


def test_mixed_statistics_from_scratch(B, ctx):
    """Mixed tiling, quant field, CfL, EPF + Gaborish, f32 and u8 outputs,
    against the oracle run from the coefficients."""
    img = synth.make_image(320, 200, 1001, y_dc_offset_q=200)
    p, lp = params_pair(B, epf=True, gab=True)
    ref = R.reconstruct(img, p)
    ref_xyb = ref['xyb_padded'][:, :200, :320]
    gpu_xyb = run(B, ctx, img, params_pair(B)[1], XYB).transpose(2, 0, 1)
    assert_xyb_close(gpu_xyb, ref_xyb)
    amb = _ambiguous_mask(img, ref_xyb, gpu_xyb.astype(np.float64), p)
    tol = rgb_tolerance(ref['xyb'], local_mag(ref['xyb'], ref_xyb), p)
    got = run(B, ctx, img, lp, F32)
    err = np.abs(np.clip(got, 0, 1) - np.clip(ref['rgb01'], 0, 1))
    ok = ~amb
    assert np.all((err <= tol)[ok])
    plain = ok[..., None] & (tol <= 1.1 * TOL01)
    assert err[plain].max() <= TOL01
    assert amb.mean() < 0.25, amb.mean()
    u8 = run(B, ctx, img, lp, U8).astype(np.int64)
    d = np.abs(u8 - R.srgb_u8(ref['rgb01']).astype(np.int64))
    assert d[plain].max() <= 1
    # the filtered XYB itself, everywhere that no decision differs
    gx = run(B, ctx, img, lp, XYB).transpose(2, 0, 1)
    ok = ~amb
    from scipy.ndimage import maximum_filter
    m = maximum_filter(np.abs(ref['xyb']), size=(1, 17, 17), mode='nearest')
    e = np.abs(gx - ref['xyb'])
    assert np.all((e <= XYB_TOL + LOCAL_REL * m)[:, ok])
    print(f"ambiguous {amb.mean():.4f}, pixels at the plain 1e-4 bound "
          f"{plain.mean():.4f}, max err there {err[plain].max():.2e}")


def test_mixed_1920x1088_sampled(B, ctx):
    """1920x1088 at the mixed statistics with both filters: the linear part
    everywhere; the filters on windows (corners, edges, interior) computed
    by the oracle from the GPU's XYB."""
    xs, ys = 1920, 1088
    img = synth.make_image(xs, ys, 1000)
    p, lp = params_pair(B, epf=True, gab=True)
    gpu_xyb = run(B, ctx, img, params_pair(B)[1], XYB).transpose(2, 0, 1)
    want = R.reconstruct_xyb(img['coeffs'], img['vmap'], img['acmul'], img['cfl'], p)
    assert_xyb_close(gpu_xyb, want[:, :ys, :xs])
    got = run(B, ctx, img, lp, F32)
    x64 = gpu_xyb.astype(np.float64)
    mag = local_mag(x64)
    for (x0, y0) in [(0, 0), (xs - 40, 0), (0, ys - 40), (xs - 40, ys - 40), (960, 544)]:
        region = (x0, y0, x0 + 40, y0 + 40)
        e = R.epf(x64, img['vmap'], img['acmul'], img['sharpness'], p,
                  region=(max(0, x0 - 1), max(0, y0 - 1), min(xs, x0 + 41), min(ys, y0 + 41)))
        xf = _gab_window(x64, e, region, p, img)
        ref = R.xyb_to_linear01(xf, p)
        tol = rgb_tolerance(xf, mag[:, y0:y0 + 40, x0:x0 + 40], p)
        err = np.abs(np.clip(got[y0:y0 + 40, x0:x0 + 40], 0, 1) - np.clip(ref, 0, 1))
        assert np.all(err <= tol), (x0, y0, float((err - tol).max()))


def _gab_window(x64, e, region, p, img):
    """Gaborish of the EPF output on `region`, given the EPF output `e` on the
    region grown by one sample (clipped to the image)."""
    xs, ys = x64.shape[2], x64.shape[1]
    x0, y0, x1, y1 = region
    ex0, ey0 = max(0, x0 - 1), max(0, y0 - 1)
    out = np.zeros((3, y1 - y0, x1 - x0))
    for c in range(3):
        w1, w2 = p.gab_w1[c], p.gab_w2[c]
        n = 1 + 4 * w1 + 4 * w2
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                wt = (1.0, w1, w2)[abs(dx) + abs(dy)] / n
                yy = R.mirror(np.arange(y0, y1)[:, None] + dy, ys) - ey0
                xx = R.mirror(np.arange(x0, x1)[None, :] + dx, xs) - ex0
                out[c] += wt * e[c][yy, xx]
    return out


# ---------------------------------------------------------------------------
# boundary behaviour
# ---------------------------------------------------------------------------
def test_invalid_maps_rejected(B, ctx):
    import torch
    img = synth.make_image(64, 64, 3)
    _, lp = params_pair(B)
    bad = dict(img)
    vm = img['vmap'].copy()
    vm[0, 0] = 5          # DCT32 at (0,0) overlapping whatever is there
    vm[1, 1] = 0
    bad['vmap'] = vm
    out = np.zeros((64, 64, 3), np.float32)
    with pytest.raises(B.JxlrError) as e:
        ctx.submit(bad, lp, out, F32, on_device=False, out_on_device=False)
    assert e.value.status == B.JXLR_EINVAL
    # device inputs: reported by poll
    dimg = B.to_device(bad, torch)
    dout = torch.empty((64, 64, 3), dtype=torch.float32, device="cuda")
    t = ctx.submit(dimg, lp, dout, F32, on_device=True)
    with pytest.raises(B.JxlrError) as e:
        ctx.poll(t)
    assert e.value.status == B.JXLR_EINVAL
    vm2 = img['vmap'].copy()
    vm2[3, 3] = 16        # no such code
    bad['vmap'] = vm2
    dimg = B.to_device(bad, torch)
    t = ctx.submit(dimg, lp, dout, F32, on_device=True)
    with pytest.raises(B.JxlrError):
        ctx.poll(t)
    # the context still works
    assert np.isfinite(run(B, ctx, img, lp, F32)).all()


def test_dequant_override(B, ctx):
    """A caller matrix table replaces C.6.1.1's defaults."""
    from oracle import tables as T
    img = synth.make_image(64, 64, 8, y_dc_offset_q=200)
    p, lp = params_pair(B)
    tab = []
    for code in range(15):
        for c in range(3):
            tab.append(T.dequant_matrix(code, c).reshape(-1) * (1.5 if c == 1 else 0.75))
    tab = np.concatenate(tab).astype(np.float32)
    assert tab.size == 10560
    tab[~np.isfinite(tab)] = 1.0
    lp.dequant = tab.ctypes.data
    got = run(B, ctx, img, lp, XYB).transpose(2, 0, 1)
    orig = T.dequant_matrix
    try:
        T.dequant_matrix = lambda code, c: orig(code, c) * (1.5 if c == 1 else 0.75)
        want = oracle_xyb(img, p)
    finally:
        T.dequant_matrix = orig
    assert_xyb_close(got, want)
    bad = tab.copy()
    bad[100] = -1.0
    lp.dequant = bad.ctypes.data
    with pytest.raises(B.JxlrError):
        run(B, ctx, img, lp, XYB)
    lp.dequant = None


def test_hbm_cap_admission(B):
    img = synth.make_image(256, 256, 4)
    _, lp = params_pair(B, epf=True, gab=True)
    with B.Context(max_slots=1, hbm_cap_bytes=1 << 20) as c:
        out = np.zeros((256, 256, 3), np.float32)
        with pytest.raises(B.JxlrError) as e:
            c.submit(img, lp, out, F32, on_device=False, out_on_device=False)
        assert e.value.status == B.JXLR_ENOMEM
    with B.Context(max_slots=1) as c:
        out = np.zeros((256, 256, 3), np.float32)
        t = c.submit(img, lp, out, F32, on_device=False, out_on_device=False)
        with pytest.raises(B.JxlrError) as e:
            c.submit(img, lp, out, F32, on_device=False, out_on_device=False)
        assert e.value.status == B.JXLR_EBUSY
        c.poll(t)
        assert c.launch_count() >= 2
