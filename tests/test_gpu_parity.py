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
The EPF decides integers (guide bytes, block sigmas) from real numbers.  The
oracle takes them in real (FP64) arithmetic; the kernels take them in
binary32 from their own XYB.  A comparison therefore excludes, and counts,
the pixels whose output depends on a decision that the two take
differently: the oracle's real-number guide byte or block sigma on its
own samples against the kernels' binary32 evaluation on theirs (their XYB
output, evaluated here in correctly rounded binary32 as the kernels do),
and only where that decision can change a weight above the cut-off
(oracle.recon.epf_undetermined), spread by one sample where Gaborish
follows.  Both differences come from rounding (binary32 against real
arithmetic, and the transforms' binary32 error) at a threshold; every
other pixel is held to the bounds above.
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


def assert_filter_stage(img, xyb, got, p, gab, name):
    """The library's filter stage on its own binary32 XYB ``xyb`` against
    the oracle's J.2 (real decisions) + J.4 on the same samples: only the
    pixels whose decisions lie within the binary32 rounding of a threshold
    (and that matter) are excluded; they are counted and must be rare."""
    want = _oracle_filters(img, xyb, p)
    amb, nd = (undetermined(img, xyb.astype(np.float64), xyb, p, gab) if p.epf
               else (np.zeros(xyb.shape[1:], bool), 0))
    assert_rare(amb, nd, name)
    g = np.where(amb[None], want, got.transpose(2, 0, 1))
    assert_xyb_close(g, want, abs_tol=5e-6, radius=8)
    print(f"{name}: undetermined {amb.sum()} of {amb.size} pixels ({nd} decisions)")
    return amb


@pytest.mark.parametrize("epf,gab", [(True, False), (False, True), (True, True)])
@pytest.mark.parametrize("xs,ys", [(64, 64), (131, 77), (9, 13)])
def test_filter_stage_on_identical_samples(B, ctx, epf, gab, xs, ys):
    """J.2 + J.4 + L.2 on the same binary32 XYB on both sides: every decision
    the rounding of binary32 cannot move agrees with the real-number one,
    and the result is then within float rounding."""
    img = synth.make_image(xs, ys, 31 * xs + ys, y_dc_offset_q=200)
    p, lp = params_pair(B, epf=epf, gab=gab)
    xyb, got = _filters_on_gpu_xyb(B, ctx, img, lp, epf, gab, XYB)
    assert_filter_stage(img, xyb, got, p, gab, f"{xs}x{ys}")


@pytest.mark.parametrize("epf,gab", [(True, False), (True, True)])
@pytest.mark.parametrize("xs,ys,mix", [(136, 104, 'mixed'), (97, 61, 3), (64, 64, 14)])
def test_filter_stage_where_the_epf_acts(B, ctx, epf, gab, xs, ys, mix):
    """As above on inputs where most EPF weights survive the cut-off (small
    AC, smooth DC, AcMul 0.5): with the workload's coefficient statistics
    the EPF leaves almost every sample unchanged."""
    img = synth.make_image(xs, ys, 13 * xs + ys, mix=mix, coef_scale=2.0, acmul=0.5, dc='smooth')
    p, lp = params_pair(B, epf=epf, gab=gab)
    xyb, got = _filters_on_gpu_xyb(B, ctx, img, lp, epf, gab, XYB)
    assert np.mean(np.abs(R.epf(xyb.astype(np.float64), img['vmap'], img['acmul'],
                                img["sharpness"], p) - xyb) > 1e-7) > 0.03
    assert_filter_stage(img, xyb, got, p, gab, f"{xs}x{ys} {mix}")


def test_full_path_equals_staged_path(B, ctx):
    """Submit with filters == recon to XYB then the filter entry point."""
    img = synth.make_image(200, 136, 9, y_dc_offset_q=200)
    p, lp = params_pair(B, epf=True, gab=True)
    _, staged = _filters_on_gpu_xyb(B, ctx, img, lp, True, True, F32)
    full = run(B, ctx, img, lp, F32)
    np.testing.assert_array_equal(full, staged)


AMBIG_MAX = 1e-3           # largest share of pixels a comparison may exclude
# Largest share of RGB samples, at the workload's coefficient statistics, held
# to the relaxed bound: there the draft's default 32x8 / 8x32 matrices give XYB
# samples of 1e2..1e4, where binary32 cannot carry 1e-4 through L.2's cube
# (1.5-2.5% by the oracle's own count; at realistic magnitudes <= 1%)
WORKLOAD_RELAXED = 0.03


def decisions_binary32(img, x_gpu, p):
    """The guide bytes and block sigmas that the kernels take from their
    samples x_gpu (3, h, w), evaluated here step by step in correctly
    rounded binary32 arithmetic (numpy's float32 operations round as the
    kernels' __fsub_rn / __fmul_rn / __frcp_rn do): scaled = fl(fl(v - min)
    * scale) with binary32 parameters; guide = trunc(clamp(scaled, 0, 255));
    per block and channel fl(max - min) of scaled over the in-image
    samples, the largest over channels and over the varblock's blocks;
    sigma = trunc(min(fl(fl(min(range, range_max) * range_mul) * lut),
    fl(fl(1 / AcMul) * quant_mul), sigma_max)), at most 672.  This is the
    error model of the comparison, not a reference: the oracle decides in
    real arithmetic on its own samples."""
    f32 = np.float32
    im3 = (p.target_nits_div50 * 50.0 / 250.0) ** (1.0 / 3.0)
    x = np.asarray(x_gpu, f32)
    s = np.stack([(x[c] - f32((-0.03 if c == 0 else 0.0) * im3)) * f32(p.epf_scale[c])
                  for c in range(3)])
    g = np.trunc(np.clip(s, f32(0), f32(255))).astype(np.int64)
    rng = R.block_ranges(s, img['vmap'])            # binary32 differences, exact maxima
    bh, bw = rng.shape
    lut = np.asarray(p.epf_sharp_lut, f32)[img['sharpness'][:bh, :bw].astype(np.int64)]
    a = (np.minimum(rng.astype(f32), f32(p.epf_range_max)) * f32(p.epf_range_mul)) * lut
    q = (f32(1.0) / img['acmul'][:bh, :bw].astype(f32)) * f32(p.epf_quant_mul)
    sg = np.minimum(np.minimum(a, q), f32(p.epf_sigma_max))
    return g, np.clip(np.trunc(sg).astype(np.int64), 0, 672)


def undetermined(img, x_ref, x_gpu, p, gab, region=None):
    """Pixels (over ``region``) whose J.2 output depends on a decision that
    the real-number definition on the oracle's samples x_ref and the
    kernels' binary32 evaluation on their samples x_gpu take differently,
    where that decision can change a weight above the cut-off; grown by the
    Gaborish reach when ``gab``.  Returns the mask and the number of
    decisions (guide bytes and block sigmas) taken differently."""
    from scipy.ndimage import binary_dilation
    x_ref = np.asarray(x_ref, np.float64)
    g32, s32 = decisions_binary32(img, x_gpu, p)
    ndiff = (int(np.sum(g32 != R.guide(x_ref, p)))
             + int(np.sum(s32 != R.epf_sigma(x_ref, img['vmap'], img['acmul'], img['sharpness'], p))))
    u = R.epf_undetermined(x_ref, img['vmap'], img['acmul'], img['sharpness'], p,
                           region=region, guide_alt=g32, sigma_alt=s32)
    if gab:
        u = binary_dilation(u, structure=np.ones((3, 3), bool))
    return u, ndiff


def assert_rare(amb, ndiff, name):
    """Excluded pixels are rare: at most AMBIG_MAX of them, or, on images
    too small for a share to mean anything (one decision reaches up to
    ~150 pixels), at most 2 decisions taken differently."""
    assert amb.mean() <= AMBIG_MAX or (amb.size < 10 ** 6 and ndiff <= 2), (name, amb.mean(), ndiff)


def local_mag(*views, radius=8):
    """Largest |XYB| per channel within `radius` samples (the filter window)."""
    from scipy.ndimage import maximum_filter
    mag = np.max([np.abs(v) for v in views], axis=0)
    return maximum_filter(mag, size=(1, 2 * radius + 1, 2 * radius + 1), mode='nearest')


ERR_REL = 1e-6   # XYB error of the FP32 path relative to the local magnitude: 4x the
                 # largest measured (2.4e-7); a binary32 sum of products errs in
                 # proportion to the magnitude of its terms


def _through_l2(x, dx, p):
    """|d linear RGB01 / d XYB| . dx per output sample (central differences)."""
    tol = np.zeros(x.shape[1:] + (3,))
    for c in range(3):
        d = np.zeros_like(x)
        d[c] = 1e-6 * np.maximum(1.0, np.abs(x[c]))
        jac = (R.xyb_to_linear01(x + d, p) - R.xyb_to_linear01(x - d, p)) / (2 * d[c][..., None])
        tol += np.abs(jac) * dx[c][..., None]
    return tol


def rgb_tolerance(x, m, p, rel=LOCAL_REL):
    """Per-sample bound for linear RGB in [0, 1] at XYB samples x (3, h, w):
    TOL01 plus the XYB bound XYB_TOL + rel * m (m from local_mag) carried
    through L.2 by its Jacobian.  Where the XYB samples are O(1) the added
    term is small; it grows where the synthetic coefficients meet large
    default matrix entries and samples reach 1e2..1e4."""
    return TOL01 + _through_l2(x, XYB_TOL + rel * m, p)


def rgb_attainable(x, m, p, err_rel=ERR_REL):
    """The RGB error that the reconstruction can be held to at XYB samples x:
    err_rel * m (+ 1e-7) carried through L.2 (err_rel: the path's XYB error
    relative to the local magnitude).  Where it is within TOL01 the flat
    1e-4 bound applies."""
    return _through_l2(x, err_rel * m + 1e-7, p)


def assert_from_scratch(img, ref, gpu_xyb, f32, u8, p, name, region=None, relaxed_max=0.01,
                        xyb_rel=LOCAL_REL, err_rel=ERR_REL, f16=None):
    """The library's output against the oracle's, both from the coefficients.

    ``ref``: oracle.recon.reconstruct of ``img``; ``gpu_xyb``: the library's
    XYB before the filters (3, h, w); ``f32`` / ``u8``: its outputs over
    ``region`` (x0, y0, x1, y1; the whole image when None).  Bounds: the XYB
    bound before the filters everywhere; on every pixel the decisions fix
    (see the module docstring) u8 within +-1, and linear RGB within 1e-4
    wherever binary32 can attain it (rgb_attainable <= 1e-4), else within
    1e-4 plus the XYB bound carried through L.2 (rgb_tolerance).  The RGB
    samples of the second kind whose oracle value is not clamped away from
    [0, 1] by more than that bound are counted and must be at most
    ``relaxed_max`` of them (None: the caller checks the counts returned);
    excluded pixels must be rare (assert_rare).  Returns (excluded pixels,
    decisions taken differently, relaxed samples counted, samples).
    ``xyb_rel`` / ``err_rel``: the path's XYB bound and error model relative
    to the local magnitude (wider for the tensor-core path).  ``f16``: a
    float16 linear output checked instead of ``f32`` (the bound widened by
    half an f16 ulp of the oracle's value); ``f32`` and ``f16`` None: no
    linear output; ``u8`` None: no u8 output."""
    ys, xs = img['ysize'], img['xsize']
    if region is None:
        region = (0, 0, xs, ys)
    x0, y0, x1, y1 = region
    ref_xyb = ref['xyb_padded'][:, :ys, :xs]
    assert_xyb_close(gpu_xyb, ref_xyb, rel=xyb_rel)
    amb, nd = (undetermined(img, ref_xyb, gpu_xyb, p, p.gab, region) if p.epf
               else (np.zeros((y1 - y0, x1 - x0), bool), 0))
    ok = np.broadcast_to(~amb[..., None], (y1 - y0, x1 - x0, 3))
    rx = ref['xyb'][:, y0:y1, x0:x1]
    mag = local_mag(ref['xyb'], ref_xyb)[:, y0:y1, x0:x1]
    tol = rgb_tolerance(rx, mag, p, xyb_rel)
    plain = ok & (rgb_attainable(rx, mag, p, err_rel) <= TOL01)
    relaxed = ok & ~plain
    want01 = ref['rgb01'][y0:y1, x0:x1]
    bound = np.where(plain, TOL01, tol)
    if f32 is None and f16 is not None:   # float16 output: its rounding on top (half an ulp)
        f32 = f16.astype(np.float64)
        w16 = np.abs(np.clip(want01, 0, 1)).astype(np.float16)
        bound = bound + 0.5 * np.spacing(w16).astype(np.float64)
    err = (np.zeros(want01.shape) if f32 is None else
           np.abs(np.clip(f32, 0, 1) - np.clip(want01, 0, 1)))
    bad = (err > bound) & ok
    if bad.any():
        i = np.unravel_index(np.where(bad, err - bound, -1).argmax(), err.shape)
        raise AssertionError(f"{name}: {bad.sum()} RGB samples out of bound ({(bad & plain).sum()} "
                             f"plain); worst at {i}: err {err[i]:.3g} bound {bound[i]:.3g}")
    live = relaxed & (want01 >= -tol) & (want01 <= 1 + tol)
    d = (np.zeros(want01.shape, np.int64) if u8 is None else
         np.abs(u8.astype(np.int64) - R.srgb_u8(want01).astype(np.int64)))
    print(f"{name}: undetermined {amb.mean():.2e} of pixels ({nd} decisions); RGB samples held "
          f"to 1e-4: {plain.mean():.4f} (max err {err[plain].max():.2e}); to the relaxed bound and "
          f"not clamped away: {live.mean():.4f} (max err "
          f"{err[live].max() if live.any() else 0:.2e}); u8 max diff {d[ok].max()} "
          f"(over all pixels {d.max()})")
    assert d[ok].max() <= 1, name
    if relaxed_max is not None:
        assert live.mean() <= relaxed_max, (name, live.mean())
        assert_rare(amb, nd, name)
    return int(amb.sum()), nd, int(live.sum()), live.size


def test_mixed_statistics_from_scratch(B, ctx):
    """Mixed tiling, quant field, CfL, EPF + Gaborish, f32 and u8 outputs,
    against the oracle run from the coefficients."""
    img = synth.make_image(320, 200, 1001, y_dc_offset_q=200)
    p, lp = params_pair(B, epf=True, gab=True)
    ref = R.reconstruct(img, p)
    gpu_xyb = run(B, ctx, img, params_pair(B)[1], XYB).transpose(2, 0, 1)
    assert_from_scratch(img, ref, gpu_xyb, run(B, ctx, img, lp, F32),
                        run(B, ctx, img, lp, U8), p, "320x200", relaxed_max=WORKLOAD_RELAXED)
    # the filtered XYB itself, everywhere the decisions fix
    amb, _ = undetermined(img, ref['xyb_padded'][:, :200, :320], gpu_xyb, p, True)
    gx = run(B, ctx, img, lp, XYB).transpose(2, 0, 1)
    assert_xyb_close(np.where(amb[None], ref['xyb'], gx), ref['xyb'])


@pytest.mark.parametrize("stats", ['workload', 'active'])
def test_1920x1088_from_scratch(B, ctx, stats):
    """1920x1088 at the mixed statistics with both filters, whole image, f32
    and u8, against the oracle from the coefficients (and at statistics
    under which the EPF acts on most blocks)."""
    kw = {} if stats == 'workload' else dict(coef_scale=2.0, acmul=0.5, dc='smooth')
    img = synth.make_image(1920, 1088, 1000, **kw)
    p, lp = params_pair(B, epf=True, gab=True)
    ref = R.reconstruct(img, p)
    gpu_xyb = run(B, ctx, img, params_pair(B)[1], XYB).transpose(2, 0, 1)
    assert_from_scratch(img, ref, gpu_xyb, run(B, ctx, img, lp, F32),
                        run(B, ctx, img, lp, U8), p, f"1920x1088 {stats}",
                        relaxed_max=WORKLOAD_RELAXED if stats == 'workload' else 0.01)


def crop_input(img, x0, y0, x1, y1):
    """The inputs of the 64-aligned rectangle [x0, x1) x [y0, y1) as an image
    of its own (every varblock and CfL tile lies wholly inside it); its
    size reaches the source image's edge where the rectangle does."""
    assert x0 % 64 == 0 and y0 % 64 == 0
    Wp, Hp = img['coeffs'].shape[2], img['coeffs'].shape[1]
    x1, y1 = min(x1, Wp), min(y1, Hp)
    return {'xsize': min(x1, img['xsize']) - x0, 'ysize': min(y1, img['ysize']) - y0,
            'coeffs': img['coeffs'][:, y0:y1, x0:x1].copy(),
            'vmap': img['vmap'][y0 // 8:y1 // 8, x0 // 8:x1 // 8].copy(),
            'acmul': img['acmul'][y0 // 8:y1 // 8, x0 // 8:x1 // 8].copy(),
            'sharpness': img['sharpness'][y0 // 8:y1 // 8, x0 // 8:x1 // 8].copy(),
            'cfl': img['cfl'][y0 // 64:(y1 + 63) // 64, x0 // 64:(x1 + 63) // 64].copy()}


def test_4096_windows_from_scratch(B, ctx):
    """The 4096x4096 image of the throughput measurement (seed 2000, mixed
    statistics, EPF + Gaborish), one full-size run; the oracle from the
    coefficients on 64x64 windows (corners, edges, interior, random) of it,
    each from a 64-aligned crop with a margin of at least 64 samples (the
    filters reach 7 samples plus the window's varblocks) or the image edge."""
    import torch
    xs = ys = 4096
    img = synth.make_image(xs, ys, 2000)
    p, lp = params_pair(B, epf=True, gab=True)
    dimg = B.to_device(img, torch)
    outs = {}
    for dt, tdt in ((XYB, torch.float32), (F32, torch.float32), (U8, torch.uint8)):
        o = torch.empty((ys, xs, 3), dtype=tdt, device="cuda")
        ctx.poll(ctx.submit(dimg, params_pair(B)[1] if dt == XYB else lp, o, dt, on_device=True))
        outs[dt] = o.cpu().numpy()
    del dimg
    rng = np.random.default_rng(4096)
    wins = [(0, 0), (xs - 64, 0), (0, ys - 64), (xs - 64, ys - 64), (2048, 0), (0, 1344),
            (1984, 2048)] + [(int(64 * rng.integers(1, 62)), int(64 * rng.integers(1, 62)))
                             for _ in range(3)]
    tot = np.zeros(4, np.int64)
    for wx, wy in wins:
        cx0, cy0 = max(0, wx - 64), max(0, wy - 64)
        sub = crop_input(img, cx0, cy0, wx + 128, wy + 128)
        ref = R.reconstruct(sub, p)
        region = (wx - cx0, wy - cy0, wx - cx0 + 64, wy - cy0 + 64)
        gx = outs[XYB][cy0:cy0 + sub['ysize'], cx0:cx0 + sub['xsize']].transpose(2, 0, 1)
        tot += assert_from_scratch(sub, ref, gx, outs[F32][wy:wy + 64, wx:wx + 64],
                                   outs[U8][wy:wy + 64, wx:wx + 64], p,
                                   f"4096^2 window ({wx}, {wy})", region=region, relaxed_max=None)
    amb, nd, live, n = (int(v) for v in tot)
    print(f"4096^2 windows: undetermined {amb} of {n // 3} pixels ({nd} decisions), relaxed "
          f"samples not clamped away {live / n:.4f}")
    assert live / n <= WORKLOAD_RELAXED
    assert amb / (n // 3) <= AMBIG_MAX or nd <= 2


def _tiled_image(base, xs, ys):
    """base (a square image whose side is a multiple of 64) repeated to cover
    xs x ys: every varblock and CfL tile of base stays whole, so the result
    is a well-formed image whose every 64-aligned crop is one base would give
    at the same place modulo its side."""
    s = base['xsize']
    assert base['ysize'] == s and s % 64 == 0
    wp, hp = (xs + 7) // 8 * 8, (ys + 7) // 8 * 8
    assert hp % 32 == 0   # the last row of varblocks whole
    nx, ny = -(-wp // s), -(-hp // s)
    col = np.tile(base['coeffs'], (1, ny, 1))[:, :hp]
    coeffs = np.empty((3, hp, wp), np.int16)
    for j in range(nx):
        w = min(s, wp - j * s)
        coeffs[:, :, j * s:j * s + w] = col[:, :, :w]
    del col

    def per_block(a, k):
        return np.ascontiguousarray(np.tile(a, (ny, nx) + (1,) * (a.ndim - 2))[:hp // k, :wp // k])
    return {'xsize': xs, 'ysize': ys, 'coeffs': coeffs, 'vmap': per_block(base['vmap'], 8),
            'acmul': per_block(base['acmul'], 8), 'sharpness': per_block(base['sharpness'], 8),
            'cfl': per_block(base['cfl'], 64)}


def test_widest_image_past_2e31_samples(B, ctx):
    """The largest width the library takes (65536) at 10941 rows: 717 Mpx,
    2.15 G samples per planar image, so sample offsets in the third plane
    and in the interleaved outputs pass 2^31 (and byte offsets of the f32
    output 2^32).  The input repeats a 2048x2048 image of the workload's
    statistics (seed 2000) so that it is made in seconds; EPF + Gaborish,
    XYB, f32 and u8 outputs.  The oracle from the coefficients on 64x64
    windows at the corners, across the repeat seams and in the last rows
    (ragged: 10941 is not a multiple of 8), as in the 4096^2 test."""
    import torch
    xs, ys = 65536, 10941
    img = _tiled_image(synth.make_image(2048, 2048, 2000), xs, ys)
    p, lp = params_pair(B, epf=True, gab=True)
    wins = [(0, 0), (xs - 64, 0), (0, 10880), (xs - 64, 10880), (32768 - 64, 10880),
            (2048 - 64, 2048 - 64), (xs - 2048, 8192), (40960, 6144)]
    outs = {}
    dimg = B.to_device(img, torch)
    for dt, tdt in ((XYB, torch.float32), (F32, torch.float32), (U8, torch.uint8)):
        o = torch.empty((ys, xs, 3), dtype=tdt, device="cuda")
        ctx.poll(ctx.submit(dimg, params_pair(B)[1] if dt == XYB else lp, o, dt, on_device=True))
        if dt == XYB:   # the windows' crops (margin 64)
            outs[dt] = {w: o[max(0, w[1] - 64):w[1] + 128, max(0, w[0] - 64):w[0] + 128].cpu().numpy()
                        for w in wins}
        else:
            outs[dt] = {w: o[w[1]:w[1] + 64, w[0]:w[0] + 64].cpu().numpy() for w in wins}
        del o
    del dimg
    torch.cuda.empty_cache()
    tot = np.zeros(4, np.int64)
    for wx, wy in wins:
        cx0, cy0 = max(0, wx - 64), max(0, wy - 64)
        sub = crop_input(img, cx0, cy0, wx + 128, wy + 128)
        ref = R.reconstruct(sub, p)
        h, w = min(64, ys - wy), min(64, xs - wx)
        region = (wx - cx0, wy - cy0, wx - cx0 + w, wy - cy0 + h)
        gx = outs[XYB][(wx, wy)][:sub['ysize'], :sub['xsize']].transpose(2, 0, 1)
        assert gx.shape[1:] == (sub['ysize'], sub['xsize'])
        tot += assert_from_scratch(sub, ref, gx, outs[F32][(wx, wy)], outs[U8][(wx, wy)], p,
                                   f"65536x10941 window ({wx}, {wy})", region=region,
                                   relaxed_max=None)
    amb, nd, live, n = (int(v) for v in tot)
    print(f"65536x10941 windows: undetermined {amb} of {n // 3} pixels ({nd} decisions), "
          f"relaxed samples not clamped away {live / n:.4f}")
    assert live / n <= WORKLOAD_RELAXED
    assert amb / (n // 3) <= AMBIG_MAX or nd <= 2


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
