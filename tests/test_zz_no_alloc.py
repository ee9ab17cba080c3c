"""The entry point for callers that cannot allocate device memory.

jxl_recon_run_noalloc() serves callers that may not call cudaMalloc (their
device memory is owned and accounted by another allocator, or an
allocation's implicit synchronisation is not allowed where they run).  It
uses a fixed scratch array inside the library instead of allocating.  This
file is collected last so that, if it fails, a run that stops at the first
failure has already run every other test.  It passes both alone in a fresh
process (the first call does the per-device set-up) and after the others.
"""
import numpy as np
import pytest

from paper_1908_03565_gb300 import synth

pytestmark = pytest.mark.gpu

TOL01 = 1e-4   # the linear-RGB tolerance of the parity tests


def test_noalloc_matches_submit_on_two_calls_in_a_row():
    import torch
    assert torch.cuda.is_available()
    from paper_1908_03565_gb300 import binding as B
    B.load()
    stream = torch.cuda.Stream()
    cases = [((320, 200), 11), ((257, 129), 12)]   # the second reuses stale scratch
    with B.Context() as ctx:
        got, want = [], []
        for (xs, ys), seed in cases:
            img = synth.make_image(xs, ys, seed, y_dc_offset_q=200)
            dimg = B.to_device(img, torch)
            params = B.filter_defaults(epf=1, gab=1)
            ref = torch.empty((ys, xs, 3), dtype=torch.float32, device="cuda")
            t = ctx.submit(dimg, params, ref, B.OUT_F32_LINEAR, on_device=True)
            ctx.poll(t)
            out = torch.full((ys, xs, 3), float("nan"), dtype=torch.float32, device="cuda")
            B.run_noalloc(dimg, params, out, B.OUT_F32_LINEAR, stream=stream.cuda_stream)
            stream.synchronize()
            got.append(out.cpu().numpy())
            want.append(ref.cpu().numpy())
        for g, w in zip(got, want):
            assert np.isfinite(g).all()
            err = np.abs(np.clip(g, 0, 1) - np.clip(w, 0, 1)).max()
            assert err <= TOL01, err


def test_noalloc_rejects_oversized_images():
    import torch
    from paper_1908_03565_gb300 import binding as B
    img = {'xsize': 4096, 'ysize': 4096}
    dummy = torch.zeros(16, dtype=torch.int16, device="cuda")
    img['coeffs'] = torch.zeros((3, 8, 4096), dtype=torch.int16, device="cuda")
    for k in ('vmap', 'acmul', 'cfl', 'sharpness'):
        img[k] = dummy
    out = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(B.JxlrError) as e:
        B.run_noalloc(img, B.filter_defaults(epf=1, gab=1), out, B.OUT_F32_LINEAR,
                      out_stride=12 * 4096)
    assert e.value.status == B.JXLR_EINVAL
    assert "scratch" in str(e.value)
