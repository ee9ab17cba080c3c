"""The entry point for callers that cannot allocate device memory.

jxl_recon_run_noalloc() serves callers that may not call cudaMalloc (their
device memory is owned and accounted by another allocator, or an
allocation's implicit synchronisation is not allowed where they run).  It
uses a fixed scratch array inside the library instead of allocating.  This
file is collected last so that, if it fails, a run that stops at the first
failure has already run every other test.  It passes both alone in a fresh
process (the first call does the per-device set-up) and after the others.

Every filter combination runs the same arithmetic as the submit path: no
filter (the transform kernel writes the pixels), Gaborish alone (the
ordinary-load form of the Gaborish / colour kernel, bit-identical to the TMA
form the submit path takes), and the EPF with or without Gaborish (the
single-launch EPF, bit-identical to the block-list EPF).  So the outputs
must equal the submit path's bit for bit, for every output type and on two
calls in a row (the second reading scratch the first left behind).
"""
import numpy as np
import pytest

from paper_1908_03565_gb300 import synth

pytestmark = pytest.mark.gpu

# (epf, gab) combinations and output types
FILTERS = [(0, 0), (0, 1), (1, 0), (1, 1)]


def _dtypes(B):
    import torch
    return [(B.OUT_F32_LINEAR, torch.float32, float("nan")),
            (B.OUT_F16_LINEAR, torch.float16, float("nan")),
            (B.OUT_U8_SRGB, torch.uint8, 7)]


@pytest.mark.parametrize("epf,gab", FILTERS)
def test_noalloc_matches_submit_on_two_calls_in_a_row(epf, gab):
    import torch
    assert torch.cuda.is_available()
    from paper_1908_03565_gb300 import binding as B
    B.load()
    stream = torch.cuda.Stream()
    cases = [((320, 200), 11), ((257, 129), 12)]   # the second reuses stale scratch
    with B.Context() as ctx:
        for dt, tdt, fill in _dtypes(B):
            got, want = [], []
            for (xs, ys), seed in cases:
                img = synth.make_image(xs, ys, seed, y_dc_offset_q=200)
                dimg = B.to_device(img, torch)
                params = B.filter_defaults(epf=epf, gab=gab)
                ref = torch.empty((ys, xs, 3), dtype=tdt, device="cuda")
                ctx.poll(ctx.submit(dimg, params, ref, dt, on_device=True))
                out = torch.full((ys, xs, 3), fill, dtype=tdt, device="cuda")
                # the fill and the inputs were queued on the current stream
                stream.wait_stream(torch.cuda.current_stream())
                B.run_noalloc(dimg, params, out, dt, stream=stream.cuda_stream)
                stream.synchronize()
                got.append(out.cpu().numpy())
                want.append(ref.cpu().numpy())
            for g, w in zip(got, want):
                np.testing.assert_array_equal(g, w)


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
