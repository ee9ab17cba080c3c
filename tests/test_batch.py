"""Multi-image batches (one launch per kernel kind, CUDA-graph replay):
every image equals its per-image result."""
import numpy as np
import pytest

from paper_1908_03565_gb300 import synth

pytestmark = pytest.mark.gpu


def _jobs(B, torch, n=30, seed=7000):
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(n):
        xs, ys = (int(v) for v in np.exp(rng.uniform(np.log(8), np.log(700), 2)))
        img = B.to_device(synth.make_image(xs, ys, seed + i, y_dc_offset_q=200), torch)
        dtype = (B.OUT_U8_SRGB, B.OUT_F16_LINEAR, B.OUT_F32_LINEAR, B.OUT_F32_XYB)[i % 4]
        mode = i % 5
        params = B.filter_defaults(epf=int(mode in (0, 1, 2)), gab=int(mode in (0, 3)))
        shape, npd = B.out_shape(img, dtype)
        tdt = {np.float32: torch.float32, np.float16: torch.float16, np.uint8: torch.uint8}[npd]
        jobs.append((img, params, torch.zeros(shape, dtype=tdt, device="cuda"), dtype))
    return jobs


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_equals_per_image(autotune):
    import torch
    from paper_1908_03565_gb300 import binding as B
    jobs = _jobs(B, torch)
    with B.Context(max_slots=1) as ctx:
        want = []
        for img, params, out, dtype in jobs:
            t = ctx.submit(img, params, out, dtype, on_device=True)
            ctx.poll(t)
            want.append(out.cpu().numpy().copy())
            out.zero_()
        b = ctx.batch(jobs, autotune=autotune)
        info = b.info()
        assert info["images"] == len(jobs) and info["kernels_per_launch"] == 3
        # every scratch allows TMA tile loads: the untuned batch takes them;
        # the autotuner may choose either form (the same bits)
        assert info["filter_tma"] == 1 or autotune
        stream = torch.cuda.Stream()
        for rep in range(2):                       # graph replayed twice
            b.launch(stream.cuda_stream)
            stream.synchronize()
            for (img, params, out, dtype), w in zip(jobs, want):
                np.testing.assert_array_equal(out.cpu().numpy(), w)
                out.zero_()
        assert b.status() == 0
        b.close()


def test_batch_of_thin_images():
    """Images one pixel wide or high (every tile an edge tile, the ring
    mirrored on all sides) next to ordinary ones, with and without the EPF
    and Gaborish: the TMA tile loads of the batch equal the per-image results."""
    import torch
    from paper_1908_03565_gb300 import binding as B
    sizes = [(1, 1), (1, 37), (37, 1), (33, 2), (2, 45), (9, 13), (64, 40), (131, 77)]
    jobs = []
    for i, (xs, ys) in enumerate(sizes * 2):
        img = B.to_device(synth.make_image(xs, ys, 7300 + i), torch)
        dtype = (B.OUT_U8_SRGB, B.OUT_F32_LINEAR, B.OUT_F16_LINEAR)[i % 3]
        params = B.filter_defaults(epf=int(i < len(sizes)), gab=int(i % 4 != 1))
        shape, npd = B.out_shape(img, dtype)
        tdt = {np.float32: torch.float32, np.float16: torch.float16, np.uint8: torch.uint8}[npd]
        jobs.append((img, params, torch.zeros(shape, dtype=tdt, device="cuda"), dtype))
    with B.Context(max_slots=1) as ctx:
        want = []
        for img, params, out, dtype in jobs:
            ctx.poll(ctx.submit(img, params, out, dtype, on_device=True))
            want.append(out.cpu().numpy().copy())
            out.zero_()
        b = ctx.batch(jobs, autotune=False)
        assert b.info()["filter_tma"] == 1
        stream = torch.cuda.Stream()
        b.launch(stream.cuda_stream)
        stream.synchronize()
        for (img, params, out, dtype), w in zip(jobs, want):
            np.testing.assert_array_equal(out.cpu().numpy(), w)
        assert b.status() == 0
        b.close()


def test_batch_plain_loads_equal_per_image():
    """JXLR_BATCH_PLAIN_LOADS: the Gaborish / colour kernel of the batch
    with ordinary tile loads gives the per-image results too."""
    import torch
    from paper_1908_03565_gb300 import binding as B
    jobs = _jobs(B, torch, n=12, seed=7200)
    with B.Context(max_slots=1) as ctx:
        want = []
        for img, params, out, dtype in jobs:
            ctx.poll(ctx.submit(img, params, out, dtype, on_device=True))
            want.append(out.cpu().numpy().copy())
            out.zero_()
        b = ctx.batch(jobs, autotune=False, plain_loads=True)
        assert b.info()["filter_tma"] == 0
        stream = torch.cuda.Stream()
        b.launch(stream.cuda_stream)
        stream.synchronize()
        for (img, params, out, dtype), w in zip(jobs, want):
            np.testing.assert_array_equal(out.cpu().numpy(), w)
        assert b.status() == 0
        b.close()


def test_batch_rejects_bad_map():
    import torch
    from paper_1908_03565_gb300 import binding as B
    jobs = _jobs(B, torch, n=3, seed=7100)
    bad = dict(jobs[1][0])
    vm = bad['vmap'].clone()
    vm[0, 0] = 5      # a 32x32 varblock that overlaps its neighbours
    bad['vmap'] = vm
    jobs[1] = (bad,) + jobs[1][1:]
    with B.Context() as ctx:
        with pytest.raises(B.JxlrError) as e:
            ctx.batch(jobs, autotune=False)
        assert e.value.status == B.JXLR_EINVAL


def test_config3_batch_sample_against_oracle():
    """The 512-image batch of the throughput measurement as it is timed (512
    distinct images, sides log-uniform in [64, 2048] in multiples of 8, the
    workload's statistics, EPF + Gaborish, u8 sRGB and f16 linear outputs
    alternating, autotuned, one graph replay), checked against the oracle
    from the coefficients on a seeded 1% sample of its images: the whole
    image up to 320x320, else a 64x64 window at a seeded 64-aligned place
    (its oracle from a crop with a 64-sample margin).  The decisions are
    modelled on the XYB of the same image (the batch equals the per-image
    path bit for bit)."""
    import math
    import torch
    from oracle import recon as R
    from paper_1908_03565_gb300 import binding as B
    from test_gpu_parity import XYB, assert_from_scratch, crop_input, params_pair, run
    n_img, seed = 512, 3000
    rng = np.random.default_rng(seed)
    sides = (np.exp(rng.uniform(math.log(64), math.log(2048), size=(n_img, 2))) // 8 * 8).astype(int)
    imgs = [synth.make_image(int(x), int(y), seed + i) for i, (x, y) in enumerate(sides)]
    p, lp = params_pair(B, epf=True, gab=True)
    jobs = []
    for i, img in enumerate(imgs):
        dt, tdt = ((B.OUT_U8_SRGB, torch.uint8) if i % 2 == 0 else
                   (B.OUT_F16_LINEAR, torch.float16))
        out = torch.zeros((img['ysize'], img['xsize'], 3), dtype=tdt, device="cuda")
        jobs.append((B.to_device(img, torch), lp, out, dt))
    stream = torch.cuda.Stream()
    with B.Context(max_slots=1, stream=stream.cuda_stream) as ctx:
        b = ctx.batch(jobs, autotune=True)
        b.launch(stream.cuda_stream)
        stream.synchronize()
        assert b.status() == 0
        b.close()
    pick = np.random.default_rng(31).choice(n_img, n_img // 100, replace=False)
    tot = np.zeros(4, np.int64)
    with B.Context(max_slots=1) as ctx:
        for i in (int(k) for k in pick):
            img, out = imgs[i], jobs[i][2].cpu().numpy()
            xs, ys = img['xsize'], img['ysize']
            if xs * ys <= 320 * 320:
                x0 = y0 = 0
                sub, region = img, None
                w, h = xs, ys
            else:
                r = np.random.default_rng(i)
                x0 = 64 * int(r.integers(0, max(1, (xs - 1) // 64)))
                y0 = 64 * int(r.integers(0, max(1, (ys - 1) // 64)))
                cx0, cy0 = max(0, x0 - 64), max(0, y0 - 64)
                sub = crop_input(img, cx0, cy0, x0 + 128, y0 + 128)
                w, h = min(64, xs - x0), min(64, ys - y0)
                region = (x0 - cx0, y0 - cy0, x0 - cx0 + w, y0 - cy0 + h)
            ref = R.reconstruct(sub, p)
            gx = run(B, ctx, sub, params_pair(B)[1], XYB).transpose(2, 0, 1)
            o = out[y0:y0 + h, x0:x0 + w]
            u8, f16 = (o, None) if jobs[i][3] == B.OUT_U8_SRGB else (None, o)
            tot += assert_from_scratch(sub, ref, gx, None, u8, p,
                                       f"batch image {i} ({xs}x{ys}) at ({x0}, {y0})",
                                       region=region, relaxed_max=None, f16=f16)
    amb, nd, live, n = (int(v) for v in tot)
    print(f"batch sample: undetermined {amb} of {n // 3} pixels ({nd} decisions), relaxed "
          f"samples not clamped away {live / n:.4f}")
    assert live / n <= 0.03
    assert amb / (n // 3) <= 1e-3 or nd <= 2


@pytest.mark.parametrize("all_flat", [False, True])
def test_batch_j2_claims_span_images(all_flat):
    """The J.2 kernel of a batch claims the groups of all images from one
    counter and finds each group's image with a cursor over 32 images at a
    time: 70 images with the EPF (three chunks of the cursor), among them
    images with no block to filter (no AC coefficients, so every block's
    range is 0 and sigma < 16: DCT8 blocks with only their DC) next to
    images of the mixed workload; with all_flat, no image has any.  Every
    image equals its per-image result."""
    import torch
    from paper_1908_03565_gb300 import binding as B
    rng = np.random.default_rng(7400)
    jobs = []
    for i in range(70):
        xs, ys = (int(v) for v in np.exp(rng.uniform(np.log(8), np.log(300), 2)))
        flat = all_flat or i % 3 == 0
        img = B.to_device(synth.make_image(xs, ys, 7400 + i, y_dc_offset_q=200, ac=not flat,
                                           mix='dct8' if flat else 'mixed'), torch)
        dtype = (B.OUT_U8_SRGB, B.OUT_F32_LINEAR)[i % 2]
        params = B.filter_defaults(epf=1, gab=int(i % 4 != 1))
        shape, npd = B.out_shape(img, dtype)
        tdt = {np.float32: torch.float32, np.uint8: torch.uint8}[npd]
        jobs.append((img, params, torch.zeros(shape, dtype=tdt, device="cuda"), dtype))
    with B.Context(max_slots=1, timing=True) as ctx:
        want, listed = [], 0
        for img, params, out, dtype in jobs:
            t = ctx.submit(img, params, out, dtype, on_device=True)
            ctx.poll(t)
            listed += ctx.epf_stats(t)[1]
            want.append(out.cpu().numpy().copy())
            out.zero_()
        assert (listed == 0) == all_flat
        b = ctx.batch(jobs, autotune=False)
        stream = torch.cuda.Stream()
        for _ in range(2):
            b.launch(stream.cuda_stream)
            stream.synchronize()
            for (img, params, out, dtype), w in zip(jobs, want):
                np.testing.assert_array_equal(out.cpu().numpy(), w)
                out.zero_()
        assert b.status() == 0
        b.close()


def test_batch_needs_an_fp32_context():
    """Batches run the FP32 path: a context created for the tensor-core
    precision mode refuses them (no silent change of precision)."""
    import torch
    from paper_1908_03565_gb300 import binding as B
    jobs = _jobs(B, torch, n=2, seed=7500)
    with B.Context(precision=B.PREC_TC_F16X3) as ctx:
        with pytest.raises(B.JxlrError) as e:
            ctx.batch(jobs, autotune=False)
        assert e.value.status == B.JXLR_EINVAL
        assert "FP32" in str(e.value)
