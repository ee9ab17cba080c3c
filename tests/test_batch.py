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
