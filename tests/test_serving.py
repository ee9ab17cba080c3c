"""Serving: the native request loop (jxl_recon_serve) admits requests as
slots and HBM free up and runs them concurrently; every result must be the
same alone and in the mix."""
import numpy as np
import pytest

from paper_1908_03565_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [(40, 33), (300, 200), (1024, 768), (64, 512), (777, 91), (2048, 1000),
         (128, 128), (500, 500), (9, 1200), (1500, 17)]


def _jobs(B, torch):
    jobs = []
    for i, (xs, ys) in enumerate(SIZES):
        img = B.to_device(synth.make_image(xs, ys, 500 + i, y_dc_offset_q=200), torch)
        dtype = (B.OUT_U8_SRGB, B.OUT_F16_LINEAR, B.OUT_F32_LINEAR)[i % 3]
        on = i % 4 != 3
        params = B.filter_defaults(epf=int(on), gab=int(on))
        shape, npd = B.out_shape(img, dtype)
        tdt = {np.float32: torch.float32, np.float16: torch.float16, np.uint8: torch.uint8}[npd]
        out = torch.zeros(shape, dtype=tdt, device="cuda")
        jobs.append((img, params, out, dtype))
    return jobs


def test_results_alone_equal_results_in_the_mix():
    import torch
    from paper_1908_03565_gb300 import binding as B
    jobs = _jobs(B, torch)
    alone = []
    with B.Context(max_slots=1) as ctx:
        for img, params, out, dtype in jobs:
            t = ctx.submit(img, params, out, dtype, on_device=True)
            ctx.poll(t)
            alone.append(out.cpu().numpy().copy())
            out.zero_()
    rng = np.random.default_rng(3)
    schedules = [np.zeros(len(jobs)),                                   # all at once
                 np.cumsum(rng.exponential(2e-4, len(jobs)))]           # Poisson
    with B.Context(max_slots=4) as ctx:
        for arr in schedules:
            lat, stats = ctx.serve(jobs, arr)
            torch.cuda.synchronize()
            assert stats["completed"] == len(jobs)
            assert np.all(lat > 0)
            for (img, params, out, dtype), want in zip(jobs, alone):
                np.testing.assert_array_equal(out.cpu().numpy(), want)
                out.zero_()
        assert stats["max_in_flight"] >= 2


def test_hbm_cap_bounds_concurrency():
    import torch
    from paper_1908_03565_gb300 import binding as B
    jobs = []
    for i in range(8):
        img = B.to_device(synth.make_image(512, 512, 900 + i), torch)
        out = torch.zeros((512, 512, 3), dtype=torch.uint8, device="cuda")
        jobs.append((img, B.filter_defaults(epf=1, gab=1), out, B.OUT_U8_SRGB))
    # one request needs ~3.2 MB of scratch (XYB + sigma), rounded to 4 MiB
    with B.Context(max_slots=8, hbm_cap_bytes=9 << 20) as ctx:
        lat, stats = ctx.serve(jobs, np.zeros(8))
        assert stats["completed"] == 8
        assert stats["max_in_flight"] <= 2
        assert stats["busy_refusals"] > 0
        assert ctx.device_bytes() <= 9 << 20
