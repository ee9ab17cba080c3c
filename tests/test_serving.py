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


def test_server_fed_from_several_threads():
    """The request server on its own thread, fed by four producer threads at
    once and waited on from them: every result equals its result alone."""
    import threading
    import torch
    from paper_1908_03565_gb300 import binding as B
    jobs = _jobs(B, torch)
    alone = []
    with B.Context(max_slots=1) as ctx:
        for img, params, out, dtype in jobs:
            ctx.poll(ctx.submit(img, params, out, dtype, on_device=True))
            alone.append(out.cpu().numpy().copy())
            out.zero_()
    torch.cuda.synchronize()
    with B.Context(max_slots=4) as ctx:
        srv = ctx.server()
        lat = [None] * len(jobs)
        errors = []

        def producer(k):
            try:
                for i in range(k, len(jobs), 4):
                    rid = srv.enqueue(jobs[i])
                    lat[i] = srv.wait(rid)
            except Exception as e:       # reported below
                errors.append(e)

        threads = [threading.Thread(target=producer, args=(k,)) for k in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        stats = srv.stop()
        torch.cuda.synchronize()
        assert not errors, errors
        assert stats["completed"] == len(jobs) and all(v > 0 for v in lat)
        for (img, params, out, dtype), want in zip(jobs, alone):
            np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_server_admits_past_a_request_that_does_not_fit():
    """Under an HBM cap that holds one large request, a second large request
    waits while small ones behind it are admitted (bypassed > 0); with a
    zero age bound nothing passes it; every request completes correctly."""
    import torch
    from paper_1908_03565_gb300 import binding as B
    big = [B.to_device(synth.make_image(1024, 1024, 950 + i), torch) for i in range(2)]
    small = [B.to_device(synth.make_image(64, 64, 960 + i), torch) for i in range(6)]
    p = B.filter_defaults(epf=1, gab=1)
    jobs = [(img, p, torch.zeros((img['ysize'], img['xsize'], 3), dtype=torch.uint8,
                                 device="cuda"), B.OUT_U8_SRGB) for img in big + small]
    alone = []
    with B.Context(max_slots=1) as ctx:
        for img, params, out, dtype in jobs:
            ctx.poll(ctx.submit(img, params, out, dtype, on_device=True))
            alone.append(out.cpu().numpy().copy())
            out.zero_()
    # a 1024^2 request needs ~34 MB of scratch (XYB, J.2 output, lists); the
    # cap holds one of them and the small ones
    for age, want_bypass in ((1000.0, True), (0.0, False)):
        with B.Context(max_slots=8, hbm_cap_bytes=48 << 20) as ctx:
            srv = ctx.server(age_bound_ms=age)
            ids = [srv.enqueue(j) for j in jobs]
            for i in ids:
                srv.wait(i)
            stats = srv.stop()
            torch.cuda.synchronize()
        assert stats["completed"] == len(jobs)
        assert (stats["bypassed"] > 0) == want_bypass, stats
        for (img, params, out, dtype), want in zip(jobs, alone):
            np.testing.assert_array_equal(out.cpu().numpy(), want)
            out.zero_()


def test_server_runs_large_requests_alone():
    """With exclusive_mpx, a request of that size is admitted only onto an
    idle device and nothing joins it: with large requests enqueued among
    small ones, at most one request is in flight whenever a large one is,
    which shows as max_in_flight 1 when every request is large."""
    import torch
    from paper_1908_03565_gb300 import binding as B
    big = [B.to_device(synth.make_image(1024, 1024, 970 + i), torch) for i in range(4)]
    p = B.filter_defaults(epf=1, gab=1)
    jobs = [(img, p, torch.zeros((1024, 1024, 3), dtype=torch.uint8, device="cuda"),
             B.OUT_U8_SRGB) for img in big]
    with B.Context(max_slots=4) as ctx:
        srv = ctx.server(exclusive_mpx=1.0)
        ids = [srv.enqueue(j) for j in jobs]
        for i in ids:
            srv.wait(i)
        stats = srv.stop()
    assert stats["completed"] == 4 and stats["max_in_flight"] == 1
    with B.Context(max_slots=4) as ctx:
        srv = ctx.server(exclusive_mpx=0.0)
        ids = [srv.enqueue(j) for j in jobs]
        for i in ids:
            srv.wait(i)
        stats = srv.stop()
    assert stats["completed"] == 4 and stats["max_in_flight"] > 1
