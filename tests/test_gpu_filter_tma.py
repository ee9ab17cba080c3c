"""The Gaborish / colour stage with its tiles brought in by TMA loads, against
the same stage with ordinary loads (a caller XYB whose rows are not 16-byte
multiples takes those), and against the oracle, at sizes where the ring
outside the image is mirrored on every side (one-pixel rows and columns).

Both forms compute every sample with the same operations in the same order,
so they must agree bit for bit.
"""
import numpy as np
import pytest

from oracle import recon as R
from paper_1908_03565_gb300 import synth
from test_gpu_parity import B, ctx, F32, XYB, TOL01, check_rgb01  # noqa: F401

pytestmark = pytest.mark.gpu


def _xyb(xs, ys, seed):
    """Smooth planar XYB (3, ys, xs) in the range of real images."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:ys, 0:xs]
    ph = rng.uniform(0, 6.28, 3)
    return np.stack([0.03 * np.sin(xx / 7.0 + ph[0]),
                     0.5 + 0.3 * np.sin(yy / 5.0 + ph[1]) * np.cos(xx / 9.0),
                     0.4 + 0.2 * np.cos(yy / 6.0 + xx / 11.0 + ph[2])]).astype(np.float32)


def _stage(B, ctx, xyb, stride, lp, dtype=F32):
    import torch
    _, ys, xs = xyb.shape
    buf = torch.zeros((3, ys, stride), dtype=torch.float32, device="cuda")
    buf[:, :, :xs] = torch.from_numpy(xyb).cuda()
    img = synth.make_image(xs, ys, 7)
    dimg = B.to_device(img, torch)
    out = torch.full((ys, xs, 3), 7.0, dtype=torch.float32, device="cuda")
    ctx.poll(ctx.submit_xyb(buf, xs, ys, dimg['vmap'], dimg['acmul'], dimg['sharpness'], lp,
                            out, dtype))
    return out.cpu().numpy()


@pytest.mark.parametrize("xs,ys", [(64, 40), (131, 77), (1, 1), (1, 37), (37, 1), (33, 2),
                                   (200, 33)])
@pytest.mark.parametrize("noise", [0, 1])
def test_tma_loads_equal_plain_loads(B, ctx, xs, ys, noise):
    xyb = _xyb(xs, ys, 31 * xs + ys)
    lp = B.filter_defaults(gab=1, noise=noise, noise_lut=[0.5] * 16)
    aligned = xs + (-xs % 4)            # rows of 16-byte multiples: TMA tiles
    plain = aligned + 1                 # not: the all-threads tile load
    got = _stage(B, ctx, xyb, aligned, lp)
    np.testing.assert_array_equal(got, _stage(B, ctx, xyb, plain, lp))
    if not noise:
        p = R.Params(gab=True)
        want = R.xyb_to_linear01(R.gaborish(xyb.astype(np.float64), p), p)
        check_rgb01(got, want)
