"""Kernel variants of the same step give the same bits.

The transform kernel has two forms: one CTA per 32x32 cell, and a persistent
grid whose CTAs fetch the next cell's coefficients and map during the
current cell's stores.  Both run the same per-cell arithmetic in the same
order, so every output (XYB, f32, f16, u8, with and without the filters)
must agree bit for bit; a context picks its form at creation
(JXLR_RECON_VARIANT=grid|persistent).
"""
import os

import numpy as np
import pytest

from paper_1908_03565_gb300 import synth
from test_gpu_parity import B, F32, F16, U8, XYB, params_pair, run  # noqa: F401

pytestmark = pytest.mark.gpu


def _ctx(B, variant):
    old = os.environ.get("JXLR_RECON_VARIANT")
    os.environ["JXLR_RECON_VARIANT"] = variant
    try:
        return B.Context(max_slots=1)
    finally:
        if old is None:
            del os.environ["JXLR_RECON_VARIANT"]
        else:
            os.environ["JXLR_RECON_VARIANT"] = old


@pytest.fixture(scope="module")
def ctxs(B):
    a, b = _ctx(B, "grid"), _ctx(B, "persistent")
    yield a, b
    a.close()
    b.close()


@pytest.mark.parametrize("xs,ys,seed", [(1, 1, 1), (33, 17, 2), (320, 200, 3), (1000, 520, 4),
                                        (2048, 1088, 5)])
@pytest.mark.parametrize("epf,gab", [(0, 0), (0, 1), (1, 1)])
def test_transform_forms_agree(B, ctxs, xs, ys, seed, epf, gab):
    img = synth.make_image(xs, ys, seed, y_dc_offset_q=200)
    _, lp = params_pair(B, epf=bool(epf), gab=bool(gab))
    grid, pers = ctxs
    for dt in (XYB, F32, F16, U8):
        np.testing.assert_array_equal(run(B, grid, img, lp, dt), run(B, pers, img, lp, dt))
