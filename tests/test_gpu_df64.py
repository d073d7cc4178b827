"""GPU parity of the double-float solve (HR_PREC_DF64) with the FP64 oracle.

The double-float form computes the solve's sums in pairs of FP32 numbers (about 2^-47 relative
per operation).  It is held to the plain form's bar: histograms and output pixels exact, R, L and
the enhanced histogram within RTOL = 1e-9 of the oracle, LUT entries exact away from ties.
"""
import numpy as np
import pytest

from gpu_util import compare_to_oracle, params_pair, run_gpu
from paper_2510_21100_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hr():
    import paper_2510_21100_gb300 as hr
    from paper_2510_21100_gb300 import build
    build.build()
    return hr


def ctx_for(hr, **kw):
    p, po = params_pair(debug=True, precision=hr.PREC_DF64, **kw)
    return hr.Context(p), po


@pytest.mark.parametrize("W,H", [(600, 400), (1000, 664), (257, 129), (31, 7)])
def test_df64_single_images(hr, W, H):
    ctx, po = ctx_for(hr)
    img = synth.low_light_image(W, H, seed=synth.seed_for(1, W))
    out, dbg = run_gpu(ctx, img)
    compare_to_oracle(img, out, dbg, po)


@pytest.mark.parametrize("kw", [dict(alpha=1e-4, beta=1e-2), dict(alpha=1e-2, beta=1e-4, gamma=1.0),
                                dict(max_iter=3), dict(K=8)])
def test_df64_parameter_variants(hr, kw):
    ctx, po = ctx_for(hr, **kw)
    img = synth.low_light_image(320, 240, seed=77)
    if kw.get("K", 256) < 256:
        img = (img.astype(np.int64) * kw["K"] // 256).astype(np.uint8)
    out, dbg = run_gpu(ctx, img)
    compare_to_oracle(img, out, dbg, po)


def test_df64_batch_of_mixed_images(hr):
    """The batched path (one CTA per image) in double-float, image by image against the oracle."""
    import torch
    ctx, po = ctx_for(hr)
    sizes = [(320, 240), (97, 33), (1280, 720), (1, 1), (200, 301), (1919, 1079)]
    imgs = [synth.low_light_image(w, h, seed=1900 + i) for i, (w, h) in enumerate(sizes)]
    outs = ctx.enhance_batch([torch.from_numpy(im).cuda() for im in imgs])
    ctx.check()
    for i, im in enumerate(imgs):
        compare_to_oracle(im, outs[i].cpu().numpy(), ctx.debug(i), po)


def test_df64_uint16_k4096(hr):
    """K = 4096 keeps the solver vectors in the global workspace: that path in double-float."""
    import torch
    ctx, po = ctx_for(hr, K=4096, max_iter=3)
    img = synth.low_light_image(96, 64, seed=31, bits=12)
    out, dbg = run_gpu(ctx, img)
    compare_to_oracle(img, out, dbg, po)


def test_df64_full_size(hr):
    ctx, po = ctx_for(hr)
    img = synth.low_light_image(7680, 4320, seed=synth.seed_for(1, 0))
    out, dbg = run_gpu(ctx, img)
    compare_to_oracle(img, out, dbg, po)
