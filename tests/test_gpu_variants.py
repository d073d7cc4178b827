"""GPU parity of the printed-form variants (flags HR_FLAG_PRINTED_UPDATE, HR_FLAG_NEAREST_MATCH,
HR_FLAG_FORWARD_GRADIENT) with the oracle's variants: histograms, LUT and pixels bit-exact, R, L
and the enhanced histogram within RTOL (the printed update's sums are non-negative too, and ten
iterations keep a differently ordered evaluation within 2e-14 of the oracle on these images)."""
import numpy as np
import pytest

from gpu_util import assert_close, compare_to_oracle, params_pair, run_gpu
from paper_2510_21100_gb300 import synth

pytestmark = pytest.mark.gpu

FLAGS = {
    "printed": dict(printed_update=True),
    "nearest": dict(nearest_match=True),
    "forward": dict(forward_gradient=True),
    "all": dict(printed_update=True, nearest_match=True, forward_gradient=True),
}


@pytest.fixture(scope="module")
def hr():
    import paper_2510_21100_gb300 as hr
    from paper_2510_21100_gb300 import build
    build.build()
    return hr


@pytest.mark.parametrize("name", list(FLAGS))
@pytest.mark.parametrize("W,H", [(600, 400), (257, 129), (1, 1), (33, 7)])
def test_variant_single_image(hr, name, W, H):
    p, po = params_pair(debug=True, **FLAGS[name])
    ctx = hr.Context(p)
    img = synth.low_light_image(W, H, seed=synth.seed_for(0, 0) + W)
    out, dbg = run_gpu(ctx, img)
    compare_to_oracle(img, out, dbg, po)


@pytest.mark.parametrize("name", list(FLAGS))
def test_variant_k8_random(hr, name):
    rng = np.random.default_rng(17)
    img = rng.integers(0, 8, size=(23, 31, 3)).astype(np.uint8)
    p, po = params_pair(debug=True, K=8, alpha=1e-2, beta=1e-2, **FLAGS[name])
    out, dbg = run_gpu(hr.Context(p), img)
    compare_to_oracle(img, out, dbg, po)


@pytest.mark.parametrize("name", ["printed", "nearest", "forward"])
def test_variant_full_size(hr, name):
    """3840x2160 (the 16-CTA cluster solve, the strip kernel for the default gradient)."""
    p, po = params_pair(debug=True, **FLAGS[name])
    img = synth.low_light_image(3840, 2160, seed=synth.seed_for(1, 0))
    out, dbg = run_gpu(hr.Context(p), img)
    compare_to_oracle(img, out, dbg, po)


def test_variant_12bit(hr):
    p, po = params_pair(debug=True, K=4096, max_iter=3, **FLAGS["all"])
    img = synth.low_light_image(96, 64, seed=5, bits=12)
    out, dbg = run_gpu(hr.Context(p), img)
    compare_to_oracle(img, out, dbg, po)


def test_variants_in_a_batch_equal_single_calls(hr):
    """A batch (one CTA per image for 64 images) with all three variants: every image equals its
    single-image call on histograms, LUT and pixels, and a few equal the oracle."""
    import torch
    p, po = params_pair(debug=True, **FLAGS["all"])
    ctx = hr.Context(p)
    sizes = [(320, 240), (97, 33), (640, 360), (1, 1), (200, 301), (128, 128), (511, 17), (64, 700)] * 8
    imgs = [synth.low_light_image(w, h, seed=700 + i) for i, (w, h) in enumerate(sizes)]
    outs = ctx.enhance_batch([torch.from_numpy(im).cuda() for im in imgs])
    ctx.check()
    dbgs = [ctx.debug(i) for i in range(len(imgs))]
    single = hr.Context(p)
    for i in (0, 2, 5, 6, 7, 13):
        out_s, dbg_s = run_gpu(single, imgs[i])
        assert np.array_equal(outs[i].cpu().numpy(), out_s), i
        for k in ("S", "G", "lut"):
            assert np.array_equal(dbgs[i][k], dbg_s[k]), (i, k)
        for k in ("R", "L", "T"):
            assert_close(dbgs[i][k], dbg_s[k], k)
    for i in (0, 6):
        compare_to_oracle(imgs[i], outs[i].cpu().numpy(), dbgs[i], po)


def test_printed_update_needs_fp64(hr):
    """The printed update's values leave FP32's exponent range (which double-float shares): only
    the FP64 form takes it."""
    for prec in (hr.PREC_FP32, hr.PREC_DF64):
        with pytest.raises(hr.HistRetinexError) as e:
            hr.Context(hr.Params(precision=prec, printed_update=True))
        assert e.value.code == hr.ERR_UNSUPPORTED
    p, po = params_pair(debug=True, precision=hr.PREC_DF64, nearest_match=True, forward_gradient=True)
    img = synth.low_light_image(640, 480, seed=3)
    out, dbg = run_gpu(hr.Context(p), img)
    compare_to_oracle(img, out, dbg, po)


def test_variants_through_the_allocation_free_entry_point(hr):
    import torch
    p = hr.Params(**FLAGS["all"])
    img = synth.low_light_image(300, 200, seed=91)
    d_in = hr.to_device_aligned(img)
    ref = hr.Context(p).enhance(d_in, hr.aligned_empty(200, 300)).cpu().numpy()
    out = hr.enhance_noalloc(d_in, hr.aligned_empty(200, 300), p)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)
