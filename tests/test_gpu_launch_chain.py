"""GPU tests of the launch chain between calls: histograms cleared by the solve instead of a memset,
single-image calls with the image in the kernel parameters, programmatic dependent launches.

A context without debug intermediates zeroes H_C(S) and H_C(grad S) only when it cannot know them
to be zero; after that every solve clears the slots it used.  A debug context zeroes them before
every call.  Both run the same kernels on the same data, so their outputs must agree bit for bit
through any sequence of calls (sizes, batch sizes, graph replays, stream order or dependent
launches).
"""
import numpy as np
import pytest

from paper_2510_21100_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hr():
    import paper_2510_21100_gb300 as hr
    from paper_2510_21100_gb300 import build
    build.build()
    return hr


def images(sizes, seed):
    return [synth.low_light_image(w, h, seed=seed + i) for i, (w, h) in enumerate(sizes)]


def single(ctx, img):
    import torch
    out = ctx.enhance(torch.from_numpy(img).cuda())
    ctx.check()
    return out.cpu().numpy()


def batch(ctx, imgs):
    import torch
    outs = ctx.enhance_batch([torch.from_numpy(im).cuda() for im in imgs])
    ctx.check()
    return [o.cpu().numpy() for o in outs]


def test_single_image_calls_in_sequence_match_a_debug_context(hr):
    # includes a strip-kernel image (the 8-bit pass for large images) between tile-kernel ones
    imgs = images([(1920, 1080), (97, 33), (7680, 4320), (640, 480), (1, 1)], seed=4100)
    fast = hr.Context(hr.Params())
    ref = hr.Context(hr.Params(debug=True))
    want = [single(ref, im) for im in imgs]
    for _ in range(3):
        for im, w in zip(imgs, want):
            assert np.array_equal(single(fast, im), w)


def test_batch_sizes_up_and_down_match_a_debug_context(hr):
    fast = hr.Context(hr.Params())
    direct = hr.Context(hr.Params())
    direct.set_tuning(use_graph=0)
    ref = hr.Context(hr.Params(debug=True))
    ref.set_tuning(use_graph=0)
    for step, n in enumerate([5, 2, 7, 3, 7, 1]):
        sizes = synth.mixed_batch_sizes(n, 60 + step, min_wh=(64, 48), max_wh=(800, 600))
        imgs = images(sizes, seed=4200 + 10 * step)
        want = batch(ref, imgs)
        for ctx in (fast, direct):
            for got, w in zip(batch(ctx, imgs), want):
                assert np.array_equal(got, w)
        # single-image calls between batches use slot 0 only
        assert np.array_equal(single(fast, imgs[0]), want[0])


@pytest.mark.parametrize("pdl", [1, 2, 4, 7])
def test_dependent_launches_equal_stream_order(hr, pdl):
    imgs = images([(1280, 720), (333, 211), (3840, 2160)], seed=4300)
    on = hr.Context(hr.Params())
    on.set_tuning(pdl=pdl)
    off = hr.Context(hr.Params())
    off.set_tuning(pdl=0)
    for im in imgs:
        assert np.array_equal(single(on, im), single(off, im))
    for a, b in zip(batch(on, imgs), batch(off, imgs)):
        assert np.array_equal(a, b)


def test_default_dependent_launches_are_the_pixel_passes(hr):
    assert hr.Context(hr.Params()).tuning()["pdl"] == 5


def test_invalid_pdl_value_is_rejected(hr):
    ctx = hr.Context(hr.Params())
    with pytest.raises(hr.HistRetinexError):
        ctx.set_tuning(pdl=8)
    assert ctx.tuning()["pdl"] == 5
