"""GPU parity of the CUDA path (through the C ABI) with the FP64 oracle.

Histograms, LUTs and output pixels must be bit-exact with the oracle's (no tie band: a differing
LUT entry fails, and the failure says whether the oracle's decision there was a genuine FP64
near-tie); R, L and the enhanced histogram must agree within RTOL.
"""
import numpy as np
import pytest

import oracle
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
    p, po = params_pair(debug=True, **kw)
    return hr.Context(p), po


def test_small_lowlight_600x400(hr):
    """The 600x400 uint8 low-light image, K = 256, default parameters: several tiles plus ragged edges."""
    ctx, po = ctx_for(hr)
    img = synth.low_light_image(600, 400, seed=synth.seed_for(0, 0))
    out, dbg = run_gpu(ctx, img)
    compare_to_oracle(img, out, dbg, po)


@pytest.mark.parametrize("W,H", [(1, 1), (1, 9), (9, 1), (2, 2), (127, 31), (129, 33), (257, 65), (300, 7)])
def test_ragged_shapes(hr, W, H):
    ctx, po = ctx_for(hr)
    img = synth.low_light_image(W, H, seed=W * 1000 + H)
    out, dbg = run_gpu(ctx, img)
    compare_to_oracle(img, out, dbg, po)


@pytest.mark.parametrize("seed", range(6))
def test_k8_random_tiny_images(hr, seed):
    rng = np.random.default_rng(seed)
    H, W = int(rng.integers(1, 40)), int(rng.integers(1, 40))
    img = rng.integers(0, 8, size=(H, W, 3)).astype(np.uint8)
    ctx, po = ctx_for(hr, K=8, alpha=1e-2, beta=1e-2)
    out, dbg = run_gpu(ctx, img)
    compare_to_oracle(img, out, dbg, po)


@pytest.mark.parametrize("kind", ["black", "single_level", "checkerboard", "max_contrast", "gradient_ramp", "noise"])
def test_degenerate_images(hr, kind):
    H, W = 48, 70
    y, x = np.mgrid[0:H, 0:W]
    if kind == "black":
        img = np.zeros((H, W, 3), np.uint8)
    elif kind == "single_level":
        img = np.full((H, W, 3), 37, np.uint8)
    elif kind == "checkerboard":
        img = np.where(((x + y) % 2)[..., None] == 0, 10, 200).astype(np.uint8).repeat(3, axis=2)
    elif kind == "max_contrast":
        img = np.where((x < W // 2)[..., None], 0, 255).astype(np.uint8).repeat(3, axis=2)
    elif kind == "gradient_ramp":
        img = np.stack([(x * 255 // (W - 1)), (y * 255 // (H - 1)), np.zeros_like(x)], axis=2).astype(np.uint8)
    else:
        img = np.random.default_rng(3).integers(0, 256, size=(H, W, 3)).astype(np.uint8)
    ctx, po = ctx_for(hr)
    out, dbg = run_gpu(ctx, img)
    compare_to_oracle(img, out, dbg, po)


def test_padded_pitch_and_in_place(hr):
    ctx, po = ctx_for(hr)
    img = synth.low_light_image(333, 97, seed=77)
    out, dbg = run_gpu(ctx, img, pad_elems=13)
    compare_to_oracle(img, out, dbg, po)
    out2, dbg2 = run_gpu(ctx, img, pad_elems=5, inplace=True)
    assert np.array_equal(out, out2)


@pytest.mark.parametrize("kw", [dict(alpha=1e-4, beta=1e-4), dict(alpha=1e-2, beta=1e-3), dict(gamma=1.0),
                                dict(gamma=5.0), dict(max_iter=3), dict(fixed_iters=False, eps=1e3, max_iter=10)])
def test_parameter_variants(hr, kw):
    ctx, po = ctx_for(hr, **kw)
    img = synth.low_light_image(200, 150, seed=12)
    out, dbg = run_gpu(ctx, img)
    compare_to_oracle(img, out, dbg, po)


def test_uint16_12bit_k4096(hr):
    ctx, po = ctx_for(hr, K=4096, max_iter=3)
    img = synth.low_light_image(96, 64, seed=5, bits=12)
    out, dbg = run_gpu(ctx, img)
    compare_to_oracle(img, out, dbg, po)


def test_uint16_k256_small_levels(hr):
    ctx, po = ctx_for(hr, K=256)
    img = synth.low_light_image(130, 40, seed=6).astype(np.uint16)
    out, dbg = run_gpu(ctx, img)
    compare_to_oracle(img, out, dbg, po)


def test_level_out_of_range_is_reported(hr):
    import paper_2510_21100_gb300 as hrm
    ctx, _ = ctx_for(hr, K=8)
    img = np.zeros((4, 4, 3), np.uint8)
    img[1, 2, 1] = 9
    import torch
    d = torch.from_numpy(img).cuda()
    ctx.enhance(d, torch.empty_like(d))
    assert ctx.sync_status() == hrm.ERR_RANGE
    assert ctx.sync_status() == hrm.OK  # reading the status clears it


def test_invalid_arguments(hr):
    import torch
    import paper_2510_21100_gb300 as hrm
    ctx, _ = ctx_for(hr, K=4096)
    d = torch.zeros((4, 4, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(hrm.HistRetinexError):  # 8-bit data needs K <= 256
        ctx.enhance(d)
    ctx2, _ = ctx_for(hr)
    with pytest.raises(hrm.HistRetinexError):
        ctx2.enhance_ptr(d.data_ptr(), d.data_ptr(), 4, 4, 5, 12, 1)  # pitch below 3 W


def test_batch_equals_single_images(hr):
    """Each image of a mixed-size batch gets the pixels and LUT it gets alone; its FP64 histograms
    agree within RTOL (here both run on 16-CTA clusters; large batches run on smaller clusters or
    one CTA per image and sum in another order)."""
    import torch
    from gpu_util import assert_close
    ctx, po = ctx_for(hr)
    sizes = [(320, 240), (97, 33), (640, 360), (1, 1), (200, 301)]
    imgs = [synth.low_light_image(w, h, seed=900 + i) for i, (w, h) in enumerate(sizes)]
    dins = [torch.from_numpy(im).cuda() for im in imgs]
    outs = ctx.enhance_batch(dins)
    ctx.check()
    batch_dbg = [ctx.debug(i) for i in range(len(imgs))]
    for i, im in enumerate(imgs):
        out_b = outs[i].cpu().numpy()
        out_s, dbg_s = run_gpu(ctx, im)
        assert np.array_equal(out_b, out_s)
        for k in ("S", "G", "lut"):
            assert np.array_equal(batch_dbg[i][k], dbg_s[k]), k
        for k in ("R", "L", "T"):
            assert_close(batch_dbg[i][k], dbg_s[k], k)
        compare_to_oracle(im, out_b, batch_dbg[i], po)


def test_batch_of_large_images_takes_both_strip_paths(hr):
    """Two large images in one batch (few edge strips: each image's full strip columns on the
    interior path, the second image's partial last column on the edge path): histograms, LUT and
    pixels as each image gets alone in a single call."""
    import torch
    from gpu_util import assert_close
    ctx, po = ctx_for(hr)
    sizes = [(4096, 2048), (4000, 2001)]
    assert sum(-(-w // 512) * -(-h // 4) for w, h in sizes) >= 2 * 152 * 16
    imgs = [synth.low_light_image(w, h, seed=5300 + i) for i, (w, h) in enumerate(sizes)]
    dins = [hr.to_device_aligned(im) for im in imgs]
    douts = [hr.aligned_empty(h, w) for (w, h) in sizes]
    ctx.enhance_batch(dins, douts)
    ctx.check()
    batch = [(douts[i].cpu().numpy(), ctx.debug(i)) for i in range(len(imgs))]
    for i, im in enumerate(imgs):
        out_b, dbg_b = batch[i]
        out_s, dbg_s = run_gpu(ctx, im)
        for k in ("S", "G", "lut"):
            assert np.array_equal(dbg_b[k], dbg_s[k]), (i, k)
        for k in ("R", "L", "T"):
            assert_close(dbg_b[k], dbg_s[k], k)
        assert np.array_equal(out_b, out_s), i
    compare_to_oracle(imgs[1], batch[1][0], batch[1][1], po)


def test_batch_of_one_is_the_single_image_call(hr):
    """A batch of one image runs the single-image pipeline's kernels with the same cluster: the
    same bits throughout."""
    import torch
    ctx, _ = ctx_for(hr)
    img = synth.low_light_image(1280, 720, seed=4343)
    d = torch.from_numpy(img).cuda()
    out_b = ctx.enhance_batch([d])[0].cpu().numpy()
    dbg_b = ctx.debug(0)
    out_s, dbg_s = run_gpu(ctx, img)
    assert np.array_equal(out_b, out_s)
    for k in ("S", "G", "R", "L", "T", "lut"):
        assert np.array_equal(dbg_b[k], dbg_s[k]), k


def test_batch_result_independent_of_batch_composition(hr):
    """In the batched path an image's result is bit-identical whatever else is in the batch (for
    batches whose images get the same cluster size: here 16 CTAs)."""
    import torch
    ctx, _ = ctx_for(hr)
    target = synth.low_light_image(300, 200, seed=4242)
    others1 = [synth.low_light_image(w, h, seed=50 + w) for (w, h) in ((640, 480), (33, 17))]
    others2 = [synth.low_light_image(w, h, seed=70 + w) for (w, h) in ((1280, 720), (5, 5), (90, 60))]
    res = []
    for others, pos in ((others1, 1), (others2, 3)):
        batch = others[:pos] + [target] + others[pos:]
        outs = ctx.enhance_batch([torch.from_numpy(im).cuda() for im in batch])
        ctx.check()
        res.append((outs[pos].cpu().numpy(), ctx.debug(pos)))
    (o1, d1), (o2, d2) = res
    assert np.array_equal(o1, o2)
    for k in ("S", "G", "R", "L", "T", "lut"):
        assert np.array_equal(d1[k], d2[k]), k


def test_large_batch_takes_strip_histograms(hr):
    """A batch with enough 512 x 4 strips for the rolling strip histogram kernel, whose warps take
    equal runs of strip rows column by column, across image boundaries (interior and partial right
    columns on their two code paths): every image gets the histograms, LUT and pixels it gets alone,
    and a few are checked against the oracle.  Partial columns count the zero-filled pixels beyond the
    border at level 0 and take them back per warp, so S is the strongest check of that path."""
    import torch
    from gpu_util import assert_close
    ctx, po = ctx_for(hr)
    # (1056 and 528: partial last columns of whole 16-pixel lanes, no lane straddling the border)
    sizes = [(1500, 1000), (1283, 725), (700, 333), (512, 480), (1024, 769), (95, 33), (1, 1), (2047, 1031),
             (1056, 601), (528, 77)] * 4
    assert sum(-(-w // 512) * -(-h // 4) for w, h in sizes) >= 2 * 152 * 16
    imgs = [synth.low_light_image(w, h, seed=5100 + i) for i, (w, h) in enumerate(sizes)]
    dins = [hr.to_device_aligned(im) for im in imgs]
    douts = [hr.aligned_empty(h, w) for (w, h) in sizes]
    ctx.enhance_batch(dins, douts)
    ctx.check()
    batch = [(douts[i].cpu().numpy(), ctx.debug(i)) for i in range(len(imgs))]
    for i, im in enumerate(imgs):
        out_b, dbg_b = batch[i]
        out_s, dbg_s = run_gpu(ctx, im)
        for k in ("S", "G", "lut"):
            assert np.array_equal(dbg_b[k], dbg_s[k]), (i, k)
        for k in ("R", "L", "T"):
            assert_close(dbg_b[k], dbg_s[k], k)
        assert np.array_equal(out_b, out_s), i
    for i in (0, 2, 7, 8, 9):
        compare_to_oracle(imgs[i], batch[i][0], batch[i][1], po)


def test_host_entry_point_matches_device_path(hr):
    ctx, po = ctx_for(hr)
    img = synth.low_light_image(257, 129, seed=31)
    out_h = ctx.enhance_host(img)
    out_d, _ = run_gpu(ctx, img)
    assert np.array_equal(out_h, out_d)


@pytest.mark.parametrize("W,H", [(1000, 664), (3840, 2160), (7680, 4320)])
def test_full_size_single_images(hr, W, H):
    """The plain-method workloads at full size, checked pixel for pixel against the oracle."""
    ctx, po = ctx_for(hr)
    img = synth.low_light_image(W, H, seed=synth.seed_for(1, 0))
    out, dbg = run_gpu(ctx, img)
    compare_to_oracle(img, out, dbg, po)


def _strip_pad(W):
    """Row padding (elements) that makes 3 W + pad a multiple of 16: 16-byte aligned rows."""
    return (-3 * W) % 16


def test_large_ragged_image(hr):
    """A single image large enough for the rolling strip histogram kernel (512-pixel strip columns
    dealt out in runs of rows), with a partial last column (7001 = 13 * 512 + 345: a lane holding 9
    pixels) and a partial last band (4001 = 1000 * 4 + 1)."""
    ctx, po = ctx_for(hr)
    img = synth.low_light_image(7001, 4001, seed=synth.seed_for(1, 7))
    out, dbg = run_gpu(ctx, img, pad_elems=_strip_pad(7001))
    compare_to_oracle(img, out, dbg, po)


def test_large_image_below_256_levels(hr):
    """The strip kernel's clamping path (K < 256) on in-range data."""
    ctx, po = ctx_for(hr, K=128)
    img = np.minimum(synth.low_light_image(6145, 3203, seed=synth.seed_for(1, 8)), 127).astype(np.uint8)
    out, dbg = run_gpu(ctx, img, pad_elems=_strip_pad(6145))
    compare_to_oracle(img, out, dbg, po)


def test_large_image_level_out_of_range_is_reported(hr):
    import paper_2510_21100_gb300 as hrm
    ctx, _ = ctx_for(hr, K=64)
    img = synth.low_light_image(7680, 4320, seed=synth.seed_for(1, 9))
    assert img.max() >= 64
    import torch
    d = torch.from_numpy(img).cuda()
    ctx.enhance(d, torch.empty_like(d))
    assert ctx.sync_status() == hrm.ERR_RANGE


def test_repeated_calls_are_deterministic(hr):
    ctx, _ = ctx_for(hr)
    img = synth.low_light_image(640, 480, seed=8)
    a, da = run_gpu(ctx, img)
    b, db = run_gpu(ctx, img)
    assert np.array_equal(a, b)
    for k in ("R", "L", "T"):
        assert np.array_equal(da[k], db[k])
