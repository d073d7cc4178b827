"""The allocation-free entry point histretinex_enhance_noalloc, called through the C ABI.

It serves callers that cannot allocate device memory when they call (graph capture by a
framework, real-time loops, plug-ins whose host owns device memory): one image, no context, its
workspace in a fixed device array.  Its output must equal histretinex_enhance's (the tests'
bar for pixels: bit-exact) on two calls in a row, the second reusing the workspace the first
left behind.  This file is collected last so a run that stops at the first failure has already
run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2510_21100_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_equals_enhance_on_two_calls_in_a_row():
    import torch
    import paper_2510_21100_gb300 as hr
    from paper_2510_21100_gb300 import build
    build.build()
    lib = hr.library()
    p = hr.Params()
    ctx = hr.Context(p)
    imgs = [synth.low_light_image(600, 400, seed=synth.seed_for(0, 0)),
            synth.low_light_image(333, 217, seed=71)]            # second call: another size
    for img in imgs:
        H, W, _ = img.shape
        d_in = hr.to_device_aligned(img)
        ref = ctx.enhance(d_in, hr.aligned_empty(H, W)).cpu().numpy()
        d_out = hr.aligned_empty(H, W)
        cp = p.c()
        st = lib.histretinex_enhance_noalloc(
            ctypes.byref(cp), ctypes.c_void_p(d_in.data_ptr()), ctypes.c_void_p(d_out.data_ptr()), W, H,
            d_in.stride(0), d_out.stride(0), 1, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == hr.OK
        torch.cuda.synchronize()
        assert np.array_equal(d_out.cpu().numpy(), ref)
    ctx.check()


def _noalloc_call(lib, hr, p, d_in, d_out, eb):
    import torch
    H, W = int(d_in.shape[0]), int(d_in.shape[1])
    cp = p.c()
    return lib.histretinex_enhance_noalloc(
        ctypes.byref(cp), ctypes.c_void_p(d_in.data_ptr()), ctypes.c_void_p(d_out.data_ptr()), W, H,
        d_in.stride(0) * eb, d_out.stride(0) * eb, eb, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_follows_changes_of_k_gamma_and_element_size():
    """Calls in a row with K = 64, then K = 256, then another gamma, then a 16-bit image: each call
    rebuilds its own class-boundary table and clears what it accumulates, so every result equals
    histretinex_enhance's on a context made for the same parameters, bit for bit."""
    import torch
    import paper_2510_21100_gb300 as hr
    from paper_2510_21100_gb300 import build
    build.build()
    lib = hr.library()
    base = synth.low_light_image(517, 301, seed=72)
    cases = [(hr.Params(K=64), (base // 4).astype(np.uint8)),
             (hr.Params(K=256), base),
             (hr.Params(K=256, gamma=3.1), base),
             (hr.Params(K=256, gamma=3.1), base.astype(np.uint16)),
             (hr.Params(K=128, alpha=1e-2), (base // 2).astype(np.uint8))]
    for p, img in cases:
        H, W, _ = img.shape
        dt = torch.uint8 if img.dtype == np.uint8 else torch.uint16
        eb = img.dtype.itemsize
        d_in = hr.to_device_aligned(img)
        with hr.Context(p) as ctx:
            ref = ctx.enhance(d_in, hr.aligned_empty(H, W, dtype=dt)).cpu().numpy()
            ctx.check()
        d_out = hr.aligned_empty(H, W, dtype=dt)
        assert _noalloc_call(lib, hr, p, d_in, d_out, eb) == hr.OK
        torch.cuda.synchronize()
        assert np.array_equal(d_out.cpu().numpy(), ref), (p.K, p.gamma, img.dtype)


def test_noalloc_rejects_k_beyond_its_workspace():
    import paper_2510_21100_gb300 as hr
    import torch
    d = hr.aligned_empty(8, 8, dtype=torch.uint16)
    with pytest.raises(hr.HistRetinexError) as e:
        hr.enhance_noalloc(d, hr.aligned_empty(8, 8, dtype=torch.uint16), hr.Params(K=4096))
    assert e.value.code == hr.ERR_UNSUPPORTED
