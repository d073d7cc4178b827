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


def test_noalloc_rejects_k_beyond_its_workspace():
    import paper_2510_21100_gb300 as hr
    import torch
    d = hr.aligned_empty(8, 8, dtype=torch.uint16)
    with pytest.raises(hr.HistRetinexError) as e:
        hr.enhance_noalloc(d, hr.aligned_empty(8, 8, dtype=torch.uint16), hr.Params(K=4096))
    assert e.value.code == hr.ERR_UNSUPPORTED
