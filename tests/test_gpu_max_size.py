"""GPU parity at the largest image the library takes: just under 2^31 pixels (65472 x 32800).

The oracle cannot run on two billion pixels in a test, so the image is built so that its exact
results follow from the oracle's results on one small tile T (1023 x 1025): 2048 copies of T laid
out in 2 x 2 blocks [T, T mirrored left-right; T mirrored top-bottom, T mirrored both ways].  At every
seam a pixel's 3 x 3 neighbourhood then holds the same values (mirrored) as T's with the replicated
border, and mirroring keeps V and the Sobel magnitude, so H_C(S) and H_C(grad S) of the large image
are exactly 2048 times T's.  Every equation of the solve and of the target is homogeneous of degree
one in (S, G, R, L, N), and scaling by a power of two is exact in floating point, so R, L and the
enhanced histogram are 2048 times T's and the LUT is T's; the output is the same mirrored tiling of
T's output.  Images of 2^31 pixels or more are refused (HR_ERR_UNSUPPORTED) and the context stays usable.
"""
import numpy as np
import pytest

import oracle
from gpu_util import assert_close, assert_lut_equal
from paper_2510_21100_gb300 import synth

pytestmark = pytest.mark.gpu

TW, TH = 1023, 1025          # tile
BX, BY = 32, 16              # 2 x 2 blocks across and down
NT = 4 * BX * BY             # tiles: 2048 (a power of two)
W, H = 2 * BX * TW, 2 * BY * TH  # 65472 x 32800 = 2^31 - 2048 pixels


@pytest.fixture(scope="module")
def hr():
    import paper_2510_21100_gb300 as hr
    from paper_2510_21100_gb300 import build
    build.build()
    return hr


def mirrored_tiling(t):
    """(2 BY TH, 2 BX TW, 3) contiguous device tensor of 2 x 2 mirrored blocks of the device tile t."""
    import torch
    top = torch.cat([t, t.flip(1)], dim=1)
    blk = torch.cat([top, top.flip(0)], dim=0)
    return blk.repeat(BY, BX, 1)


@pytest.mark.parametrize("bits,K", [(8, 256), (12, 4096)])
def test_largest_image_against_the_oracle_on_its_tile(hr, bits, K):
    import torch
    assert W * H < 2 ** 31 and W * H == NT * TW * TH
    tile = synth.low_light_image(TW, TH, seed=9100 + bits, bits=bits)
    ref = oracle.enhance(tile, oracle.Params(K=K))
    din = mirrored_tiling(torch.from_numpy(tile).cuda())
    assert tuple(din.shape) == (H, W, 3) and din.is_contiguous()
    dout = torch.empty_like(din)
    ctx = hr.Context(hr.Params(K=K, debug=True))
    ctx.enhance(din, dout)
    ctx.check()
    dbg = ctx.debug(0)
    assert np.array_equal(dbg["S"], NT * ref.S.astype(np.uint64)), "H_C(S) differs"
    assert np.array_equal(dbg["G"], NT * ref.G.astype(np.uint64)), "H_C(grad S) differs"
    assert dbg["iters"] == ref.iters
    assert_close(dbg["R"] / NT, ref.R, "H_C(R)")
    assert_close(dbg["L"] / NT, ref.L, "H_C(L)")
    assert_close(dbg["T"] / NT, ref.T, "enhanced histogram")
    assert_lut_equal(dbg["lut"], ref.S, ref.T, ref.lut)
    del din
    want = mirrored_tiling(torch.from_numpy(ref.out).cuda())
    assert torch.equal(dout, want), "output pixels differ from the mirrored tiling of the oracle's output"
    del dout, want
    torch.cuda.empty_cache()


def test_images_of_2_31_pixels_are_refused(hr):
    import torch
    import paper_2510_21100_gb300 as hrm
    ctx = hr.Context(hr.Params(debug=True))
    d = torch.zeros((4, 4, 3), dtype=torch.uint8, device="cuda")
    # (the size check comes before any launch: the pointers are never dereferenced)
    with pytest.raises(hrm.HistRetinexError) as e:
        ctx.enhance_ptr(d.data_ptr(), d.data_ptr(), 65536, 32768, 3 * 65536, 3 * 65536, 1)
    assert e.value.code == hrm.ERR_UNSUPPORTED
    img = synth.low_light_image(96, 64, seed=9200)
    out = ctx.enhance(torch.from_numpy(img).cuda()).cpu().numpy()
    ctx.check()
    assert np.array_equal(out, oracle.enhance(img, oracle.Params(K=256)).out)
