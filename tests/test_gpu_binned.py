"""GPU parity of the binned form (K bins over M > K data levels) with the oracle's: histograms,
LUT and pixels bit-exact, R, L and the enhanced histogram within RTOL."""
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


@pytest.mark.parametrize("W,H", [(1000, 664), (257, 129), (1, 1), (31, 7)])
def test_12bit_data_in_256_bins(hr, W, H):
    p, po = params_pair(debug=True, K=256, levels=4096)
    img = synth.low_light_image(W, H, seed=synth.seed_for(3, 7) + W, bits=12)
    out, dbg = run_gpu(hr.Context(p), img)
    compare_to_oracle(img, out, dbg, po)


@pytest.mark.parametrize("K", [16, 64, 128])
def test_8bit_data_in_fewer_bins(hr, K):
    p, po = params_pair(debug=True, K=K, levels=256)
    img = synth.low_light_image(640, 480, seed=K)
    out, dbg = run_gpu(hr.Context(p), img)
    compare_to_oracle(img, out, dbg, po)


@pytest.mark.parametrize("seed", range(3))
def test_k8_over_32_levels(hr, seed):
    rng = np.random.default_rng(500 + seed)
    img = rng.integers(0, 32, size=(int(rng.integers(1, 30)), int(rng.integers(1, 30)), 3)).astype(np.uint8)
    p, po = params_pair(debug=True, K=8, levels=32, alpha=1e-2, beta=1e-2)
    out, dbg = run_gpu(hr.Context(p), img)
    compare_to_oracle(img, out, dbg, po)


def test_binned_full_size_and_variants(hr):
    p, po = params_pair(debug=True, K=512, levels=4096, nearest_match=True)
    img = synth.low_light_image(3840, 2160, seed=synth.seed_for(3, 9), bits=12)
    out, dbg = run_gpu(hr.Context(p), img)
    compare_to_oracle(img, out, dbg, po)


def test_binned_batch_equals_single_calls_and_oracle(hr):
    import torch
    p, po = params_pair(debug=True, K=256, levels=4096)
    ctx = hr.Context(p)
    sizes = [(320, 240), (97, 33), (640, 360), (200, 301)] * 4
    imgs = [synth.low_light_image(w, h, seed=900 + i, bits=12) for i, (w, h) in enumerate(sizes)]
    outs = ctx.enhance_batch([torch.from_numpy(im).cuda() for im in imgs])
    ctx.check()
    dbgs = [ctx.debug(i) for i in range(len(imgs))]
    for i in (0, 3, 9):
        compare_to_oracle(imgs[i], outs[i].cpu().numpy(), dbgs[i], po)


def test_binned_range_and_argument_errors(hr):
    import torch
    ctx = hr.Context(hr.Params(K=256, levels=4096))
    img = np.zeros((4, 4, 3), np.uint16)
    img[1, 1, 0] = 4096
    d = torch.from_numpy(img).cuda()
    ctx.enhance(d, torch.empty_like(d))
    assert ctx.sync_status() == hr.ERR_RANGE
    with pytest.raises(hr.HistRetinexError):   # 8-bit data holds at most 256 levels
        ctx.enhance(torch.zeros((4, 4, 3), dtype=torch.uint8, device="cuda"))
    for bad in (dict(K=256, levels=100), dict(K=256, levels=128), dict(K=256, levels=8192)):
        with pytest.raises(hr.HistRetinexError):
            hr.Context(hr.Params(**bad))
