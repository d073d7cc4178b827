"""GPU parity at the full sizes of the batched and reduced-precision workloads, in the launch
configuration the benchmark times (graph replay, two overlapping groups; one CTA per image).

Batched: 512 mixed 8-bit images, areas log-uniform between 320x240 and 1920x1080, cropped from 16
generated 1920x1248 images as the benchmark does.  Every image of the batch call must equal the
same image run alone, pixel for pixel, and a sample spread over the sizes must equal the FP64
oracle's output pixel for pixel (the plain form's bar; double-float is held to it as well).

Reduced precision: 1024 12-bit 1000x664 images (16 generated images, repeated), K = 4096, FP32
solve sums, in one batch call.  Repeats of one image must give identical pixels wherever they sit
in the batch, and four images must meet the stated tolerances against the oracle (enhanced
histogram within 1e-4 per bin, LUT entries equal except within one level at near-ties).
"""
import concurrent.futures as cf

import numpy as np
import pytest

import oracle
from paper_2510_21100_gb300 import synth
from test_gpu_precision import check_precision

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hr():
    import paper_2510_21100_gb300 as hr
    from paper_2510_21100_gb300 import build
    build.build()
    return hr


def mixed_batch(hr, n=512, seed=3):
    """The batched workload's images as device tensors (16-byte aligned rows) and their host copies."""
    import torch
    sizes = synth.mixed_batch_sizes(n, seed)
    rng = np.random.default_rng(seed)
    bases = []
    for i in range(16):
        lo, hi = synth.illumination_range(seed * 100 + i)
        bases.append(synth.low_light_image(1920, 1248, seed=synth.seed_for(2, i), illum_lo=lo, illum_hi=hi))
    hosts, dins = [], []
    for k, (w, h) in enumerate(sizes):
        y, x = int(rng.integers(0, 1248 - h + 1)), int(rng.integers(0, 1920 - w + 1))
        im = np.ascontiguousarray(bases[k % 16][y:y + h, x:x + w])
        hosts.append(im)
        t = hr.aligned_empty(h, w)
        t.copy_(torch.from_numpy(im))
        dins.append(t)
    return sizes, hosts, dins


@pytest.mark.parametrize("precision", ["df64", "fp64"])
def test_batched_workload_512_mixed_images(hr, precision):
    import torch
    prec = {"df64": hr.PREC_DF64, "fp64": hr.PREC_FP64}[precision]
    sizes, hosts, dins = mixed_batch(hr)
    douts = [hr.aligned_empty(h, w) for (w, h) in sizes]
    ctx = hr.Context(hr.Params(precision=prec))
    ctx.set_tuning(use_graph=1, groups=2)
    pb = hr.PreparedBatch(dins, douts)
    for _ in range(2):  # (the second call replays the captured graph)
        ctx.enhance_batch(pb)
    torch.cuda.synchronize()
    ctx.check()
    batch = [d.cpu().numpy() for d in douts]
    # every image as a single FP64 call
    single = hr.Context(hr.Params())
    for k in range(len(sizes)):
        o = hr.aligned_empty(sizes[k][1], sizes[k][0])
        single.enhance(dins[k], o)
        assert np.array_equal(o.cpu().numpy(), batch[k]), (k, sizes[k])
    single.check()
    # a sample spread over the sizes against the oracle
    order = np.argsort([w * h for w, h in sizes])
    pick = sorted(set(int(order[i]) for i in np.linspace(0, len(order) - 1, 8).round().astype(int)))
    po = oracle.Params(K=256)
    with cf.ThreadPoolExecutor(4) as ex:
        refs = list(ex.map(lambda k: oracle.enhance(hosts[k], po), pick))
    for k, ref in zip(pick, refs):
        assert np.array_equal(batch[k], ref.out), (k, sizes[k])


def test_precision_workload_1024_images(hr):
    import torch
    pool = [synth.low_light_image(1000, 664, seed=synth.seed_for(3, i), bits=12) for i in range(16)]
    dpool = [torch.from_numpy(im).cuda() for im in pool]
    n = 1024
    ins = []
    for i in range(n):
        t = hr.aligned_empty(664, 1000, dtype=torch.uint16)
        t.copy_(dpool[i % 16])
        ins.append(t)
    outs = [hr.aligned_empty(664, 1000, dtype=torch.uint16) for _ in range(n)]
    ctx = hr.Context(hr.Params(K=4096, precision=hr.PREC_FP32))
    ctx.enhance_batch(hr.PreparedBatch(ins, outs))
    torch.cuda.synchronize()
    ctx.check()
    first = [outs[i].cpu().numpy() for i in range(16)]
    for i in range(16, n, 37):  # repeats anywhere in the batch: the same pixels
        assert np.array_equal(outs[i].cpu().numpy(), first[i % 16]), i
    assert np.array_equal(outs[n - 1].cpu().numpy(), first[(n - 1) % 16])
    # the path of each image (one CTA, FP32) with its intermediates, against the oracle
    dbg = hr.Context(hr.Params(K=4096, precision=hr.PREC_FP32, debug=True))
    dbg.set_tuning(solve_cluster=1)
    douts = dbg.enhance_batch([hr.to_device_aligned(im) for im in pool[:4]],
                              [hr.aligned_empty(664, 1000, dtype=torch.uint16) for _ in range(4)])
    dbg.check()
    with cf.ThreadPoolExecutor(4) as ex:
        refs = list(ex.map(lambda im: oracle.enhance(im, oracle.Params(K=4096)), pool[:4]))
    for i in range(4):
        o = douts[i].cpu().numpy()
        assert np.array_equal(o, first[i]), i
        check_precision(pool[i], o, dbg.debug(i), 4096, ref=refs[i])
