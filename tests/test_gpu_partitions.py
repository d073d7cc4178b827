"""Single-image calls on SM partitions (green contexts): the solves of calls run in 16-SM
partitions, 16 / partition_cluster at once in each, while other calls' pixel passes run in the
rest, for calls issued on different streams.  Each image's result must be bit-identical to the
same image run unpartitioned and alone with solve_cluster = partition_cluster, whatever else is in
flight; the context's ring of workspace slots must order slot reuse by itself."""
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


@pytest.mark.parametrize("pc", [4, 16, 2])
def test_partitioned_call_matches_unpartitioned_and_oracle(hr, pc):
    p, po = params_pair(debug=True)
    part = hr.Context(p)
    part.set_tuning(partition_cluster=pc)
    plain = hr.Context(p)
    plain.set_tuning(partitions=0, solve_cluster=pc)
    for (W, H) in ((600, 400), (1, 1), (257, 129), (3840, 2160)):
        img = synth.low_light_image(W, H, seed=W + 3 * H)
        out_p, dbg_p = run_gpu(part, img)
        out_u, dbg_u = run_gpu(plain, img)
        assert np.array_equal(out_p, out_u)
        for k in ("S", "G", "R", "L", "T", "lut"):
            assert np.array_equal(dbg_p[k], dbg_u[k]), k
        compare_to_oracle(img, out_p, dbg_p, po)
    parts, sms = part.partition_info()
    assert parts == 2 and 0 < sms < 152, (parts, sms)
    assert plain.partition_info()[0] == 0


@pytest.mark.parametrize("parts,pc,n_streams", [(1, 4, 3), (0, 4, 3), (3, 16, 3), (2, 2, 8), (1, 1, 5)])
def test_overlapped_calls_on_several_streams_equal_each_image_alone(hr, parts, pc, n_streams):
    """Twelve images of mixed sizes (three of them 7680x4320) issued round-robin on several streams,
    some in place: every output equals the image's own single call run alone (the ring of slots
    orders slot reuse across streams with or without SM partitions, with one or several solves at
    once in each partition)."""
    import torch
    sizes = [(7680, 4320), (640, 480), (1920, 1080), (333, 217), (7680, 4320), (1000, 664),
             (97, 33), (3840, 2160), (1, 1), (7680, 4320), (2047, 1031), (600, 400)]
    imgs = [synth.low_light_image(w, h, seed=8800 + i) for i, (w, h) in enumerate(sizes)]
    ref = hr.Context(hr.Params())
    ref.set_tuning(partitions=0, solve_cluster=pc)
    want = []
    for im in imgs:
        d = hr.to_device_aligned(im)
        want.append(ref.enhance(d, hr.aligned_empty(im.shape[0], im.shape[1])).cpu().numpy())
    ref.check()
    ctx = hr.Context(hr.Params())
    ctx.set_tuning(partitions=parts, partition_cluster=pc, solve_cluster=pc)
    streams = [torch.cuda.Stream() for _ in range(n_streams)]
    ins = [hr.to_device_aligned(im) for im in imgs]
    torch.cuda.synchronize()
    outs = []
    for i, d in enumerate(ins):
        s = streams[i % n_streams]
        with torch.cuda.stream(s):
            o = d if i % 4 == 3 else hr.aligned_empty(d.shape[0], d.shape[1])  # every fourth in place
            ctx.enhance(d, o, stream=s)
            outs.append(o)
    torch.cuda.synchronize()
    ctx.check()
    for i, o in enumerate(outs):
        assert np.array_equal(o.cpu().numpy(), want[i]), (i, sizes[i])
    assert ctx.partition_info()[0] == parts


def test_partition_count_can_change_between_calls(hr):
    p, po = params_pair(debug=True)
    ctx = hr.Context(p)
    ctx.set_tuning(solve_cluster=4, partition_cluster=4)  # (the unpartitioned call solves alike)
    img = synth.low_light_image(800, 600, seed=42)
    outs = []
    for parts in (1, 3, 0, 2):
        ctx.set_tuning(partitions=parts)
        out, dbg = run_gpu(ctx, img)
        outs.append(out)
        assert ctx.partition_info()[0] == parts
    assert all(np.array_equal(o, outs[0]) for o in outs)
    compare_to_oracle(img, outs[0], dbg, po)


@pytest.mark.parametrize("W,H", [(7680, 4320), (3840, 2160)])
def test_benchmark_configuration_full_size_against_oracle(hr, W, H):
    """The launch configuration the benchmark times for a stream of large images (one 16-SM solve
    partition running four 4-CTA solves at once): its three images (the workload image and two
    mirrored copies), checked pixel for pixel against the oracle."""
    import sys, os
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    p, po = params_pair(debug=True)
    ctx = hr.Context(p)
    ctx.set_tuning(partitions=1, partition_cluster=4)
    for img in bench.make_images(W, H):
        out, dbg = run_gpu(ctx, img)
        compare_to_oracle(img, out, dbg, po)
    assert ctx.partition_info()[0] == 1
