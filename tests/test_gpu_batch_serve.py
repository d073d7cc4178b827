"""GPU tests of the batched form (CUDA graph replay, launch shapes, autotuner) and the server."""
import numpy as np
import pytest

from gpu_util import compare_to_oracle, params_pair
from paper_2510_21100_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hr():
    import paper_2510_21100_gb300 as hr
    from paper_2510_21100_gb300 import build
    build.build()
    return hr


def mixed_images(n, seed=0):
    sizes = synth.mixed_batch_sizes(n, seed, min_wh=(64, 48), max_wh=(640, 480))
    return [synth.low_light_image(w, h, seed=seed * 1000 + i) for i, (w, h) in enumerate(sizes)]


def run_batch(ctx, imgs):
    import torch
    ins = [torch.from_numpy(im).cuda() for im in imgs]
    outs = ctx.enhance_batch(ins)
    ctx.check()
    return [o.cpu().numpy() for o in outs]


def test_graph_replay_equals_direct_launches(hr):
    imgs = mixed_images(9, seed=1)
    p, po = params_pair(debug=True)
    g = hr.Context(p)
    d = hr.Context(p)
    d.set_tuning(use_graph=0)
    first = run_batch(g, imgs)       # captures the graph
    second = run_batch(g, imgs)      # replays it
    direct = run_batch(d, imgs)
    for a, b, c in zip(first, second, direct):
        assert np.array_equal(a, b) and np.array_equal(a, c)
    compare_to_oracle(imgs[3], first[3], g.debug(3), po)


def test_graph_is_recaptured_when_geometry_changes(hr):
    ctx = hr.Context(hr.Params())
    a = mixed_images(4, seed=2)
    b = mixed_images(6, seed=3)
    ra = run_batch(ctx, a)
    rb = run_batch(ctx, b)
    ra2 = run_batch(ctx, a)
    for x, y in zip(ra, ra2):
        assert np.array_equal(x, y)
    ref = hr.Context(hr.Params())
    ref.set_tuning(use_graph=0)
    for x, y in zip(rb, run_batch(ref, b)):
        assert np.array_equal(x, y)


def test_launch_shapes_do_not_change_results(hr):
    imgs = mixed_images(5, seed=4)
    ctx = hr.Context(hr.Params())
    base = run_batch(ctx, imgs)
    for t in (dict(hist_ctas_per_sm=2, apply_ctas_per_sm=16), dict(hist_ctas_per_sm=1, apply_ctas_per_sm=1)):
        ctx.set_tuning(**t)
        for x, y in zip(base, run_batch(ctx, imgs)):
            assert np.array_equal(x, y)


def test_invalid_tuning_rejected(hr):
    ctx = hr.Context(hr.Params())
    for bad in (dict(hist_ctas_per_sm=0), dict(apply_ctas_per_sm=33), dict(solve_cluster=3), dict(use_graph=2)):
        with pytest.raises(hr.HistRetinexError):
            ctx.set_tuning(**bad)


def test_single_image_cluster_sizes_agree(hr):
    import torch
    from gpu_util import assert_close
    img = synth.low_light_image(800, 600, seed=9)
    p, po = params_pair(debug=True)
    ctx = hr.Context(p)
    res = {}
    for C in (1, 4, 16):
        ctx.set_tuning(solve_cluster=C)
        d = torch.from_numpy(img).cuda()
        out = ctx.enhance(d).cpu().numpy()
        ctx.check()
        res[C] = (out, ctx.debug(0))
    for C in (1, 4):
        assert np.array_equal(res[C][0], res[16][0])
        assert np.array_equal(res[C][1]["lut"], res[16][1]["lut"])
        for k in ("R", "L", "T"):
            assert_close(res[C][1][k], res[16][1][k], k)
    compare_to_oracle(img, res[16][0], res[16][1], po)


def test_autotune_selects_a_valid_tuning(hr, tmp_path):
    import torch
    from paper_2510_21100_gb300 import autotune
    imgs = mixed_images(6, seed=5)
    ins = [torch.from_numpy(im).cuda() for im in imgs]
    ctx = hr.Context(hr.Params())
    best, ms = autotune.autotune(ctx, ins, reps=2, cache_path=str(tmp_path / "t.json"))
    assert ms > 0 and best["hist_ctas_per_sm"] in autotune.CANDIDATES["hist_ctas_per_sm"] + (8,)
    again, ms2 = autotune.autotune(ctx, ins, reps=2, cache_path=str(tmp_path / "t.json"))
    assert again == best and ms2 == ms  # served from the cache
    assert ctx.tuning() == best


def test_server_results_identical_alone_and_in_the_mix(hr):
    """Continuous batching: every request's result equals the result of the same image served alone."""
    import torch
    from paper_2510_21100_gb300 import serve
    pool_np = mixed_images(6, seed=6)
    pool = [torch.from_numpy(im).pin_memory() for im in pool_np]
    srv = serve.Server(hr.Params(), budget_bytes=1 << 30, streams=3, max_batch=8)
    reqs = serve.poisson_requests(pool, rate_per_s=400.0, seconds=0.5, seed=1)
    stats = srv.run(reqs, keep_outputs=True)
    assert stats.completed == len(reqs) and stats.batches >= 1
    assert all(np.isfinite(r.done) and r.done >= r.arrival for r in reqs)
    alone = {}
    for k, img in enumerate(pool):
        r = serve.Request(0, 0.0, img)
        srv.run([r], keep_outputs=True)
        alone[k] = r.out.cpu().numpy()
    for r in reqs:
        k = next(i for i, p in enumerate(pool) if p is r.image)
        assert np.array_equal(r.out.cpu().numpy(), alone[k])
    s = stats.summary()
    assert s["p99_ms"] >= s["p50_ms"] > 0 and s["max_loop_lag_ms"] >= 0
    srv.close()


def test_server_respects_the_memory_budget(hr):
    import torch
    from paper_2510_21100_gb300 import serve
    img = torch.from_numpy(synth.low_light_image(640, 480, seed=3)).pin_memory()
    srv = serve.Server(hr.Params(), budget_bytes=1, streams=1)
    with pytest.raises(ValueError):
        srv.run([serve.Request(0, 0.0, img)])
    need = srv._need(serve.Request(0, 0.0, img))
    srv2 = serve.Server(hr.Params(), budget_bytes=2 * need, streams=2, max_batch=8)
    reqs = [serve.Request(i, 0.0, img) for i in range(6)]
    st = srv2.run(reqs)
    assert st.completed == 6 and st.max_batch <= 2
    st0 = srv2.run([])
    assert st0.completed == 0 and st0.batches == 0 and st0.summary()["MP_per_s"] == 0.0
    srv.close(); srv2.close()


def test_reserve_then_batches_up_to_the_reserved_size(hr):
    """histretinex_reserve sizes the workspace up front; batches up to that size then run as usual."""
    import torch
    import paper_2510_21100_gb300 as hrm
    ctx = hrm.Context(hrm.Params())
    ctx.reserve(4)
    imgs = [torch.from_numpy(synth.low_light_image(64 + 16 * i, 48, seed=600 + i)).cuda() for i in range(4)]
    ref = [ctx.enhance(x) for x in imgs]
    outs = ctx.enhance_batch(imgs)
    ctx.check()
    for a, b in zip(ref, outs):
        assert torch.equal(a, b)
    with pytest.raises(hrm.HistRetinexError):
        ctx.reserve(0)


def test_host_sequence_equals_device_path(hr):
    """histretinex_enhance_host_many: each host image gets exactly the device path's result."""
    import torch
    import paper_2510_21100_gb300 as hrm
    ctx = hrm.Context(hrm.Params())
    sizes = [(320, 240), (96, 64), (640, 360), (640, 360), (33, 17)]
    imgs = [synth.low_light_image(w, h, seed=700 + i) for i, (w, h) in enumerate(sizes)]
    hins = [torch.from_numpy(im).pin_memory() for im in imgs]
    outs = ctx.enhance_host_many(hins)
    ctx.check()
    for im, o in zip(imgs, outs):
        ref = ctx.enhance(torch.from_numpy(im).cuda()).cpu()
        assert torch.equal(o, ref)
    outs2 = ctx.enhance_host_many(hins[:1])  # a second call reuses the buffers
    assert torch.equal(outs2[0], outs[0])


def test_two_group_batch_equals_one_group(hr):
    """A graph-replayed batch of 64 images or more runs as two groups on two streams (the second
    group's histogram pass after the first's); with one CTA per image either way (here 320
    images), every image gets the same bits as in a single group, and matches the oracle."""
    import torch
    sizes = synth.mixed_batch_sizes(320, 71, min_wh=(24, 18), max_wh=(200, 150))
    imgs = [synth.low_light_image(w, h, seed=7100 + i) for i, (w, h) in enumerate(sizes)]
    ins = [torch.from_numpy(im).cuda() for im in imgs]
    p, po = params_pair(debug=True)
    two = hr.Context(p)
    one = hr.Context(p)
    one.set_tuning(groups=1)
    assert two.tuning()["groups"] == 2
    o2 = two.enhance_batch(ins)
    two.check()
    o1 = one.enhance_batch(ins)
    one.check()
    for i in range(len(imgs)):
        assert np.array_equal(o1[i].cpu().numpy(), o2[i].cpu().numpy()), i
    for i in (0, 161, 319):
        d1, d2 = one.debug(i), two.debug(i)
        for k in ("S", "G", "R", "L", "T", "lut"):
            assert np.array_equal(d1[k], d2[k]), (i, k)
        compare_to_oracle(imgs[i], o2[i].cpu().numpy(), d2, po)
    o2b = two.enhance_batch(ins)  # graph replay
    two.check()
    for i in (3, 200):
        assert np.array_equal(o2b[i].cpu().numpy(), o2[i].cpu().numpy())


def test_prepared_batch_equals_the_list_call(hr):
    """A batch whose arguments were marshalled once (PreparedBatch), called twice, gives the pixels
    the same images get through the list form of enhance_batch."""
    import torch
    imgs = mixed_images(7, seed=11)
    ctx = hr.Context(hr.Params())
    ins = [torch.from_numpy(im).cuda() for im in imgs]
    want = [o.cpu().numpy() for o in ctx.enhance_batch(ins)]
    pb = hr.PreparedBatch(ins)
    for _ in range(2):
        got = ctx.enhance_batch(pb)
        ctx.check()
        for a, b in zip(got, want):
            assert np.array_equal(a.cpu().numpy(), b)
