"""Contexts used from several host threads at once, each thread with a context of its own (a single
context must not be shared between threads).  The contexts run different K (256 on 8-bit data, 64 on
6-bit data in 8-bit pixels, 4096 on 12-bit data), so their kernels take different amounts of shared
memory; the library keeps each kernel's shared-memory limit at one value for every call, and caches
its cluster limits per K, so concurrent calls cannot disturb each other.  Every result of every
repeated call must equal the same call made alone, pixel for pixel.
"""
import threading

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


def test_contexts_on_three_host_threads(hr):
    import torch
    jobs = [(256, synth.low_light_image(320, 200, seed=9300)),
            (64, synth.low_light_image(240, 160, seed=9301) >> 2),
            (4096, synth.low_light_image(200, 133, seed=9302, bits=12))]
    alone = []
    for K, img in jobs:
        ctx = hr.Context(hr.Params(K=K))
        alone.append(ctx.enhance(torch.from_numpy(img).cuda()).cpu().numpy())
        ctx.check()
        ctx.close()
    errors = []

    def worker(k):
        try:
            K, img = jobs[k]
            ctx = hr.Context(hr.Params(K=K))
            st = torch.cuda.Stream()
            din = torch.from_numpy(img).cuda()
            dout = torch.empty_like(din)
            for it in range(30):
                with torch.cuda.stream(st):
                    ctx.enhance(din, dout, stream=st)
                st.synchronize()
                if not np.array_equal(dout.cpu().numpy(), alone[k]):
                    errors.append((K, it))
                    break
            ctx.check()
            ctx.close()
        except Exception as e:  # (reported on the main thread)
            errors.append((jobs[k][0], repr(e)))

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(len(jobs))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
