"""Failure handling on the GPU that faults nothing: an allocation the device cannot satisfy is
reported as HR_ERR_OOM and leaves the context usable (host-side failure injection)."""
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


def test_reserve_beyond_device_memory_is_oom_and_the_context_recovers(hr):
    p, po = params_pair(debug=True)
    ctx = hr.Context(p)
    img = synth.low_light_image(320, 240, seed=61)
    out, dbg = run_gpu(ctx, img)          # the context holds a workspace before the failure
    compare_to_oracle(img, out, dbg, po)
    n = (1 << 41) // ctx.workspace_bytes() + 1   # workspaces for more than 2 TB of device memory
    with pytest.raises(hr.HistRetinexError) as e:
        ctx.reserve(n)
    assert e.value.code == hr.ERR_OOM
    out2, dbg2 = run_gpu(ctx, img)        # the next call allocates what it needs again
    compare_to_oracle(img, out2, dbg2, po)
    ctx.reserve(4)                        # and a satisfiable reservation succeeds
    out3, _ = run_gpu(ctx, img)
    assert (out3 == out).all()
