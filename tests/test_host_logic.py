"""Host-side logic that needs no GPU: the autotuner's cache key, the serving request stream and its
statistics, the synthetic workload shapes, and the tuning record the C ABI validates."""
import ctypes
import math

import numpy as np
import pytest

from paper_2510_21100_gb300 import autotune, serve, synth


def test_workload_key_buckets_batch_size_and_image_size():
    one = autotune.workload_key("GB300", 256, 1, [(7680, 4320)])
    assert one == "GB300|K256|b1|n1|mp32"
    # batch sizes round up to a power of two, mean megapixels to the nearest power of two
    a = autotune.workload_key("GB300", 256, 1, [(1000, 664)] * 300)
    b = autotune.workload_key("GB300", 256, 1, [(1000, 664)] * 512)
    assert a == b and "|n512|" in a
    assert autotune.workload_key("GB300", 4096, 2, [(1000, 664)] * 2).endswith("|n2|mp0.5")
    assert "|mp1|" in autotune.workload_key("GB300", 256, 1, [(1200, 800)] * 4) + "|"


def test_autotune_candidates_are_valid_tunings():
    # every candidate is accepted by histretinex_set_tuning's rules (checked here without a device)
    for v in autotune.CANDIDATES["hist_ctas_per_sm"] + autotune.CANDIDATES["apply_ctas_per_sm"]:
        assert 1 <= v <= 32
    for v in autotune.CANDIDATES["solve_cluster"]:
        assert v in (1, 2, 4, 8, 16)
    assert set(autotune.CANDIDATES["pdl"]) <= set(range(8))
    assert set(autotune.CANDIDATES["groups"]) == {1, 2}


def test_poisson_requests_are_seeded_ordered_and_at_the_rate():
    pool = [np.zeros((2, 2, 3), np.uint8), np.zeros((4, 4, 3), np.uint8)]
    a = serve.poisson_requests(pool, 400.0, 5.0, seed=3)
    b = serve.poisson_requests(pool, 400.0, 5.0, seed=3)
    assert [r.arrival for r in a] == [r.arrival for r in b]
    assert all(0.0 < x.arrival < 5.0 for x in a)
    assert all(p.arrival < q.arrival for p, q in zip(a, a[1:]))
    assert [r.rid for r in a] == list(range(len(a)))
    # 2000 expected arrivals: within five standard deviations
    assert abs(len(a) - 2000) < 5 * math.sqrt(2000)
    w = serve.poisson_requests(pool, 400.0, 5.0, seed=4, weights=[1.0, 0.0])
    assert all(r.image is pool[0] for r in w)


def test_serve_stats_percentiles_and_summary():
    st = serve.ServeStats(completed=100, seconds=2.0, megapixels=50.0, latencies_ms=list(range(1, 101)),
                          batches=40, max_batch=5)
    assert st.percentile(50) == 50 and st.percentile(99) == 99 and st.percentile(100) == 100
    s = st.summary()
    assert s["MP_per_s"] == 25.0 and s["p50_ms"] == 50 and s["p99_ms"] == 99 and s["max_batch"] == 5
    assert s["max_loop_lag_ms"] == 0.0
    assert math.isnan(serve.ServeStats(0, 1.0, 0.0).percentile(50))
    empty = serve.ServeStats(0, 0.0, 0.0).summary()
    assert empty["requests"] == 0 and empty["MP_per_s"] == 0.0 and math.isnan(empty["p99_ms"])


def test_mixed_batch_sizes_span_the_stated_range():
    sizes = synth.mixed_batch_sizes(512, 3)
    areas = np.array([w * h for w, h in sizes], dtype=np.float64)
    assert len(sizes) == 512
    assert areas.min() >= 0.97 * 320 * 240 and areas.max() <= 1.03 * 1920 * 1080
    aspects = {round(w / h, 1) for w, h in sizes}
    assert aspects <= {1.3, 1.4, 1.5, 1.7, 1.8}
    assert sizes == synth.mixed_batch_sizes(512, 3)


def test_tuning_record_matches_the_header(tmp_path):
    """The binding's ctypes record has the header's fields in order (a mismatch would shift them)."""
    import os
    import re
    import paper_2510_21100_gb300 as hr
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "include", "histretinex.h")).read()
    body = re.search(r"typedef struct \{([^}]*)\} hr_tuning;", src).group(1)
    fields = re.findall(r"int\s+(\w+);", body)
    assert [f for f, _ in hr.hr_tuning._fields_] == fields
    assert ctypes.sizeof(hr.hr_tuning) == 4 * len(fields)


def test_set_tuning_validation_without_a_device():
    """histretinex_set_tuning rejects out-of-range fields before touching a device."""
    import paper_2510_21100_gb300 as hr
    lib = hr.library()
    t = hr.hr_tuning(8, 16, 16, 1, 5, 2)
    # a null context is an argument error whatever the record says
    assert lib.histretinex_set_tuning(None, ctypes.byref(t)) == hr.ERR_INVALID_ARG


def test_prepared_batch_argument_checks():
    """PreparedBatch marshals a batch's arguments once and refuses what enhance_batch refuses."""
    import torch
    import paper_2510_21100_gb300 as hr
    a = torch.zeros((4, 6, 3), dtype=torch.uint8)
    b = torch.zeros((5, 7, 3), dtype=torch.uint8)
    pb = hr.PreparedBatch([a, b], [torch.zeros_like(a), torch.zeros_like(b)])
    assert pb.n == 2 and pb.eb == 1 and list(pb.args[2]) == [6, 7] and list(pb.args[3]) == [4, 5]
    assert list(pb.args[4]) == [18, 21]
    import pytest
    with pytest.raises(ValueError):
        hr.PreparedBatch([a], [torch.zeros_like(b)])          # output shape differs
    with pytest.raises(ValueError):
        hr.PreparedBatch([a, b.to(torch.int16)[..., :3]])      # element type
    with pytest.raises(ValueError):
        hr.PreparedBatch([], [])
