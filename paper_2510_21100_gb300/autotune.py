"""Launch-shape autotuner for the HistRetinex pipeline.

Times candidate launch shapes (CTAs per SM of the two pixel passes, cluster size of a single
image's solve, which kernels are programmatic dependent launches) on the caller's own images with CUDA events, keeps the fastest, applies it to the
context and caches it in a JSON file keyed by GPU, K, element size, batch-size bucket and
image-size bucket.  Coordinate descent: one field at a time, the others held at their best.
"""
from __future__ import annotations

import json
import math
import os

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "histretinex", "tuning.json")

CANDIDATES = {
    "hist_ctas_per_sm": (2, 4, 8),
    "apply_ctas_per_sm": (4, 8, 16),
    "solve_cluster": (4, 8, 16),
    "pdl": (0, 1, 5),  # dependent launches: none, histogram pass, histogram and apply passes
    "groups": (1, 2),  # a large batch as one group or two overlapping ones
}


def workload_key(device_name: str, K: int, elem_bytes: int, sizes) -> str:
    n = len(sizes)
    mp = sum(w * h for w, h in sizes) / max(n, 1) / 1e6
    nb = 1 if n == 1 else 2 ** math.ceil(math.log2(n))
    mb = 2 ** round(math.log2(max(mp, 1e-3)))
    return f"{device_name}|K{K}|b{elem_bytes}|n{nb}|mp{mb:g}"


def _time(ctx, ins, outs, reps, torch):
    if len(ins) == 1:
        run = lambda: ctx.enhance(ins[0], outs[0])
    else:
        from . import PreparedBatch
        pb = PreparedBatch(ins, outs)  # (the batch's arguments marshalled once: time the GPU, not Python)
        run = lambda: ctx.enhance_batch(pb)
    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(ctx, ins, outs=None, reps: int = 5, cache_path: str | None = DEFAULT_CACHE, use_cache: bool = True):
    """Tunes ctx for the images `ins` (device tensors); returns (tuning dict, ms per call)."""
    import torch
    if outs is None:
        outs = [torch.empty_like(t) for t in ins]
    sizes = [(int(t.shape[1]), int(t.shape[0])) for t in ins]
    key = workload_key(torch.cuda.get_device_name(ctx.device), ctx.params.K, ins[0].element_size(), sizes)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        ctx.set_tuning(**cache[key]["tuning"])
        return cache[key]["tuning"], cache[key]["ms"]
    best = ctx.tuning()
    best_ms = _time(ctx, ins, outs, reps, torch)
    fields = ["hist_ctas_per_sm", "apply_ctas_per_sm"] + (["solve_cluster"] if len(ins) == 1 else ["groups"]) + ["pdl"]
    for field in fields:
        for v in CANDIDATES[field]:
            if v == best[field]:
                continue
            trial = dict(best, **{field: v})
            ctx.set_tuning(**trial)
            ms = _time(ctx, ins, outs, reps, torch)
            if ms < best_ms:
                best, best_ms = trial, ms
        ctx.set_tuning(**best)
    if cache_path:
        cache[key] = {"tuning": best, "ms": best_ms}
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return best, best_ms
