"""Continuous-batching request server for HistRetinex on one GPU.

Requests (host images) arrive over time.  The server keeps a FIFO queue and several CUDA
streams, each with its own library context (a context's workspace serves one batch at a time).
Whenever a stream is free it admits queued requests, oldest first, while the device-memory
budget allows (input + output image + per-image workspace), copies them to the device on that
stream, and launches one batched pipeline call for them; batches on different streams overlap
on the device, and requests arriving while others run are admitted as soon as a stream and
memory free up.  Results stay resident on the device.  Each request's latency runs from its
arrival time to the completion of its batch.  The statistics also give the longest iteration of
the host loop that did not wait on the device on purpose: when the serving process itself is held
up (descheduled, or stuck in the operating system), that lag says so.
"""
from __future__ import annotations

import math
import random
import time
from dataclasses import dataclass, field

import paper_2510_21100_gb300 as hr


@dataclass
class Request:
    rid: int
    arrival: float          # seconds since the start of the run
    image: object           # pinned host tensor (H, W, 3) uint8/uint16
    done: float = math.nan  # completion time (seconds since the start)
    out: object = None      # device tensor with the result (kept when keep_outputs)

    @property
    def megapixels(self) -> float:
        return self.image.shape[0] * self.image.shape[1] / 1e6


@dataclass
class ServeStats:
    completed: int
    seconds: float
    megapixels: float
    latencies_ms: list = field(default_factory=list)
    batches: int = 0
    max_batch: int = 0
    max_loop_lag_ms: float = 0.0

    def percentile(self, q: float) -> float:
        v = sorted(self.latencies_ms)
        if not v:
            return math.nan
        k = min(len(v) - 1, max(0, int(math.ceil(q / 100.0 * len(v))) - 1))
        return v[k]

    def summary(self) -> dict:
        mps = self.megapixels / self.seconds if self.seconds > 0 else 0.0
        return {"requests": self.completed, "seconds": self.seconds, "MP_per_s": mps,
                "p50_ms": self.percentile(50), "p99_ms": self.percentile(99), "batches": self.batches,
                "max_batch": self.max_batch, "max_loop_lag_ms": self.max_loop_lag_ms}


def window_stats(requests, start: float, end: float | None = None) -> dict:
    """Latency percentiles and served MP/s of the requests that arrived in [start, end) of a run (the
    first seconds of a run, while streams and caches warm up, are left out this way)."""
    sel = [r for r in requests if r.arrival >= start and (end is None or r.arrival < end)]
    if not sel:
        return {"requests": 0}
    lat = sorted((r.done - r.arrival) * 1e3 for r in sel)
    pick = lambda q: lat[min(len(lat) - 1, max(0, int(math.ceil(q / 100.0 * len(lat))) - 1))]
    span = max(r.done for r in sel) - min(r.arrival for r in sel)
    return {"requests": len(sel), "window_s": span, "MP_per_s": sum(r.megapixels for r in sel) / span,
            "p50_ms": pick(50), "p99_ms": pick(99)}


def plain_throughput(requests, params: hr.Params | None = None, streams: int = 4, partitions: int | None = None,
                     device: int = 0) -> dict:
    """The plain form on the same requests: each image copied to the device and enhanced by its own
    histretinex_enhance call, the calls going round-robin to `streams` streams of one context (calls
    on different streams overlap on the device), all issued at once.  Returns MP/s over the
    makespan (host issue to the last completion)."""
    import torch
    ctx = hr.Context(params or hr.Params(), device=device)
    if partitions is not None:
        ctx.set_tuning(partitions=partitions)
    sts = [torch.cuda.Stream(device=device) for _ in range(streams)]
    warm = requests[: min(8, len(requests))]
    for k, r in enumerate(warm):
        with torch.cuda.stream(sts[k % streams]):
            d = hr.to_device_aligned(r.image, f"cuda:{device}")
            ctx.enhance(d, hr.aligned_empty(int(d.shape[0]), int(d.shape[1]), d.dtype, f"cuda:{device}"),
                        stream=sts[k % streams])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    outs = []
    for k, r in enumerate(requests):
        st = sts[k % streams]
        with torch.cuda.stream(st):
            d = hr.to_device_aligned(r.image, f"cuda:{device}")
            o = hr.aligned_empty(int(d.shape[0]), int(d.shape[1]), d.dtype, f"cuda:{device}")
            ctx.enhance(d, o, stream=st)
            outs.append(o)
        if len(outs) > 4 * streams:  # keep device memory bounded: results are dropped as they complete
            outs.pop(0)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    ctx.check()
    ctx.close()
    mp = sum(r.megapixels for r in requests)
    return {"requests": len(requests), "seconds": el, "MP_per_s": mp / el, "streams": streams,
            "partitions": partitions}


class Server:
    def __init__(self, params: hr.Params | None = None, budget_bytes: int = 40 << 30, streams: int = 3,
                 max_batch: int = 64, device: int = 0):
        import torch
        self.torch = torch
        self.params = params or hr.Params()
        self.budget = int(budget_bytes)
        self.max_batch = max_batch
        self.device = device
        self.streams = [torch.cuda.Stream(device=device) for _ in range(streams)]
        self.ctxs = [hr.Context(self.params, device=device) for _ in range(streams)]
        for c in self.ctxs:
            # each batch has its own geometry, so a captured graph would never be replayed; and the
            # workspace of the largest batch is allocated now, not while requests wait
            c.set_tuning(use_graph=0)
            c.reserve(max_batch)
        self.slot_bytes = self.ctxs[0].workspace_bytes()  # library workspace per admitted image

    def _need(self, req: Request) -> int:
        H, W = int(req.image.shape[0]), int(req.image.shape[1])
        row = (3 * W * req.image.element_size() + 15) // 16 * 16
        return 2 * H * row + self.slot_bytes

    def run(self, requests: list[Request], keep_outputs: bool = False, poll_sleep: float = 50e-6) -> ServeStats:
        """Serves `requests` (sorted by arrival) in real time; returns the statistics.  Python's
        cyclic garbage collector is paused while serving (collected once before), so that its
        pauses do not land on request latencies."""
        import gc
        gc.collect()
        was_enabled = gc.isenabled()
        gc.disable()
        try:
            return self._run(requests, keep_outputs, poll_sleep)
        finally:
            if was_enabled:
                gc.enable()

    def _run(self, requests, keep_outputs, poll_sleep) -> ServeStats:
        torch = self.torch
        pending = sorted(requests, key=lambda r: r.arrival)
        queue: list[Request] = []
        inflight = []  # (stream index, event, [requests], bytes)
        free_streams = list(range(len(self.streams)))
        used = 0
        nxt = 0
        batches = 0
        max_b = 0
        t0 = time.perf_counter()
        done: list[Request] = []
        lag = 0.0  # longest loop iteration, less its intended sleep, that did not wait on the device
        while len(done) < len(pending):
            now = time.perf_counter() - t0
            waited = False
            while nxt < len(pending) and pending[nxt].arrival <= now:
                queue.append(pending[nxt])
                nxt += 1
            # retire finished batches
            still = []
            for s, ev, reqs, nbytes in inflight:
                if ev.query():
                    t = time.perf_counter() - t0
                    for r in reqs:
                        r.done = t
                        if not keep_outputs:
                            r.out = None
                    done.extend(reqs)
                    used -= nbytes
                    free_streams.append(s)
                else:
                    still.append((s, ev, reqs, nbytes))
            inflight = still
            # admit: one batch per free stream, oldest requests first, within the memory budget
            while free_streams and queue:
                batch, nbytes = [], 0
                while queue and len(batch) < self.max_batch and used + nbytes + self._need(queue[0]) <= self.budget:
                    r = queue.pop(0)
                    batch.append(r)
                    nbytes += self._need(r)
                if not batch:
                    if not inflight and self._need(queue[0]) > self.budget:
                        raise ValueError(f"request {queue[0].rid} needs more device memory than the budget")
                    break
                s = free_streams.pop(0)
                st = self.streams[s]
                with torch.cuda.stream(st):
                    ins = [hr.to_device_aligned(r.image, f"cuda:{self.device}") for r in batch]
                    outs = [hr.aligned_empty(int(x.shape[0]), int(x.shape[1]), x.dtype, f"cuda:{self.device}")
                            for x in ins]
                    self.ctxs[s].enhance_batch(ins, outs, stream=st)
                    ev = torch.cuda.Event()
                    ev.record(st)
                for r, o in zip(batch, outs):
                    r.out = o
                used += nbytes
                inflight.append((s, ev, batch, nbytes))
                batches += 1
                max_b = max(max_b, len(batch))
            if inflight and (not free_streams or not queue):
                if nxt >= len(pending) and not queue:
                    inflight[0][1].synchronize()  # nothing left to admit: wait for the oldest batch
                    waited = True
                else:
                    time.sleep(poll_sleep)
                    now += poll_sleep
            elif not inflight and not queue and nxt < len(pending):
                nap = min(poll_sleep, max(0.0, pending[nxt].arrival - (time.perf_counter() - t0)))
                time.sleep(nap)
                now += nap
            if not waited:
                lag = max(lag, time.perf_counter() - t0 - now)
        seconds = max((r.done for r in done), default=0.0)
        for ctx in self.ctxs:
            ctx.check()
        lat = [(r.done - r.arrival) * 1e3 for r in done]
        return ServeStats(len(done), seconds, sum(r.megapixels for r in done), lat, batches, max_b, lag * 1e3)

    def close(self):
        for c in self.ctxs:
            c.close()


def poisson_requests(pool, rate_per_s: float, seconds: float, seed: int = 0, weights=None) -> list[Request]:
    """Poisson arrivals over `seconds`; each request draws a pool image (by `weights` if given)."""
    rng = random.Random(seed)
    t, out = 0.0, []
    while True:
        t += rng.expovariate(rate_per_s)
        if t >= seconds:
            break
        img = rng.choices(pool, weights=weights, k=1)[0]
        out.append(Request(len(out), t, img))
    return out
