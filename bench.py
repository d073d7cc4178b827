#!/usr/bin/env python
"""Benchmark of the HistRetinex GB300 pipeline.

One step = one full pass of the per-image pipeline (histograms, Algorithm 1, Eq. 20 target,
matching LUT, apply) over the plain-method workload: a 7680x4320 uint8 synthetic low-light
image, K = 256, 10 iterations.  Three distinct input/output buffer pairs rotate so every step
reads an image that is not L2-resident (3 x 199 MB > 129 MB L2).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "enhanced MP/s (RGB in->out), plain single image"
UNIT = "MP/s"


# DRAM bytes (read + write) per launch of each kernel at 7680x4320, K = 256, from one ncu capture
# of the current kernels (profiles/pipeline_7680x4320_launches.md); the apply's writes still in L2
# when the kernel ends are not counted there.
PROFILED_DRAM_BYTES = {"hist_u8s_kernel": 104_434_176, "solve_kernel<double>": 261_376, "apply_u8v_kernel": 145_962_240}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--width", type=int, default=7680)
    ap.add_argument("--height", type=int, default=4320)
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, per-size and CPU-baseline legs")
    ap.add_argument("--streams", type=int, default=16, help="CUDA streams the timed steps go to, round-robin")
    ap.add_argument("--partitions", type=int, default=1, help="16-SM solve partitions of single-image calls")
    ap.add_argument("--partition-cluster", type=int, default=4,
                    help="CTAs per solve of a partitioned call (each partition runs 16 / this many at once)")
    ap.add_argument("--serving-seconds", type=float, default=0.0,
                    help="long serving runs: seconds per rate (first 5 s left out of the statistics)")
    ap.add_argument("--serving-rates", default="800,1600", help="request rates of the long serving runs")
    ap.add_argument("--only", default="",
                    help="comma-separated extra legs to run (e2e, per_size, batched, serving, precision, gamma, "
                         "ablation, cpu); default all")
    return ap.parse_args()


def workload_config(W, H, streams=1, partitions=0, partition_cluster=16):
    return {"workload": f"plain single image {W}x{H} uint8 RGB, K=256, T=10 fixed iterations, gamma=2.2, "
                        f"alpha=beta=1e-3, FP64 solve; one histretinex_enhance call per step, steps round-robin on "
                        f"{streams} CUDA stream(s); 3 rotating input/output buffers (inputs larger than L2 in aggregate)",
            "image": f"{W}x{H}", "K": 256, "iterations": 10, "elem": "uint8", "l2": "rotating inputs > L2",
            "streams": streams, "solve_partitions": partitions, "partition_cluster": partition_cluster}


def make_images(W, H, rank=0):
    """This rank's seeded synthetic image plus two mirrored copies (distinct buffers for L2 rotation);
    every rank draws its own image (rank 0's is the single-GPU workload image)."""
    import numpy as np
    from paper_2510_21100_gb300 import shard, synth
    img = synth.low_light_image(W, H, seed=shard.rank_image_seeds(rank, 1)[0])
    return [img, np.ascontiguousarray(img[:, ::-1]), np.ascontiguousarray(img[::-1])]


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None

    def __enter__(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        pass

    def result(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "note": "nvidia-smi unavailable"}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def cpu_oracle_rate(imgs_np, seconds=10.0, rows=None):
    """The FP64 C oracle on the host cores: MP/s over a bounded sample, single thread."""
    import oracle
    img = imgs_np[0] if rows is None else imgs_np[0][:rows]
    p = oracle.Params()
    oracle.enhance(img[:64, :64], p)  # compile and load outside the timing
    done, t0 = 0, time.perf_counter()
    while True:
        oracle.enhance(img, p)
        done += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    mp = img.shape[0] * img.shape[1] * done / 1e6
    return mp / el, done, img.shape


def cpu_oracle_batch_rate(seconds=10.0, n_threads=None):
    """The FP64 C oracle over images on all host cores (one image per thread at a time; ctypes
    releases the GIL during each call): MP/s on mixed-size images of the batched workload."""
    import concurrent.futures as cf
    import oracle
    from paper_2510_21100_gb300 import synth
    n_threads = n_threads or os.cpu_count() or 1
    sizes = synth.mixed_batch_sizes(4 * n_threads, 3)
    imgs = [synth.low_light_image(w, h, seed=synth.seed_for(2, i)) for i, (w, h) in enumerate(sizes)]
    p = oracle.Params()
    oracle.enhance(imgs[0][:32, :32], p)
    done_mp, t0 = 0.0, time.perf_counter()
    with cf.ThreadPoolExecutor(n_threads) as ex:
        while time.perf_counter() - t0 < seconds:
            list(ex.map(lambda im: oracle.enhance(im, p), imgs))
            done_mp += sum(im.shape[0] * im.shape[1] for im in imgs) / 1e6
    return done_mp / (time.perf_counter() - t0), n_threads, len(imgs)


def run_reference(a, rank, world):
    """The oracle as the reference arm: each step one bounded sample of the workload on the host."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2510_21100_gb300 import synth
    W, H = a.width, a.height
    rows = max(1, min(H, (8_300_000 + W - 1) // W))  # about 8.3 MP per step: a few seconds per step
    img = synth.low_light_image(W, H, seed=synth.seed_for(1, 0))[:rows]
    p = oracle.Params()
    oracle.enhance(img[:32, :32], p)
    for _ in range(a.warmup):
        oracle.enhance(img, p)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        oracle.enhance(img, p)
    el = time.perf_counter() - t0
    v = rows * W * a.steps / 1e6 / el
    sample = f"rows 0-{rows - 1} of the {W}x{H} image ({rows * W / 1e6:.2f} MP) per step, single-threaded FP64 C oracle"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": el * 1000 / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(W, H, a.streams, a.partitions, a.partition_cluster),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batched_leg(torch, hr, local, precision, n_imgs=512, steps=10, warmup=3, seed=3):
    """The batched form: n mixed-size 8-bit images (areas log-uniform in 320x240 .. 1920x1080, aspect
    4:3/16:9/3:2) per graph-replayed batch call.  Images are crops of 16 generated 1920x1248 images
    (the largest 4:3 image of that area is 1663x1247).  precision: the solve's arithmetic (FP64, or
    double-float, which the GPU tests hold to the same tolerance)."""
    import numpy as np
    from paper_2510_21100_gb300 import autotune, synth
    sizes = synth.mixed_batch_sizes(n_imgs, seed)
    rng = np.random.default_rng(seed)
    bases = []
    for i in range(16):
        lo, hi = synth.illumination_range(seed * 100 + i)
        bases.append(torch.from_numpy(synth.low_light_image(1920, 1248, seed=synth.seed_for(2, i),
                                                            illum_lo=lo, illum_hi=hi)).cuda())
    ins = []
    for k, (w, h) in enumerate(sizes):
        b = bases[k % 16]
        y, x = int(rng.integers(0, 1248 - h + 1)), int(rng.integers(0, 1920 - w + 1))
        t = hr.aligned_empty(h, w, device=f"cuda:{local}")
        t.copy_(b[y:y + h, x:x + w])
        ins.append(t)
    outs = [hr.aligned_empty(int(t.shape[0]), int(t.shape[1]), device=f"cuda:{local}") for t in ins]
    ctx = hr.Context(hr.Params(precision=precision), device=local)
    tune, _ = autotune.autotune(ctx, ins, outs, reps=2, cache_path=None)
    mp = sum(w * h for w, h in sizes) / 1e6
    pb = hr.PreparedBatch(ins, outs)  # (arguments marshalled once, as a C caller passes its arrays)
    for _ in range(warmup):
        ctx.enhance_batch(pb)
    torch.cuda.synchronize()
    l0 = ctx.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        ctx.enhance_batch(pb)
    e1.record()
    torch.cuda.synchronize()
    ctx.check()
    ms = e0.elapsed_time(e1) / steps
    byts = 3 * 3 * mp * 1e6  # read for the histograms, read + write for the apply
    arith = {hr.PREC_FP64: "FP64", hr.PREC_DF64: "double-float"}[precision]
    # the same images, one histretinex_enhance call each, round-robin on 16 streams (unpartitioned:
    # the fastest single-call form for images of this size)
    ns = 16
    single = hr.Context(hr.Params(precision=precision), device=local)
    single.set_tuning(partitions=0)
    sts = [torch.cuda.current_stream()] + [torch.cuda.Stream() for _ in range(ns - 1)]
    for k in range(8):
        single.enhance(ins[k], outs[k], stream=sts[k % ns])
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(sts[0])
    for st in sts[1:]:
        st.wait_event(f0)
    reps = 3
    for _ in range(reps):
        for k in range(n_imgs):
            single.enhance(ins[k], outs[k], stream=sts[k % ns])
    for st in sts[1:]:
        ev = torch.cuda.Event()
        ev.record(st)
        sts[0].wait_event(ev)
    f1.record(sts[0])
    torch.cuda.synchronize()
    single.check()
    ms_single = f0.elapsed_time(f1) / reps
    single.close()
    return {"workload": f"{n_imgs} mixed uint8 images, {mp:.1f} MP per batch call, K=256, T=10, {arith} solve",
            "images": n_imgs,
            "MP": mp, "ms_per_batch": ms, "MP_per_s": mp / (ms / 1e3), "tuning": tune,
            "gpu_launches_per_batch": (ctx.kernel_launches() - l0) / steps, "pipeline_GBps": byts / (ms / 1e3) / 1e9,
            "same_images_single_calls": {"ms": ms_single, "MP_per_s": mp / (ms_single / 1e3),
                                         "how": "one histretinex_enhance per image, round-robin on 16 streams, "
                                                "unpartitioned"}}


def precision_leg(torch, hr, local, n_imgs=1024, steps=2, warmup=1):
    """The reduced-precision form: 1024 1000x664 12-bit (uint16) images (16 generated images,
    repeated) in one batch call, K=4096, FP32 solve sums."""
    from paper_2510_21100_gb300 import synth
    pool = [torch.from_numpy(synth.low_light_image(1000, 664, seed=synth.seed_for(3, i), bits=12)).cuda()
            for i in range(16)]
    ins = []
    for i in range(n_imgs):
        t = hr.aligned_empty(664, 1000, dtype=torch.uint16, device=f"cuda:{local}")
        t.copy_(pool[i % 16])
        ins.append(t)
    outs = [hr.aligned_empty(664, 1000, dtype=torch.uint16, device=f"cuda:{local}") for _ in ins]
    ctx = hr.Context(hr.Params(K=4096, precision=hr.PREC_FP32, stage_timing=False), device=local)
    pb = hr.PreparedBatch(ins, outs)
    for _ in range(warmup):
        ctx.enhance_batch(pb)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        ctx.enhance_batch(pb)
    e1.record()
    torch.cuda.synchronize()
    ctx.check()
    ms = e0.elapsed_time(e1) / steps
    mp = 1000 * 664 * n_imgs / 1e6
    ctx.close()
    # accuracy of the FP32 form against the FP64 oracle on four of the images: max relative error of
    # the enhanced histogram (per bin, relative to max(T, 1 pixel)) and LUT entries that differ, with
    # how many of those lie where the oracle's own decision is within 1e-4 of a tie
    import concurrent.futures as cf
    import numpy as np
    import oracle
    hosts = [synth.low_light_image(1000, 664, seed=synth.seed_for(3, i), bits=12) for i in range(4)]
    with cf.ThreadPoolExecutor(4) as ex:
        refs = list(ex.map(lambda im: oracle.enhance(im, oracle.Params(K=4096)), hosts))
    errs, mism, mism_tie = [], 0, 0
    c32 = hr.Context(hr.Params(K=4096, precision=hr.PREC_FP32, debug=True), device=local)
    c32.set_tuning(solve_cluster=1)  # one CTA per image, as in the 1024-image batch
    c32.enhance_batch([p.clone() for p in pool[:4]])
    for i, ref in enumerate(refs):
        d32 = c32.debug(i)
        errs.append(float(np.max(np.abs(d32["T"] - ref.T) / np.maximum(ref.T, 1.0))))
        diff = np.nonzero(d32["lut"].astype(np.int64) != ref.lut.astype(np.int64))[0]
        mism += int(diff.size)
        N = float(ref.S.sum())
        CT = np.cumsum(ref.T)
        CS = np.cumsum(ref.S.astype(np.float64))
        for s_ in diff:
            rhs = CS[s_] * CT[-1]
            mism_tie += int(np.min(np.abs(CT * N - rhs)) <= 1e-4 * rhs)
    c32.close()
    return {"workload": f"{n_imgs} x 1000x664 uint16 (12-bit) images, K=4096, FP32 solve", "images": n_imgs,
            "ms_per_batch": ms, "MP_per_s": mp / (ms / 1e3),
            "accuracy_vs_oracle": {"images": 4, "max_rel_err_T": max(errs), "lut_entries_differing": mism,
                                   "differing_at_ties": mism_tie, "lut_entries": 4 * 4096,
                                   "reference": "FP64 CPU oracle, same images"}}


def gamma_leg(hr, local):
    """The gamma-sensitivity study (Table III analogue) on a synthetic 1000x664 image through the
    GPU path: PSNR / SSIM / LOE to the input, mean V, and PSNR / SSIM to the scene's normal-light
    rendering, for gamma = 1, 1.5, 2.2, 5, 10."""
    from paper_2510_21100_gb300 import quality, synth
    W, H = 1000, 664
    seed = synth.seed_for(6, 0)
    img = synth.low_light_image(W, H, seed=seed)
    ref = synth.normal_light_image(W, H, seed=seed)
    d = hr.to_device_aligned(img, f"cuda:{local}")
    rows = []
    for g in (1.0, 1.5, 2.2, 5.0, 10.0):
        with hr.Context(hr.Params(gamma=g, alpha=1e-4, beta=1e-4), device=local) as ctx:
            out = ctx.enhance(d, hr.aligned_empty(H, W, device=f"cuda:{local}")).cpu().numpy()
            ctx.check()
        rows.append({"gamma": g, "psnr_input": round(quality.psnr(out, img), 4),
                     "ssim_input": round(quality.ssim(out, img), 4), "loe": round(quality.loe(img, out), 3),
                     "mean_V": round(quality.mean_value(out), 3), "psnr_reference": round(quality.psnr(out, ref), 4),
                     "ssim_reference": round(quality.ssim(out, ref), 4)})
    return {"workload": "synthetic 1000x664 uint8 low-light image (seed 6000000) and its normal-light rendering, "
                        "K=256, T=10, alpha=beta=1e-4", "input_mean_V": round(quality.mean_value(img), 3),
            "rows": rows}


def ablation_leg(torch, hr, local, n=512, K=256, reps=5):
    """The tcgen05 ablation of the reduced-precision form: Eq. 11 class totals of n images at K = 256
    (reflectance and illumination histograms of synthetic low-light images: R = H_C(grad S) / N,
    L = H_C(S) / N, the solve's first iterate) by the FP32 gather on the CUDA cores, the BF16 one-hot
    GEMM on tcgen05 and its split hi + lo form; kernel time (mean of reps) and max relative error
    against exact FP64 totals."""
    import numpy as np
    import oracle
    from paper_2510_21100_gb300 import synth
    R, L = np.zeros((n, K)), np.zeros((n, K))
    base = [synth.low_light_image(320, 240, seed=synth.seed_for(7, i)) for i in range(16)]
    for k in range(n):
        img = np.ascontiguousarray(np.roll(base[k % 16], 7 * k, axis=1))
        S, G = oracle.histograms(img, K)
        R[k], L[k] = G / G.sum(), S / S.sum()
    i = np.arange(K)[:, None]
    j = np.arange(K)[None, :]
    cm = ((2 * i * j + (K - 1)) // (2 * (K - 1))).ravel()
    want = np.zeros((n, K))
    for k in range(n):
        np.add.at(want[k], cm, np.outer(R[k], L[k]).ravel())
    dR = torch.from_numpy(R.astype(np.float32)).to(f"cuda:{local}")
    dL = torch.from_numpy(L.astype(np.float32)).to(f"cuda:{local}")
    nz = want > 0
    out = {"workload": f"{n} images, K={K}: Eq. 11 class totals of the first iterate (one step of the solve)"}
    for m, name in ((0, "fp32_gather_cuda_cores"), (1, "bf16_onehot_gemm_tcgen05"), (2, "bf16x2_split_onehot_gemm_tcgen05")):
        hr.ablation_class_totals(dR, dL, m)
        times, P = [], None
        for _ in range(reps):
            P, ms = hr.ablation_class_totals(dR, dL, m)
            times.append(ms)
        P = P.cpu().numpy().astype(np.float64)
        out[name] = {"ms": sum(times) / len(times), "max_rel_err": float(np.max(np.abs(P[nz] - want[nz]) / want[nz])),
                     "zero_pattern_exact": bool(np.array_equal(P != 0, nz))}
    fp32 = out["fp32_gather_cuda_cores"]["ms"]
    for name in ("bf16_onehot_gemm_tcgen05", "bf16x2_split_onehot_gemm_tcgen05"):
        out[name]["time_vs_fp32_gather"] = out[name]["ms"] / fp32
    out["tolerance_of_the_precision_form"] = 1e-4
    return out


def serving_pool(torch, synth, seed=5):
    """The serving request mix: 70% 0.3-2 MP, 25% 2-8 MP (log-uniform area, aspect 4:3/16:9/3:2), 5%
    the 7680x4320 workload image; a pool of 6 + 3 generated images and the large one."""
    import math
    import numpy as np
    rng = np.random.default_rng(seed)
    pool, weights = [], []
    for band, (lo, hi), count, share in (("small", (0.3e6, 2e6), 6, 0.70), ("medium", (2e6, 8e6), 3, 0.25)):
        for i in range(count):
            area = math.exp(rng.uniform(math.log(lo), math.log(hi)))
            ar = [4 / 3, 16 / 9, 3 / 2][int(rng.integers(0, 3))]
            w = int(round(math.sqrt(area * ar))); h = int(round(area / w))
            pool.append(torch.from_numpy(synth.low_light_image(w, h, seed=synth.seed_for(5, len(pool)))).pin_memory())
            weights.append(share / count)
    return pool, weights


def serving_leg(torch, hr, local, big_img, seconds=5.0, rates=(400.0,), seed=5, warm_s=0.0, capacity_requests=1500,
                repeats=3):
    """Continuous batching under Poisson arrivals of mixed-size 8-bit requests (40 GB device budget,
    3 streams), at each rate in `rates` for `seconds`, `repeats` times (statistics over the requests
    arriving after warm_s); then capacity: `capacity_requests` requests all queued at once, served by the same
    server, against the same requests sent one by one through histretinex_enhance on 16 streams."""
    from paper_2510_21100_gb300 import serve, synth
    pool, weights = serving_pool(torch, synth, seed)
    pool.append(torch.from_numpy(big_img).pin_memory())
    weights.append(0.05)
    srv = serve.Server(hr.Params(), budget_bytes=40 << 30, streams=3, max_batch=32, device=local)
    srv.run(serve.poisson_requests(pool, rates[0], 0.5, seed=seed + 1, weights=weights))
    out = {"workload": "Poisson arrivals, 70% 0.3-2 MP / 25% 2-8 MP / 5% 7680x4320, uint8, K=256, 40 GB budget, "
                       "3 streams, continuous batching", "rates": []}
    for rate in rates:
        # the same arrivals `repeats` times; the row is the run with the median p99, and every run's
        # p50, p99 and longest host-loop lag are listed (a host stall of the serving process shows
        # as a lag of tens of ms in the run whose p99 it inflates)
        runs = []
        for _ in range(repeats):
            reqs = serve.poisson_requests(pool, rate, seconds, seed=seed, weights=weights)
            st = srv.run(reqs)
            runs.append((st.summary(), reqs))
        order = sorted(range(repeats), key=lambda k: runs[k][0]["p99_ms"])
        row, reqs = runs[order[repeats // 2]]
        row = dict(row)
        row.update({"rate_req_per_s": rate, "seconds_offered": seconds,
                    "offered_MP_per_s": sum(r.megapixels for r in reqs) / seconds,
                    "runs": [{k: r[k] for k in ("p50_ms", "p99_ms", "max_loop_lag_ms")} for r, _ in runs]})
        if warm_s > 0:
            row["after_warmup"] = serve.window_stats(reqs, warm_s)
        out["rates"].append(row)
    # capacity: every request queued at t = 0 (the same mix), served vs plain single-image calls
    cap = serve.poisson_requests(pool, 1e6, capacity_requests / 1e6, seed=seed + 2, weights=weights)
    for r in cap:
        r.arrival = 0.0
    sc = srv.run(cap).summary()
    srv.close()
    pl = serve.plain_throughput(cap, hr.Params(), streams=16, partitions=0, device=local)
    out["capacity"] = {"requests": len(cap), "MP": sum(r.megapixels for r in cap),
                       "served_MP_per_s": sc["MP_per_s"], "served_p50_ms": sc["p50_ms"], "served_batches": sc["batches"],
                       "plain_MP_per_s": pl["MP_per_s"], "plain": "one histretinex_enhance per request, 16 streams, "
                       "unpartitioned, host-to-device copy of each request included (as in the server)"}
    return out


def timed_loop(ctx, dins, douts, steps, warmup, dist, torch, staged=False, n_streams=1):
    """K steps (one image each) between CUDA events on the current stream.  With n_streams > 1 the
    steps go round-robin to that many streams (buffer pair k on stream k, so no buffer crosses
    streams), which start after the first event and end before the second: calls on different
    streams overlap on the device (one image's solve beside other images' pixel passes)."""
    n = len(dins)
    main_st = torch.cuda.current_stream()
    sts = [main_st] + [torch.cuda.Stream() for _ in range(n_streams - 1)]

    def issue(k):
        st = sts[k % n_streams]
        ctx.enhance(dins[k % n], douts[k % n], stream=st)

    for s in range(warmup):
        issue(s)
    torch.cuda.synchronize()
    if staged:
        ctx.stage_times(reset=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = ctx.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(main_st)
    for st in sts[1:]:
        st.wait_event(e0)
    for s in range(steps):
        issue(s)
    for st in sts[1:]:
        ev = torch.cuda.Event()
        ev.record(st)
        main_st.wait_event(ev)
    e1.record(main_st)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms_total = e0.elapsed_time(e1)
    launches = ctx.kernel_launches() - l0
    ctx.check()
    if not staged:
        return ms_total, launches, None
    h, so, ap, calls = ctx.stage_times(reset=True)
    return ms_total, launches, (h / calls, so / calls, ap / calls)


def latency_ms(ctx, din, dout, reps, torch):
    """Per-image latency: one call at a time, each timed alone between events (mean, p50, max)."""
    for _ in range(3):
        ctx.enhance(din, dout)
    torch.cuda.synchronize()
    t = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.enhance(din, dout)
        e1.record()
        e1.synchronize()
        t.append(e0.elapsed_time(e1))
    t.sort()
    return {"mean": sum(t) / len(t), "p50": t[len(t) // 2], "max": t[-1], "calls": reps}


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        return run_reference(a, rank, world)

    import numpy as np
    import torch
    import paper_2510_21100_gb300 as hr
    from paper_2510_21100_gb300 import build

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()

    W, H = a.width, a.height
    imgs = make_images(W, H, rank)
    dins = [torch.from_numpy(im).cuda() for im in imgs]
    douts = [torch.empty_like(d) for d in dins]
    ctx = hr.Context(hr.Params(), device=local)
    ctx.set_tuning(partitions=a.partitions, partition_cluster=a.partition_cluster)
    # per-kernel durations: a second timed loop of the same workload on a context that records CUDA
    # events around each stage (events between the kernels keep them from overlapping, so the
    # headline loop above runs without them), its solves on clusters of the headline's size
    sctx = hr.Context(hr.Params(stage_timing=True), device=local)
    sctx.set_tuning(solve_cluster=a.partition_cluster if a.partitions > 0 else 16)

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid) if hasattr(
            torch.cuda.get_device_properties(local), "uuid") else None
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid).__enter__()
    ms_total, launches, _ = timed_loop(ctx, dins, douts, a.steps, a.warmup, dist, torch, n_streams=a.streams)
    clocks = sampler.result()
    ms_one, _, _ = timed_loop(ctx, dins, douts, a.steps, a.warmup, dist, torch, n_streams=1)
    ms_staged, _, stage = timed_loop(sctx, dins, douts, a.steps, a.warmup, dist, torch, staged=True)
    lat = latency_ms(ctx, dins[0], douts[0], max(20, min(100, a.steps // 4)), torch)
    part_info = ctx.partition_info()

    from paper_2510_21100_gb300 import shard
    ms_step = shard.max_over_ranks(ms_total / a.steps, dist, device="cuda")
    mp = W * H / 1e6
    value = shard.job_throughput(world, mp, ms_step)

    pk, pk_src = peaks()
    b = 1
    n_px = W * H
    hist_bytes = 3 * b * n_px                 # read RGB once
    apply_bytes = 2 * 3 * b * n_px            # read RGB, write RGB
    # FP64 work of the solve: class totals, both updates (one FMA per support cell each, T iterations)
    # and the Eq. 20 target sum (one FMA per cell).
    with hr.Context(hr.Params(debug=True), device=local) as dctx:
        dctx.enhance(dins[0], douts[0])
        dbg = dctx.debug(0)
    cells = int(np.count_nonzero(dbg["G"])) * int(np.count_nonzero(dbg["S"]))
    solve_flops = 2.0 * cells * (3 * dbg["iters"] + 1)
    h_ms, s_ms, a_ms = stage
    stages = {"hist": h_ms, "solve": s_ms, "apply": a_ms}
    # the dominant kernel by SM time (duration x SMs it holds): the solve's cluster holds a few SMs
    # while the pixel passes hold them all
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    sm_time = {"hist": h_ms * n_sm, "solve": s_ms * (a.partition_cluster if a.partitions > 0 else 16),
               "apply": a_ms * n_sm}
    dom = max(sm_time, key=sm_time.get)
    # FP64 peak: 2 DFMA per SM per clock x 152 SMs x 2.07 GHz x 2 flops = 1259 GFLOP/s; a throughput
    # probe of dependent-free DFMA loops measured 1190-1200 on this GPU (no measured FP64 peak)
    fp64_peak = 1200.0
    # the strip kernel runs when the image has at least 2 strips (512 x 4 pixels) per warp of a full grid
    hist_name = "hist_u8s_kernel" if -(-W // 512) * -(-H // 4) >= 2 * 8 * 152 else "hist_u8v_kernel"
    kern = {
        "hist": {"kernel": hist_name, "bound": "hbm", "achieved": hist_bytes / (h_ms / 1e3) / 1e9,
                 "peak": pk["hbm_gbs"], "unit": "GB/s", "peak_source": pk_src},
        "solve": {"kernel": "solve_kernel<double>", "bound": "alu", "achieved": solve_flops / (s_ms / 1e3) / 1e9,
                  "peak": fp64_peak, "unit": "GFLOP/s",
                  "peak_source": "builder's FP64 throughput probe (1190-1200 GFLOP/s measured)"},
        "apply": {"kernel": "apply_u8v_kernel", "bound": "hbm", "achieved": apply_bytes / (a_ms / 1e3) / 1e9,
                  "peak": pk["hbm_gbs"], "unit": "GB/s", "peak_source": pk_src},
    }
    for v in kern.values():
        v["frac"] = v["achieved"] / v["peak"]
        v["traffic"] = PROFILED_DRAM_BYTES.get(v["kernel"]) if (W, H) == (7680, 4320) else None
    roof = dict(kern[dom])
    e2e_bytes = 3 * b * n_px
    min_bytes = hist_bytes + apply_bytes
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic", "config": workload_config(W, H, a.streams, a.partitions, a.partition_cluster),
        "gpu_launches": launches,
        "stages_ms": stages, "stage_sm_ms": sm_time, "dominant_by": "SM time (stage duration x SMs held)",
        "streams": a.streams,
        "partitions": {"solve_partitions": part_info[0], "pixel_sms": part_info[1],
                       "partition_cluster": a.partition_cluster,
                       "note": f"single-image calls: solves on 16-SM green-context partitions, each running "
                               f"{16 // a.partition_cluster} {a.partition_cluster}-CTA solves at once, pixel passes "
                               f"on the remaining SMs; steps on different streams overlap"},
        "single_stream": {"ms_per_step": ms_one / a.steps, "MP_per_s": mp / (ms_one / a.steps / 1e3)},
        "latency_ms": lat,
        "stage_loop": {"ms_per_step": ms_staged / a.steps,
                       "note": "stages_ms come from a second timed loop of the same workload with CUDA events "
                               "around each stage; those events keep the kernels from overlapping"},
        "pipeline_roofline": {"min_bytes": min_bytes, "roofline_ms": min_bytes / (pk["hbm_gbs"] * 1e9) * 1e3,
                              "frac": (min_bytes / (pk["hbm_gbs"] * 1e9) * 1e3) / ms_step,
                              "frac_without_solve": (min_bytes / (pk["hbm_gbs"] * 1e9) * 1e3) / (h_ms + a_ms)},
        "solve": {"cells": cells, "iters": dbg["iters"], "fp64_flops": solve_flops},
        "roofline": roof, "kernel_rooflines": kern, "clocks": clocks,
    }

    legs = set(x for x in a.only.split(",") if x)
    want = lambda leg: not legs or leg in legs
    if rank == 0 and not a.no_extras and want("e2e"):
        # end to end through the public host-buffer API: pinned host images in, pinned host images out,
        # 64 images per histretinex_enhance_host_many call (each through the plain pipeline; the copies
        # of one image overlap the neighbours' compute, so only the first copy in and the last copy out of
        # a call stand alone); per-image calls reported beside it
        hins = [torch.from_numpy(im).pin_memory() for im in imgs]
        seq = [hins[k % len(hins)] for k in range(64)]
        houts = [torch.empty_like(x).pin_memory() for x in seq]
        ctx.enhance_host_many(seq, houts)
        calls = 2
        t0 = time.perf_counter()
        for _ in range(calls):
            ctx.enhance_host_many(seq, houts)
        el = time.perf_counter() - t0
        n_e2e = len(seq) * calls
        ctx.enhance_host(hins[0], houts[0])
        t1 = time.perf_counter()
        for k in range(8):
            ctx.enhance_host(hins[k % len(hins)], houts[k])
        el1 = time.perf_counter() - t1
        line["e2e"] = {"value": mp * n_e2e / el, "unit": UNIT, "h2d_bytes_per_step": e2e_bytes,
                       "d2h_bytes_per_step": e2e_bytes, "steps": n_e2e,
                       "api": f"histretinex_enhance_host_many, {len(seq)} pinned host images per call",
                       "per_image_calls_MP_per_s": mp * 8 / el1}
    if rank == 0 and not a.no_extras and want("per_size"):
        # the other plain-method sizes, same pipeline
        per = {}
        for (w2, h2) in ((1000, 664), (3840, 2160)):
            ims = make_images(w2, h2)
            di = [hr.to_device_aligned(im, f"cuda:{local}") for im in ims]
            do = [hr.aligned_empty(h2, w2, device=f"cuda:{local}") for _ in ims]
            st = max(100, a.steps // 2)
            # single-image calls on a.streams streams: unpartitioned, and on 1 or 2 solve partitions
            # of four 4-CTA solves each; the best of the three is the size's figure
            tried = {}
            for tn, tk in (("unpartitioned", dict(partitions=0)),
                           ("1 partition, 4-CTA solves", dict(partitions=1, partition_cluster=4)),
                           ("2 partitions, 4-CTA solves", dict(partitions=2, partition_cluster=4))):
                c2 = hr.Context(hr.Params(), device=local)
                c2.set_tuning(**tk)
                mt, _, _ = timed_loop(c2, di, do, st, max(3, a.warmup // 2), None, torch, n_streams=a.streams)
                tried[tn] = mt / st
                if tn == "unpartitioned":
                    m1, _, _ = timed_loop(c2, di, do, st, max(3, a.warmup // 2), None, torch)
                c2.close()
            best = min(tried, key=tried.get)
            c3 = hr.Context(hr.Params(stage_timing=True), device=local)
            _, _, stg = timed_loop(c3, di, do, st, max(3, a.warmup // 2), None, torch, staged=True)
            c3.close()
            ms2 = tried[best]
            rl = (2 * 3 * w2 * h2 + 3 * w2 * h2) / (pk["hbm_gbs"] * 1e9) * 1e3
            per[f"{w2}x{h2}"] = {"MP_per_s": w2 * h2 / 1e6 / (ms2 / 1000), "ms_per_image": ms2,
                                 "streams": a.streams, "tuning": best,
                                 "ms_per_image_by_tuning": tried, "single_stream_ms_per_image": m1 / st,
                                 "stages_ms": {"hist": stg[0], "solve": stg[1], "apply": stg[2]},
                                 "roofline_frac": rl / ms2}
        line["per_size"] = per
    if rank == 0 and not a.no_extras and want("batched"):
        line["batched"] = batched_leg(torch, hr, local, hr.PREC_DF64)
        line["batched_fp64"] = batched_leg(torch, hr, local, hr.PREC_FP64)
    if rank == 0 and not a.no_extras and want("serving"):
        torch.cuda.synchronize()
        torch.cuda.empty_cache()  # the legs' device buffers go back before the latency-sensitive one
        if a.serving_seconds > 0:
            line["serving"] = serving_leg(torch, hr, local, imgs[0], seconds=a.serving_seconds,
                                          rates=tuple(float(x) for x in a.serving_rates.split(",")), warm_s=5.0)
        else:
            line["serving"] = serving_leg(torch, hr, local, imgs[0])
    if rank == 0 and not a.no_extras and want("precision"):
        line["precision"] = precision_leg(torch, hr, local)
    if rank == 0 and not a.no_extras and want("gamma"):
        line["gamma_sensitivity"] = gamma_leg(hr, local)
    if rank == 0 and not a.no_extras and want("ablation"):
        line["precision_ablation"] = ablation_leg(torch, hr, local)
    if rank == 0 and not a.no_extras and want("cpu"):
        rate, reps, shape = cpu_oracle_rate(imgs, seconds=10.0)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{reps} x full {shape[1]}x{shape[0]} image, single-threaded FP64 C oracle"}
        brate, nthr, nimg = cpu_oracle_batch_rate(seconds=10.0)
        line["cpu_baseline_all_cores"] = {"value": brate, "unit": UNIT, "cores": nthr, "kind": "oracle",
                                          "sample": f"{nimg} mixed-size images of the batched workload, one per "
                                                    f"host thread at a time, {nthr} threads, about 10 s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
