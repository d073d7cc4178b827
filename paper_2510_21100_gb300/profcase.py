"""A small, fixed workload for profilers: a few pipeline calls on synthetic low-light images.

    python -m paper_2510_21100_gb300.profcase --size 7680x4320 --calls 5
    python -m paper_2510_21100_gb300.profcase --batch 64 --precision df64

Runs each call on the default stream and synchronises at the end; prints nothing but a one-line
summary, so that a profiler's launch list covers exactly these calls.
"""
from __future__ import annotations

import argparse

import paper_2510_21100_gb300 as hr
from paper_2510_21100_gb300 import synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--size", default="7680x4320", help="WxH of the single image")
    ap.add_argument("--calls", type=int, default=5)
    ap.add_argument("--batch", type=int, default=0, help="n mixed images per batch call instead of one image")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "df64", "fp32"])
    ap.add_argument("--K", type=int, default=256)
    a = ap.parse_args()
    import torch
    prec = {"fp64": hr.PREC_FP64, "df64": hr.PREC_DF64, "fp32": hr.PREC_FP32}[a.precision]
    ctx = hr.Context(hr.Params(K=a.K, precision=prec))
    if a.batch:
        sizes = synth.mixed_batch_sizes(a.batch, 3)
        ins = [hr.to_device_aligned(synth.low_light_image(w, h, seed=synth.seed_for(2, i))) for i, (w, h) in
               enumerate(sizes)]
        outs = [hr.aligned_empty(int(t.shape[0]), int(t.shape[1])) for t in ins]
        for _ in range(a.calls):
            ctx.enhance_batch(ins, outs)
        mp = sum(w * h for w, h in sizes) / 1e6 * a.calls
    else:
        W, H = (int(v) for v in a.size.split("x"))
        d = hr.to_device_aligned(synth.low_light_image(W, H, seed=synth.seed_for(1, 0)))
        o = hr.aligned_empty(H, W)
        for _ in range(a.calls):
            ctx.enhance(d, o)
        mp = W * H / 1e6 * a.calls
    torch.cuda.synchronize()
    ctx.check()
    print(f"profcase: {a.calls} calls, {mp:.1f} MP, {ctx.kernel_launches()} launches")
    ctx.close()


if __name__ == "__main__":
    main()
