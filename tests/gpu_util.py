"""Helpers of the GPU parity tests: run the CUDA path through the C ABI and the oracle on the same input."""
from __future__ import annotations

import numpy as np

import oracle

# Tolerance for the FP64 histograms R, L and T.  Both sides compute every sum of non-negative
# terms in FP64 but in different orders (left to right vs pieces and trees); for n terms the two
# results differ by at most about 2 n u relative (u = 2^-53), n <= K^2 = 65536 cells, and ten
# iterations of a contraction keep the difference at that level: 2 * 65536 * 1.1e-16 = 1.5e-11,
# so 1e-9 leaves a wide margin while still catching any wrong term (which moves values by >> 1e-6).
RTOL = 1e-9


def params_pair(**kw):
    import paper_2510_21100_gb300 as hr
    p = hr.Params(**kw)
    variants = (oracle.VAR_PRINTED_UPDATE if p.printed_update else 0) | \
        (oracle.VAR_NEAREST_MATCH if p.nearest_match else 0) | (oracle.VAR_FORWARD_GRADIENT if p.forward_gradient else 0)
    po = oracle.Params(K=p.K, alpha=p.alpha, beta=p.beta, gamma=p.gamma, eps=p.eps, max_iter=p.max_iter,
                       fixed_iters=p.fixed_iters, variants=variants, levels=p.levels)
    return p, po


def lut_decision_margin(S, T, s):
    """Smallest relative distance |CT(z) N - CS(s) TT| / (CS(s) TT) over the levels z, for the
    matching decision of source level s (the oracle's S and T).  A GPU LUT entry that differs
    from the oracle's where this margin is far above RTOL is a bug; where it is below, the two
    FP64 orders of summation could legitimately decide differently (a genuine near-tie)."""
    N = float(np.sum(S))
    CT = np.cumsum(np.asarray(T, dtype=np.float64))
    CS = float(np.sum(np.asarray(S, dtype=np.float64)[: s + 1]))
    rhs = CS * CT[-1]
    return float(np.min(np.abs(CT * N - rhs)) / max(rhs, 1e-300))


def assert_close(got, want, what):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert np.array_equal(got == 0, want == 0), f"{what}: zero pattern differs"
    nz = want != 0
    if nz.any():
        err = np.max(np.abs(got[nz] - want[nz]) / np.abs(want[nz]))
        assert err <= RTOL, f"{what}: max relative error {err:.3e} > {RTOL}"


def assert_lut_equal(lut, ref_S, ref_T, ref_lut, what="LUT"):
    """The plain form's LUT must equal the oracle's entry for entry.  A differing entry fails
    the test; the message says whether the oracle's decision there was a genuine FP64 near-tie
    (margin below 1e-9) or not."""
    lut = np.asarray(lut, dtype=np.int64)
    ref = np.asarray(ref_lut, dtype=np.int64)
    diff = np.nonzero(lut != ref)[0]
    if diff.size:
        info = [(int(s), int(lut[s]), int(ref[s]), lut_decision_margin(ref_S, ref_T, int(s))) for s in diff[:8]]
        kinds = ["near-tie" if m < RTOL else "not a tie" for *_, m in info]
        raise AssertionError(f"{what} differs from the oracle at {diff.size} levels: "
                             f"(level, gpu, oracle, decision margin) {info} -> {kinds}")


def compare_to_oracle(img: np.ndarray, out: np.ndarray, dbg: dict, po, check_fp=True):
    """Parity of one image with the oracle: histograms, LUT and output pixels bit-exact; R, L and
    the enhanced histogram within RTOL."""
    ref = oracle.enhance(img, po)
    assert np.array_equal(dbg["S"], ref.S), "H_C(S) differs"
    assert np.array_equal(dbg["G"], ref.G), "H_C(grad S) differs"
    if check_fp:
        assert dbg["iters"] == ref.iters
        assert_close(dbg["R"], ref.R, "H_C(R)")
        assert_close(dbg["L"], ref.L, "H_C(L)")
        assert_close(dbg["T"], ref.T, "enhanced histogram")
    assert_lut_equal(dbg["lut"], ref.S, ref.T, ref.lut)
    assert np.array_equal(out, ref.out), "output pixels differ from the oracle's"
    return ref


def run_gpu(ctx, img: np.ndarray, pad_elems: int = 0, inplace: bool = False):
    """Run one image through histretinex_enhance, optionally with padded rows and in place."""
    import torch
    H, W, _ = img.shape
    row = W * 3 + pad_elems
    host = torch.zeros((H, row), dtype=torch.from_numpy(img[:1, :1]).dtype)
    host[:, : W * 3] = torch.from_numpy(np.ascontiguousarray(img)).reshape(H, W * 3)
    dev_in = host.cuda()
    din = dev_in.as_strided((H, W, 3), (row, 3, 1))
    if inplace:
        dout = din
    else:
        dev_out = torch.zeros_like(dev_in)
        dout = dev_out.as_strided((H, W, 3), (row, 3, 1))
    ctx.enhance(din, dout)
    ctx.check()
    return dout.contiguous().cpu().numpy(), ctx.debug(0)
