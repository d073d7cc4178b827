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
# A LUT decision CT(z) N >= CS(s) TT whose two sides lie closer than this (relative) can
# legitimately flip under the tolerance above; all others must match exactly.
LUT_MARGIN = 1e-7


def params_pair(**kw):
    import paper_2510_21100_gb300 as hr
    p = hr.Params(**kw)
    po = oracle.Params(K=p.K, alpha=p.alpha, beta=p.beta, gamma=p.gamma, eps=p.eps, max_iter=p.max_iter,
                       fixed_iters=p.fixed_iters)
    return p, po


def ambiguous_lut_levels(S, T):
    """Levels s whose LUT decision lies within LUT_MARGIN of a tie, from the oracle's S and T."""
    N = float(np.sum(S))
    CT = np.cumsum(np.asarray(T, dtype=np.float64))
    TT = CT[-1]
    CS = np.cumsum(np.asarray(S, dtype=np.float64))
    lhs = CT * N
    amb = []
    for s in range(len(S)):
        if CS[s] == N:  # top of the source CDF: decided exactly (last occupied target level)
            continue
        rhs = CS[s] * TT
        if np.any(np.abs(lhs - rhs) <= LUT_MARGIN * max(abs(rhs), 1.0)):
            amb.append(s)
    return set(amb)


def assert_close(got, want, what):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    assert np.array_equal(got == 0, want == 0), f"{what}: zero pattern differs"
    nz = want != 0
    if nz.any():
        err = np.max(np.abs(got[nz] - want[nz]) / np.abs(want[nz]))
        assert err <= RTOL, f"{what}: max relative error {err:.3e} > {RTOL}"


def compare_to_oracle(img: np.ndarray, out: np.ndarray, dbg: dict, po, check_fp=True):
    """Parity of one image: histograms exact, R/L/T within RTOL, LUT exact away from ties,
    output pixels exact (against the oracle's apply of the GPU's own LUT, and against the
    oracle's output wherever the LUTs agree)."""
    ref = oracle.enhance(img, po)
    assert np.array_equal(dbg["S"], ref.S), "H_C(S) differs"
    assert np.array_equal(dbg["G"], ref.G), "H_C(grad S) differs"
    if check_fp:
        assert dbg["iters"] == ref.iters
        assert_close(dbg["R"], ref.R, "H_C(R)")
        assert_close(dbg["L"], ref.L, "H_C(L)")
        assert_close(dbg["T"], ref.T, "enhanced histogram")
    amb = ambiguous_lut_levels(ref.S, ref.T)
    lut = dbg["lut"].astype(np.int64)
    diff = np.nonzero(lut != ref.lut.astype(np.int64))[0]
    bad = [int(s) for s in diff if s not in amb or abs(int(lut[s]) - int(ref.lut[s])) > 1]
    assert not bad, f"LUT differs at non-tie levels {bad[:10]}"
    assert np.array_equal(out, oracle.apply(img, dbg["lut"], po.K)), "apply differs from the oracle's apply"
    if diff.size == 0:
        assert np.array_equal(out, ref.out), "output pixels differ"
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
