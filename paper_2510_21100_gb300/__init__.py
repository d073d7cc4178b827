"""HistRetinex on GB300: Python binding of the C-ABI library ``libhistretinex.so``.

Argument marshalling only: every step of the pipeline runs in the library's CUDA kernels.
PyTorch tensors provide device memory and streams; only raw pointers, sizes and a
cudaStream_t cross the C ABI (``include/histretinex.h``).  The binding refuses to run
without the compiled library: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhistretinex.so")

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_OOM, ERR_CUDA, ERR_RANGE, ERR_TIMEOUT = range(7)
PREC_FP64, PREC_FP32, PREC_DF64 = 0, 1, 4
FLAG_FIXED_ITERS, FLAG_DEBUG_OUT, FLAG_STAGE_TIMING = 1, 2, 4
FLAG_PRINTED_UPDATE, FLAG_NEAREST_MATCH, FLAG_FORWARD_GRADIENT = 8, 16, 32

# Every symbol include/histretinex.h declares.
EXPORTS = (
    "histretinex_default_params", "histretinex_create", "histretinex_enhance", "histretinex_enhance_batch",
    "histretinex_enhance_host", "histretinex_get_debug", "histretinex_sync_status", "histretinex_destroy",
    "histretinex_status_string", "histretinex_kernel_launches", "histretinex_stage_times",
    "histretinex_profile_solve", "histretinex_set_tuning", "histretinex_get_tuning",
    "histretinex_workspace_bytes", "histretinex_enhance_noalloc", "histretinex_reserve",
    "histretinex_enhance_host_many", "histretinex_gradient_levels", "histretinex_partition_info",
    "histretinex_ablation_class_totals",
)


class hr_params(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int),
        ("alpha", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("flags", ctypes.c_uint),
        ("levels", ctypes.c_int),
    ]


class hr_tuning(ctypes.Structure):
    _fields_ = [
        ("hist_ctas_per_sm", ctypes.c_int),
        ("apply_ctas_per_sm", ctypes.c_int),
        ("solve_cluster", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("pdl", ctypes.c_int),
        ("groups", ctypes.c_int),
        ("partitions", ctypes.c_int),
        ("partition_cluster", ctypes.c_int),
    ]


class HistRetinexError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        msg = _lib().histretinex_status_string(code).decode() if _LIB is not None else str(code)
        super().__init__(f"{what}: {msg} (status {code})" if what else f"{msg} (status {code})")
        self.code = code


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build the CUDA library first "
                "(python -m paper_2510_21100_gb300.build); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, sz, u = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_uint
        L.histretinex_default_params.argtypes = [ctypes.POINTER(hr_params)]
        L.histretinex_default_params.restype = None
        L.histretinex_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(hr_params), i]
        L.histretinex_enhance.argtypes = [vp, vp, vp, i, i, sz, sz, i, vp]
        L.histretinex_enhance_batch.argtypes = [vp, i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i),
                                                ctypes.POINTER(i), ctypes.POINTER(sz), ctypes.POINTER(sz), i, vp]
        L.histretinex_enhance_host.argtypes = [vp, vp, vp, i, i, sz, sz, i, vp]
        L.histretinex_enhance_host_many.argtypes = [vp, i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i),
                                                    ctypes.POINTER(i), ctypes.POINTER(sz), ctypes.POINTER(sz), i, vp]
        L.histretinex_enhance_host_many.restype = ctypes.c_int
        L.histretinex_get_debug.argtypes = [vp, i, vp, vp, vp, vp, vp, vp, ctypes.POINTER(i)]
        L.histretinex_sync_status.argtypes = [vp, vp]
        L.histretinex_destroy.argtypes = [vp]
        L.histretinex_status_string.argtypes = [i]
        L.histretinex_status_string.restype = ctypes.c_char_p
        L.histretinex_kernel_launches.argtypes = [vp]
        L.histretinex_kernel_launches.restype = ctypes.c_uint64
        L.histretinex_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i), i]
        L.histretinex_stage_times.restype = ctypes.c_int
        L.histretinex_profile_solve.argtypes = [vp, i, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(i)]
        L.histretinex_profile_solve.restype = ctypes.c_int
        L.histretinex_set_tuning.argtypes = [vp, ctypes.POINTER(hr_tuning)]
        L.histretinex_set_tuning.restype = ctypes.c_int
        L.histretinex_get_tuning.argtypes = [vp, ctypes.POINTER(hr_tuning)]
        L.histretinex_get_tuning.restype = ctypes.c_int
        L.histretinex_enhance_noalloc.argtypes = [ctypes.POINTER(hr_params), vp, vp, i, i, sz, sz, i, vp]
        L.histretinex_enhance_noalloc.restype = ctypes.c_int
        L.histretinex_reserve.argtypes = [vp, i]
        L.histretinex_reserve.restype = ctypes.c_int
        L.histretinex_partition_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.histretinex_partition_info.restype = ctypes.c_int
        L.histretinex_ablation_class_totals.argtypes = [i, i, vp, vp, vp, i, ctypes.POINTER(ctypes.c_float), vp]
        L.histretinex_ablation_class_totals.restype = ctypes.c_int
        L.histretinex_gradient_levels.argtypes = [i, i, i, i, vp, vp]
        L.histretinex_gradient_levels.restype = ctypes.c_int
        L.histretinex_workspace_bytes.argtypes = [vp]
        L.histretinex_workspace_bytes.restype = ctypes.c_size_t
        for name in ("histretinex_create", "histretinex_enhance", "histretinex_enhance_batch",
                     "histretinex_enhance_host", "histretinex_get_debug", "histretinex_sync_status",
                     "histretinex_destroy"):
            getattr(L, name).restype = ctypes.c_int
        _LIB = L
    return _LIB


def library():
    """The loaded ctypes library (raises if it has not been built)."""
    return _lib()


@dataclass
class Params:
    """Method parameters (see hr_params in include/histretinex.h)."""
    K: int = 256
    alpha: float = 1e-3
    beta: float = 1e-3
    gamma: float = 2.2
    eps: float = 0.0
    max_iter: int = 10
    precision: int = PREC_FP64
    fixed_iters: bool = True
    debug: bool = False
    stage_timing: bool = False
    printed_update: bool = False    # Eq. 12 / Eq. 13 as printed (the weight K_ij divides)
    nearest_match: bool = False     # matching to the nearest cumulative share
    forward_gradient: bool = False  # gradient image by forward differences
    levels: int = 0                 # M data levels binned into the K bins (0: M = K)

    def c(self) -> hr_params:
        flags = (FLAG_FIXED_ITERS if self.fixed_iters else 0) | (FLAG_DEBUG_OUT if self.debug else 0) | \
            (FLAG_STAGE_TIMING if self.stage_timing else 0) | (FLAG_PRINTED_UPDATE if self.printed_update else 0) | \
            (FLAG_NEAREST_MATCH if self.nearest_match else 0) | (FLAG_FORWARD_GRADIENT if self.forward_gradient else 0)
        return hr_params(self.K, self.alpha, self.beta, self.gamma, self.eps, self.max_iter, self.precision, flags,
                         self.levels)


def _check(code, what=""):
    if code != OK:
        raise HistRetinexError(code, what)


def aligned_empty(H: int, W: int, dtype=None, device="cuda"):
    """An (H, W, 3) image tensor whose rows start on 16-byte boundaries (the pixel passes' fast
    path needs that); the row pitch is 3 W rounded up to 16 bytes."""
    import torch
    dtype = dtype or torch.uint8
    eb = torch.empty((), dtype=dtype).element_size()
    row = (3 * W * eb + 15) // 16 * 16 // eb
    buf = torch.empty((H, row), dtype=dtype, device=device)
    return buf.as_strided((H, W, 3), (row, 3, 1))


def to_device_aligned(img, device="cuda", stream=None):
    """Copies a host image (numpy array or CPU tensor, (H, W, 3)) into aligned_empty() storage."""
    import numpy as np
    import torch
    t = torch.from_numpy(np.ascontiguousarray(img)) if isinstance(img, np.ndarray) else img
    out = aligned_empty(t.shape[0], t.shape[1], t.dtype, device)
    out.copy_(t, non_blocking=True)
    return out


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _geom(t):
    """(W, H, pitch_bytes, elem_bytes) of an (H, W, 3) uint8/uint16 tensor with unit channel stride."""
    import torch
    if t.dim() != 3 or t.shape[2] != 3 or t.dtype not in (torch.uint8, torch.uint16):
        raise ValueError("images are (H, W, 3) uint8 or uint16 tensors")
    eb = t.element_size()
    if t.stride(2) != 1 or t.stride(1) != 3:
        raise ValueError("pixels must be interleaved RGB (channel stride 1, pixel stride 3)")
    return int(t.shape[1]), int(t.shape[0]), int(t.stride(0)) * eb, eb


class PreparedBatch:
    """The argument arrays of one histretinex_enhance_batch call, marshalled once: a batch called
    again and again on the same device buffers (a pipeline that reuses its input and output tensors)
    then costs no per-image work in Python, which for hundreds of images takes milliseconds, longer
    than the batch itself on the GPU.  The object keeps the tensors alive; it must not outlive a change
    of their storage (resize_, set_)."""

    def __init__(self, ins, outs=None):
        import torch
        if outs is None:
            outs = [torch.empty_like(t) for t in ins]
        n = len(ins)
        if n != len(outs) or n == 0:
            raise ValueError("need matching, non-empty input and output lists")
        g = [_geom(t) for t in ins]
        go = [_geom(t) for t in outs]
        eb = g[0][3]
        if any(x[3] != eb for x in g + go) or any(a[:2] != b[:2] for a, b in zip(g, go)):
            raise ValueError("all images must share one element type and outputs must match inputs")
        VP, I, SZ = ctypes.c_void_p * n, ctypes.c_int * n, ctypes.c_size_t * n
        self.ins, self.outs, self.n, self.eb = list(ins), list(outs), n, eb
        self.args = (VP(*[t.data_ptr() for t in ins]), VP(*[t.data_ptr() for t in outs]), I(*[x[0] for x in g]),
                     I(*[x[1] for x in g]), SZ(*[x[2] for x in g]), SZ(*[x[2] for x in go]))


def enhance_noalloc(d_in, d_out, params: "Params | None" = None, stream=None):
    """histretinex_enhance_noalloc: one device image, no context, no device allocation (K <= 256)."""
    W, H, pin, eb = _geom(d_in)
    W2, H2, pout, eb2 = _geom(d_out)
    if (W, H, eb) != (W2, H2, eb2):
        raise ValueError("input and output images differ in shape or type")
    cp = (params or Params()).c()
    _check(_lib().histretinex_enhance_noalloc(ctypes.byref(cp), ctypes.c_void_p(d_in.data_ptr()),
                                              ctypes.c_void_p(d_out.data_ptr()), W, H, pin, pout, eb,
                                              _stream_ptr(stream)), "histretinex_enhance_noalloc")
    return d_out


def gradient_levels(form: int, K: int, m2_first: int, n: int, stream=None):
    """histretinex_gradient_levels: the gradient levels of m2 in [m2_first, m2_first + n) by the
    device code of histogram kernel form 0 (strips), 1 (staged tiles) or 2 (generic), as a
    uint16 tensor on the current device (a self-test hook)."""
    import torch
    out = torch.empty(n, dtype=torch.uint16, device="cuda")
    _check(_lib().histretinex_gradient_levels(form, K, m2_first, n, ctypes.c_void_p(out.data_ptr()),
                                              _stream_ptr(stream)), "histretinex_gradient_levels")
    return out


def ablation_class_totals(R, L, method: int, stream=None):
    """histretinex_ablation_class_totals: Eq. 11 class totals of n images (R, L: (n, K) float32 CUDA
    tensors) by the FP32 gather (method 0), the BF16 one-hot GEMM on tcgen05 (method 1) or its split
    hi + lo form (method 2); returns
    (P as an (n, K) float32 tensor, kernel ms)."""
    import torch
    n, K = int(R.shape[0]), int(R.shape[1])
    P = torch.empty((n, K), dtype=torch.float32, device=R.device)
    ms = ctypes.c_float(0.0)
    _check(_lib().histretinex_ablation_class_totals(K, n, ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(L.data_ptr()),
                                                    ctypes.c_void_p(P.data_ptr()), method, ctypes.byref(ms),
                                                    _stream_ptr(stream)), "histretinex_ablation_class_totals")
    return P, ms.value


class Context:
    """A HistRetinex context on one CUDA device (owns workspace and per-K tables)."""

    def __init__(self, params: Params | None = None, device: int = 0):
        self.params = params or Params()
        self._h = ctypes.c_void_p()
        cp = self.params.c()
        _check(_lib().histretinex_create(ctypes.byref(self._h), ctypes.byref(cp), device), "histretinex_create")
        self.device = device

    def close(self):
        if self._h:
            _lib().histretinex_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def enhance(self, d_in, d_out=None, stream=None):
        """Enhance one device image (torch tensor (H, W, 3) uint8/uint16); d_out may be d_in."""
        if d_out is None:
            import torch
            d_out = torch.empty_like(d_in)
        W, H, pin, eb = _geom(d_in)
        W2, H2, pout, eb2 = _geom(d_out)
        if (W, H, eb) != (W2, H2, eb2):
            raise ValueError("input and output images differ in shape or type")
        _check(_lib().histretinex_enhance(self._h, ctypes.c_void_p(d_in.data_ptr()), ctypes.c_void_p(d_out.data_ptr()),
                                          W, H, pin, pout, eb, _stream_ptr(stream)), "histretinex_enhance")
        return d_out

    def enhance_ptr(self, in_ptr: int, out_ptr: int, W: int, H: int, in_pitch: int, out_pitch: int, elem_bytes: int,
                    stream=None):
        _check(_lib().histretinex_enhance(self._h, ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), W, H, in_pitch,
                                          out_pitch, elem_bytes, _stream_ptr(stream)), "histretinex_enhance")

    def enhance_batch(self, ins, outs=None, stream=None):
        """Enhance a list of device images with one launch per pipeline stage.  `ins` may instead be a
        PreparedBatch (then `outs` is not given): its arrays are passed as they are."""
        pb = ins if isinstance(ins, PreparedBatch) else PreparedBatch(ins, outs)
        _check(_lib().histretinex_enhance_batch(self._h, pb.n, *pb.args, pb.eb, _stream_ptr(stream)),
               "histretinex_enhance_batch")
        return pb.outs

    def enhance_host(self, h_in, h_out=None, stream=None):
        """End to end from host memory: numpy arrays or (pinned) CPU tensors, (H, W, 3) uint8/uint16."""
        import numpy as np
        if h_out is None:
            h_out = np.empty_like(h_in) if isinstance(h_in, np.ndarray) else h_in.new_empty(h_in.shape)
        if isinstance(h_in, np.ndarray):
            H, W, _ = h_in.shape
            eb = h_in.dtype.itemsize
            pin, pout = h_in.strides[0], h_out.strides[0]
            pi, po = h_in.ctypes.data, h_out.ctypes.data
        else:
            W, H, pin, eb = _geom(h_in)
            _, _, pout, _ = _geom(h_out)
            pi, po = h_in.data_ptr(), h_out.data_ptr()
        _check(_lib().histretinex_enhance_host(self._h, ctypes.c_void_p(pi), ctypes.c_void_p(po), W, H, pin, pout, eb,
                                               _stream_ptr(stream)), "histretinex_enhance_host")
        return h_out

    def enhance_host_many(self, h_ins, h_outs=None, stream=None):
        """A sequence of host images ((pinned) CPU tensors (H, W, 3), one element size), each through the
        plain pipeline, with host-device copies overlapped with the neighbouring images' compute."""
        n = len(h_ins)
        if h_outs is None:
            h_outs = [x.new_empty(x.shape) for x in h_ins]
        geo = [_geom(x) for x in h_ins]
        geo_o = [_geom(x) for x in h_outs]
        eb = geo[0][3]
        if any(g[3] != eb for g in geo):
            raise ValueError("all images of one call need the same element size")
        arr = lambda t, v: (t * n)(*v)
        _check(_lib().histretinex_enhance_host_many(
            self._h, n, arr(ctypes.c_void_p, [x.data_ptr() for x in h_ins]),
            arr(ctypes.c_void_p, [x.data_ptr() for x in h_outs]), arr(ctypes.c_int, [g[0] for g in geo]),
            arr(ctypes.c_int, [g[1] for g in geo]), arr(ctypes.c_size_t, [g[2] for g in geo]),
            arr(ctypes.c_size_t, [g[2] for g in geo_o]), eb, _stream_ptr(stream)), "histretinex_enhance_host_many")
        return h_outs

    def sync_status(self, stream=None):
        return _lib().histretinex_sync_status(self._h, _stream_ptr(stream))

    def check(self, stream=None):
        _check(self.sync_status(stream), "device status")

    def debug(self, image: int = 0):
        """Intermediates of the last call (needs Params(debug=True)): dict of numpy arrays."""
        import numpy as np
        K = self.params.K
        S = np.zeros(K, np.uint64)
        G = np.zeros(K, np.uint64)
        R = np.zeros(K, np.float64)
        L = np.zeros(K, np.float64)
        T = np.zeros(K, np.float64)
        lut = np.zeros(K, np.uint16)
        it = ctypes.c_int(0)
        p = lambda a: ctypes.c_void_p(a.ctypes.data)
        _check(_lib().histretinex_get_debug(self._h, image, p(S), p(G), p(R), p(L), p(T), p(lut), ctypes.byref(it)),
               "histretinex_get_debug")
        return dict(S=S, G=G, R=R, L=L, T=T, lut=lut, iters=it.value)

    def stage_times(self, reset: bool = False):
        """(hist_ms, solve_ms, apply_ms, calls) summed since the last reset (needs stage_timing=True)."""
        ms = (ctypes.c_double * 3)()
        calls = ctypes.c_int(0)
        _check(_lib().histretinex_stage_times(self._h, ms, ctypes.byref(calls), int(reset)), "histretinex_stage_times")
        return ms[0], ms[1], ms[2], calls.value

    def workspace_bytes(self) -> int:
        """Device workspace bytes per image of a batch."""
        return int(_lib().histretinex_workspace_bytes(self._h))

    def tuning(self) -> dict:
        t = hr_tuning()
        _check(_lib().histretinex_get_tuning(self._h, ctypes.byref(t)), "histretinex_get_tuning")
        return {k: getattr(t, k) for k, _ in hr_tuning._fields_}

    def set_tuning(self, **kw):
        """Changes launch shapes (histretinex_set_tuning; fields as in hr_tuning): hist_ctas_per_sm,
        apply_ctas_per_sm (1..32), solve_cluster (1, 2, 4, 8, 16), use_graph (0/1), pdl (mask 0..7 of
        the kernels launched as programmatic dependent launches), groups (1/2 for large batches),
        partitions (0..4 solve partitions of 16 SMs for single-image calls), partition_cluster (1, 2, 4,
        8, 16: CTAs per solve of a partitioned call; each partition runs 16 / partition_cluster at once).
        Fields not given keep their current values; invalid values raise and change nothing."""
        cur = self.tuning()
        cur.update(kw)
        t = hr_tuning(**cur)
        _check(_lib().histretinex_set_tuning(self._h, ctypes.byref(t)), "histretinex_set_tuning")

    def profile_solve(self, image: int = 0):
        """Solve-phase timestamps (ns) of the last call (needs Params(debug=True))."""
        buf = (ctypes.c_longlong * 48)()
        n = ctypes.c_int(48)
        _check(_lib().histretinex_profile_solve(self._h, image, buf, ctypes.byref(n)), "histretinex_profile_solve")
        return list(buf[: n.value])

    def reserve(self, n_images: int) -> None:
        """Allocates the workspace for batches of up to n_images now (later calls then allocate nothing)."""
        _check(_lib().histretinex_reserve(self._h, int(n_images)), "histretinex_reserve")

    def partition_info(self):
        """(solve partitions in use, SMs of the pixel partition) of single-image calls."""
        a, b = ctypes.c_int(0), ctypes.c_int(0)
        _check(_lib().histretinex_partition_info(self._h, ctypes.byref(a), ctypes.byref(b)),
               "histretinex_partition_info")
        return a.value, b.value

    def kernel_launches(self) -> int:
        return int(_lib().histretinex_kernel_launches(self._h))
