"""Python access to the HistRetinex CPU oracle (``histretinex_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product path never imports this package.

The C oracle is compiled with gcc on first use (``-O2 -ffp-contract=off`` so that every
written FP64 operation is one IEEE operation, and fma() is libm's correctly rounded fma).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "histretinex_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhistretinex_oracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_INVALID_ARG = 1
ERR_RANGE = 5


class _Params(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int),
        ("alpha", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("fixed_iters", ctypes.c_int),
        ("variants", ctypes.c_int),
        ("levels", ctypes.c_int),
    ]


# Printed forms of three points the default readings settle otherwise (bits of Params.variants).
VAR_PRINTED_UPDATE = 1     # Eq. 12 / Eq. 13 as printed: the weight K_ij divides
VAR_NEAREST_MATCH = 2      # matching to the nearest cumulative share instead of the first that reaches it
VAR_FORWARD_GRADIENT = 4   # the gradient image as forward differences instead of the Sobel operator


@dataclass
class Params:
    """Method parameters: K levels, prior weights alpha/beta (Eq. 9), gamma (Eq. 17),
    stopping threshold eps and iteration cap T (Algorithm 1)."""
    K: int = 256
    alpha: float = 1e-3
    beta: float = 1e-3
    gamma: float = 2.2
    eps: float = 0.0
    max_iter: int = 10
    fixed_iters: bool = True
    variants: int = 0
    levels: int = 0   # M data levels binned into K bins (0: M = K)

    def c(self) -> _Params:
        return _Params(self.K, self.alpha, self.beta, self.gamma, self.eps, self.max_iter, int(self.fixed_iters),
                       int(self.variants), int(self.levels))


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent); returns its path."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        vp, i, sz, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_double
        L.orc_histograms.argtypes = [vp, i, i, sz, i, i, vp, vp]
        L.orc_value_channel.argtypes = [vp, i, i, sz, i, i, vp]
        L.orc_class_index.argtypes = [i, i, i]
        L.orc_class_index.restype = ctypes.c_uint32
        L.orc_iterate.argtypes = [vp, vp, i, d, d, vp, vp, vp, vp, vp, vp, vp, vp]
        L.orc_iterate_v.argtypes = [vp, vp, i, d, d, i, vp, vp, vp, vp, vp, vp, vp, vp]
        L.orc_histograms_v.argtypes = [vp, i, i, sz, i, i, i, vp, vp]
        L.orc_lut_v.argtypes = [vp, vp, i, i, vp]
        L.orc_histograms_b.argtypes = [vp, i, i, sz, i, i, i, i, vp, vp]
        L.orc_bin_location.argtypes = [i, i, i]
        L.orc_bin_location.restype = d
        L.orc_class_table.argtypes = [i, i, vp]
        L.orc_index1_table_b.argtypes = [i, i, d, vp]
        L.orc_target_b.argtypes = [vp, vp, i, i, d, ctypes.c_uint64, vp]
        L.orc_apply_b.argtypes = [vp, vp, i, i, sz, sz, i, i, i, vp]
        L.orc_iterate_b.argtypes = [vp, vp, i, i, d, d, i, vp, vp, vp, vp, vp, vp, vp, vp]
        L.orc_solve.argtypes = [vp, vp, ctypes.POINTER(_Params), vp, vp, ctypes.POINTER(ctypes.c_int)]
        L.orc_index1_table.argtypes = [i, d, vp]
        L.orc_target.argtypes = [vp, vp, i, d, ctypes.c_uint64, vp]
        L.orc_lut.argtypes = [vp, vp, i, vp]
        L.orc_apply.argtypes = [vp, vp, i, i, sz, sz, i, i, vp]
        L.orc_enhance.argtypes = [vp, vp, i, i, sz, sz, i, ctypes.POINTER(_Params), vp, vp, vp, vp, vp, vp,
                                  ctypes.POINTER(ctypes.c_int)]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _img_args(img: np.ndarray):
    if img.ndim != 3 or img.shape[2] != 3 or img.dtype not in (np.uint8, np.uint16):
        raise ValueError("image must be (H, W, 3) uint8 or uint16")
    img = np.ascontiguousarray(img)
    H, W, _ = img.shape
    eb = img.dtype.itemsize
    return img, W, H, W * 3 * eb, eb


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle returned status {code}")
        self.code = code


def _check(st):
    if st != OK:
        raise OracleError(st)


def value_channel(img: np.ndarray, K: int) -> np.ndarray:
    img, W, H, pitch, eb = _img_args(img)
    V = np.zeros((H, W), dtype=np.uint32)
    _check(lib().orc_value_channel(_ptr(img), W, H, pitch, eb, K, _ptr(V)))
    return V


def histograms(img: np.ndarray, K: int, forward: bool = False):
    """(S, G): Eq. 3 histogram of V and histogram of the gradient image, uint64[K] each
    (forward: forward-difference gradient instead of Sobel)."""
    img, W, H, pitch, eb = _img_args(img)
    S = np.zeros(K, dtype=np.uint64)
    G = np.zeros(K, dtype=np.uint64)
    _check(lib().orc_histograms_v(_ptr(img), W, H, pitch, eb, K, int(forward), _ptr(S), _ptr(G)))
    return S, G


def class_index(K: int, i: int, j: int) -> int:
    return int(lib().orc_class_index(K, i, j))


def iterate(S, G, R, L, K: int, alpha: float, beta: float, printed: bool = False):
    """One iteration of Algorithm 1; returns dict with P, q, Ru, Lu (before Eq. 14/15), Rn, Ln
    (printed: Eq. 12 / Eq. 13 as printed, the weight dividing)."""
    S = np.ascontiguousarray(S, dtype=np.uint64)
    G = np.ascontiguousarray(G, dtype=np.uint64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    out = {k: np.zeros(K, dtype=np.float64) for k in ("P", "q", "Ru", "Lu", "Rn", "Ln")}
    _check(lib().orc_iterate_v(_ptr(S), _ptr(G), K, alpha, beta, int(printed), _ptr(R), _ptr(L), _ptr(out["P"]),
                               _ptr(out["q"]), _ptr(out["Ru"]), _ptr(out["Lu"]), _ptr(out["Rn"]), _ptr(out["Ln"])))
    return out


def solve(S, G, p: Params):
    """Algorithm 1: returns (R, L, iterations)."""
    S = np.ascontiguousarray(S, dtype=np.uint64)
    G = np.ascontiguousarray(G, dtype=np.uint64)
    R = np.zeros(p.K, dtype=np.float64)
    L = np.zeros(p.K, dtype=np.float64)
    it = ctypes.c_int(0)
    cp = p.c()
    _check(lib().orc_solve(_ptr(S), _ptr(G), ctypes.byref(cp), _ptr(R), _ptr(L), ctypes.byref(it)))
    return R, L, it.value


def index1_table(K: int, gamma: float) -> np.ndarray:
    t = np.zeros((K, K), dtype=np.uint32)
    _check(lib().orc_index1_table(K, gamma, _ptr(t)))
    return t


def target(R, L, K: int, gamma: float, N: int) -> np.ndarray:
    """Eq. 17-20: the enhanced histogram."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    T = np.zeros(K, dtype=np.float64)
    _check(lib().orc_target(_ptr(R), _ptr(L), K, gamma, int(N), _ptr(T)))
    return T


def lut(S, T, K: int, nearest: bool = False) -> np.ndarray:
    """Histogram matching LUT from the histogram S of V to the target T (nearest: the target level
    of nearest cumulative share instead of the first that reaches the source's)."""
    S = np.ascontiguousarray(S, dtype=np.uint64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    out = np.zeros(K, dtype=np.uint16)
    _check(lib().orc_lut_v(_ptr(S), _ptr(T), K, int(nearest), _ptr(out)))
    return out


def apply(img: np.ndarray, lut_: np.ndarray, K: int) -> np.ndarray:
    img, W, H, pitch, eb = _img_args(img)
    lut_ = np.ascontiguousarray(lut_, dtype=np.uint16)
    out = np.zeros_like(img)
    _check(lib().orc_apply(_ptr(img), _ptr(out), W, H, pitch, pitch, eb, K, _ptr(lut_)))
    return out


@dataclass
class Result:
    out: np.ndarray
    S: np.ndarray
    G: np.ndarray
    R: np.ndarray
    L: np.ndarray
    T: np.ndarray
    lut: np.ndarray
    iters: int


def enhance(img: np.ndarray, p: Params) -> Result:
    """The whole per-image pipeline, with every intermediate."""
    img, W, H, pitch, eb = _img_args(img)
    K = p.K
    S = np.zeros(K, dtype=np.uint64)
    G = np.zeros(K, dtype=np.uint64)
    R = np.zeros(K, dtype=np.float64)
    L = np.zeros(K, dtype=np.float64)
    T = np.zeros(K, dtype=np.float64)
    lt = np.zeros(K, dtype=np.uint16)
    out = np.zeros_like(img)
    it = ctypes.c_int(0)
    cp = p.c()
    _check(lib().orc_enhance(_ptr(img), _ptr(out), W, H, pitch, pitch, eb, ctypes.byref(cp), _ptr(S), _ptr(G),
                             _ptr(R), _ptr(L), _ptr(T), _ptr(lt), ctypes.byref(it)))
    return Result(out, S, G, R, L, T, lt, it.value)


# ---- binned data: K bins over M data levels ----

def histograms_binned(img: np.ndarray, K: int, M: int, forward: bool = False):
    img, W, H, pitch, eb = _img_args(img)
    S = np.zeros(K, dtype=np.uint64)
    G = np.zeros(K, dtype=np.uint64)
    _check(lib().orc_histograms_b(_ptr(img), W, H, pitch, eb, K, M, int(forward), _ptr(S), _ptr(G)))
    return S, G


def bin_location(k: int, K: int, M: int) -> float:
    return float(lib().orc_bin_location(k, K, M))


def class_table(K: int, M: int) -> np.ndarray:
    t = np.zeros((K, K), dtype=np.uint32)
    _check(lib().orc_class_table(K, M, _ptr(t)))
    return t


def index1_table_binned(K: int, M: int, gamma: float) -> np.ndarray:
    t = np.zeros((K, K), dtype=np.uint32)
    _check(lib().orc_index1_table_b(K, M, gamma, _ptr(t)))
    return t


def target_binned(R, L, K: int, M: int, gamma: float, N: int) -> np.ndarray:
    R = np.ascontiguousarray(R, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    T = np.zeros(K, dtype=np.float64)
    _check(lib().orc_target_b(_ptr(R), _ptr(L), K, M, gamma, int(N), _ptr(T)))
    return T


def apply_binned(img: np.ndarray, lut_: np.ndarray, K: int, M: int) -> np.ndarray:
    img, W, H, pitch, eb = _img_args(img)
    lut_ = np.ascontiguousarray(lut_, dtype=np.uint16)
    out = np.zeros_like(img)
    _check(lib().orc_apply_b(_ptr(img), _ptr(out), W, H, pitch, pitch, eb, K, M, _ptr(lut_)))
    return out


def iterate_binned(S, G, R, L, K: int, M: int, alpha: float, beta: float, printed: bool = False):
    S = np.ascontiguousarray(S, dtype=np.uint64)
    G = np.ascontiguousarray(G, dtype=np.uint64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    L = np.ascontiguousarray(L, dtype=np.float64)
    out = {k: np.zeros(K, dtype=np.float64) for k in ("P", "q", "Ru", "Lu", "Rn", "Ln")}
    _check(lib().orc_iterate_b(_ptr(S), _ptr(G), K, M, alpha, beta, int(printed), _ptr(R), _ptr(L), _ptr(out["P"]),
                               _ptr(out["q"]), _ptr(out["Ru"]), _ptr(out["Lu"]), _ptr(out["Rn"]), _ptr(out["Ln"])))
    return out
