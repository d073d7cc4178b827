"""The C-ABI library builds, loads and exports every symbol include/histretinex.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "histretinex.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(histretinex_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_21100_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("histretinex_create", "histretinex_enhance", "histretinex_enhance_batch", "histretinex_destroy"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    import paper_2510_21100_gb300 as hr
    assert sorted(hr.EXPORTS) == declared_functions()


def test_default_params_and_status_strings_without_gpu(lib):
    import paper_2510_21100_gb300 as hr
    p = hr.hr_params()
    lib.histretinex_default_params.argtypes = [ctypes.POINTER(hr.hr_params)]
    lib.histretinex_default_params(ctypes.byref(p))
    assert (p.K, p.max_iter, p.gamma) == (256, 10, 2.2)
    lib.histretinex_status_string.restype = ctypes.c_char_p
    assert lib.histretinex_status_string(5) == b"image level >= K"


def test_invalid_params_rejected_before_device_use(lib):
    import paper_2510_21100_gb300 as hr
    h = ctypes.c_void_p()
    for bad in (hr.Params(K=300), hr.Params(K=8192), hr.Params(alpha=0.0), hr.Params(max_iter=0)):
        cp = bad.c()
        lib.histretinex_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(hr.hr_params), ctypes.c_int]
        assert lib.histretinex_create(ctypes.byref(h), ctypes.byref(cp), 0) == hr.ERR_INVALID_ARG


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2510_21100_gb300 as hr
    monkeypatch.setattr(hr, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(hr, "_LIB", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        hr.library()


def test_noalloc_entry_point_validates_before_device_use(lib):
    import paper_2510_21100_gb300 as hr
    f = lib.histretinex_enhance_noalloc
    f.argtypes = [ctypes.POINTER(hr.hr_params), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                  ctypes.c_size_t, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p]
    ok = hr.Params().c()
    big = hr.Params(K=512).c()
    fake = ctypes.c_void_p(16)  # never dereferenced: every case below is refused first
    assert f(ctypes.byref(big), fake, fake, 8, 8, 24, 24, 2, None) == hr.ERR_UNSUPPORTED  # K > 256
    assert f(ctypes.byref(ok), None, fake, 8, 8, 24, 24, 1, None) == hr.ERR_INVALID_ARG
    assert f(ctypes.byref(ok), fake, fake, 0, 8, 24, 24, 1, None) == hr.ERR_INVALID_ARG
    assert f(ctypes.byref(ok), fake, fake, 8, 8, 20, 24, 1, None) == hr.ERR_INVALID_ARG  # pitch < 3 W
    assert f(ctypes.byref(ok), fake, fake, 8, 8, 24, 24, 3, None) == hr.ERR_INVALID_ARG  # element size
    assert f(ctypes.byref(ok), fake, fake, 65536, 32768, 196608, 196608, 1, None) == hr.ERR_UNSUPPORTED
