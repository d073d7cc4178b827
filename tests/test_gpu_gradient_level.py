"""Exhaustive check of the histogram kernels' gradient-level arithmetic, through the C ABI.

Step 1 rounds each Sobel magnitude sqrt(m2) half up to an integer level and clips it to K - 1.
The three histogram kernels compute that level by different device code: the strip kernel from a
hardware square-root estimate of the clipped m2 plus a 2^23 rounding add, the staged-tile kernel
from an estimate corrected by an exact integer test, the generic kernel by integer corrections of
a float square root.  Each form is driven through every squared magnitude its images can produce
(8-bit images: |gx|, |gy| <= 4 * 255, so m2 <= 2 * 1020^2) and compared with the integer
definition: n = floor(sqrt(m2)), level = n + (m2 > n^2 + n), clipped to K - 1.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

M2_MAX_8BIT = 2 * 1020 * 1020          # largest gx^2 + gy^2 of an 8-bit image
M2_MAX_12BIT = 2 * (4 * 4095) ** 2     # largest of a 12-bit image (K = 4096)


@pytest.fixture(scope="module")
def hr():
    import paper_2510_21100_gb300 as hr
    from paper_2510_21100_gb300 import build
    build.build()
    return hr


def expected_levels(m2_first, n, K):
    m2 = np.arange(m2_first, m2_first + n, dtype=np.int64)
    r = np.floor(np.sqrt(m2.astype(np.float64))).astype(np.int64)
    r -= (r * r > m2).astype(np.int64)           # integer corrections of the float estimate
    r += ((r + 1) * (r + 1) <= m2).astype(np.int64)
    level = r + (m2 > r * r + r).astype(np.int64)  # sqrt(m2) >= r + 1/2  <=>  m2 > r^2 + r
    return np.minimum(level, K - 1)


def test_integer_definition_on_known_values():
    # the reference itself: 0 -> 0, 2 (1.414) -> 1, 3 (1.732) -> 2, 6 (2.449) -> 2, 7 (2.646) -> 3,
    # n^2 + n -> n (sqrt below n + 1/2), n^2 + n + 1 -> n + 1
    got = expected_levels(0, 13, 4096)
    assert list(got) == [0, 1, 1, 2, 2, 2, 2, 3, 3, 3, 3, 3, 3]
    for r in (5, 100, 1020, 23170):
        assert expected_levels(r * r + r, 2, 1 << 20).tolist() == [r, r + 1]


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("K", [8, 16, 32, 64, 128, 256])
def test_8bit_forms_every_m2(hr, form, K):
    import torch
    got = hr.gradient_levels(form, K, 0, M2_MAX_8BIT + 1)
    torch.cuda.synchronize()
    want = expected_levels(0, M2_MAX_8BIT + 1, K)
    got = got.cpu().numpy().astype(np.int64)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, f"form {form}, K {K}: {bad.size} levels differ, first m2 {bad[:5].tolist()}"


@pytest.mark.parametrize("K", [256, 4096])
def test_generic_form_low_range_and_top(hr, K):
    """The generic kernel (16-bit images and unaligned rows): every m2 below 2^24 and the top 2^20
    values a 12-bit image can produce."""
    import torch
    for first, n in ((0, 1 << 24), (M2_MAX_12BIT + 1 - (1 << 20), 1 << 20)):
        got = hr.gradient_levels(2, K, first, n)
        torch.cuda.synchronize()
        want = expected_levels(first, n, K)
        bad = np.nonzero(got.cpu().numpy().astype(np.int64) != want)[0]
        assert bad.size == 0, f"K {K}: {bad.size} levels differ from m2 {first + bad[:5]}"


def test_generic_form_rounding_boundaries(hr):
    """Windows around the rounding boundaries r^2 + r | r^2 + r + 1 and the squares r^2 for r
    spread over the 12-bit range above 2^12 (below it the exhaustive test covers them)."""
    import torch
    top = int(np.sqrt(M2_MAX_12BIT))
    for r in list(range(4096, top, 97)) + [top - 1]:
        first = r * r - 16
        n = min(r + 48, M2_MAX_12BIT + 1 - first)
        got = hr.gradient_levels(2, 4096, first, n)
        torch.cuda.synchronize()
        want = expected_levels(first, n, 4096)
        bad = np.nonzero(got.cpu().numpy().astype(np.int64) != want)[0]
        assert bad.size == 0, f"{bad.size} levels differ from m2 {first + bad[:5]}"


def test_rejects_out_of_range_requests(hr):
    with pytest.raises(hr.HistRetinexError):
        hr.gradient_levels(1, 256, (1 << 23) - 4, 8)   # the staged-tile form needs m2 < 2^23
    with pytest.raises(hr.HistRetinexError):
        hr.gradient_levels(0, 4096, 0, 16)              # 8-bit forms: K <= 256
    with pytest.raises(hr.HistRetinexError):
        hr.gradient_levels(3, 256, 0, 16)               # no such form
