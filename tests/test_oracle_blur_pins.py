"""Pins of the oracle's smoothing step (the Gaussian filter of the paper's
iterated ECC + smoothing pipeline, Sec. 4 "GPU-only pipeline", Table 2)
against scipy's convolution with the same reflection, exact impulse
responses and closed forms."""
import numpy as np
import pytest
from scipy import ndimage

import oracle


def gaussian_taps(sigma: float, radius: int = 6) -> np.ndarray:
    k = np.arange(-radius, radius + 1, dtype=np.float64)
    w = np.exp(-0.5 * (k / sigma) ** 2)
    return (w / w.sum()).astype(np.float32)


def test_reflection_is_half_sample_symmetric():
    assert list(oracle.reflect_index(np.arange(-4, 9), 4)) == [3, 2, 1, 0, 0, 1, 2, 3, 3, 2, 1, 0, 0]
    assert list(oracle.reflect_index(np.arange(-3, 4), 1)) == [0] * 7


@pytest.mark.parametrize("shape", [(40, 57), (9, 13, 17), (3, 2), (1, 30)])
def test_blur_matches_scipy_reflect_convolution(shape):
    rng = np.random.default_rng(51)
    img = rng.normal(size=shape).astype(np.float32)
    w = gaussian_taps(2.0)
    want = img.astype(np.float64)
    for axis in range(img.ndim):
        want = ndimage.convolve1d(want, w.astype(np.float64)[::-1], axis=axis, mode="reflect")
    got = oracle.blur(img, w)
    assert got.dtype == np.float32
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-6 * np.abs(img).max() * img.ndim)


def test_impulse_response_is_the_outer_product_exactly():
    w = gaussian_taps(1.7)
    img = np.zeros((31, 33, 29), np.float32)
    img[15, 16, 14] = 1.0
    got = oracle.blur(img, w)
    # passes run x, then y, then z: the value is ((w_x * w_y) * w_z) rounded at each step
    exp = np.zeros_like(got)
    for a in range(13):
        for b in range(13):
            for c in range(13):
                exp[15 - 6 + a, 16 - 6 + b, 14 - 6 + c] = np.float32(np.float32(w[c] * w[b]) * w[a])
    assert np.array_equal(got, exp)


def test_constant_is_kept_and_asymmetric_taps_are_not_flipped():
    w = gaussian_taps(3.0)
    c = np.full((20, 21), 2.5, np.float32)
    np.testing.assert_allclose(oracle.blur(c, w), 2.5, rtol=3e-7 * 13)
    # a one-sided kernel shifts the image by one pixel: out[x] = in[x + 1]
    shift = np.zeros(3, np.float32)
    shift[2] = 1.0
    img = np.arange(12, dtype=np.float32).reshape(1, 12)
    got = oracle.blur_axis(img, shift, axis=1)
    assert list(got[0]) == list(np.arange(1, 12, dtype=np.float32)) + [11.0]
