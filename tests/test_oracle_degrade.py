"""Pins of the oracle's degradation operator D_s B (Sec. 2.1; g of Eq. 6)."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import zoom_oracle as O


def test_blur_equals_scipy_gaussian_filter(rng):
    # Library special case: scipy's Gaussian filter with radius 1 and
    # nearest-edge borders is the same normalised 3-tap Gaussian.
    x = rng.random((13, 17))
    ref = ndimage.gaussian_filter(x, 0.8, truncate=1.25, mode="nearest")
    np.testing.assert_allclose(O.blur(x, O.gaussian_taps(0.8)), ref, atol=1e-14)


def test_taps_values():
    # Published-style closed form for sigma = 0.8: exp(-1/1.28) = 0.457833...
    np.testing.assert_allclose(O.gaussian_taps(0.8), [0.238994, 0.522011, 0.238994], atol=1e-6)


@pytest.mark.parametrize("s", [2, 3])
def test_constant_image_maps_to_constant(s):
    x = np.full((12, 18), 0.3125)
    np.testing.assert_allclose(O.degrade(x, s, 0.8), np.full((12 // s, 18 // s), 0.3125), atol=1e-15)


@pytest.mark.parametrize("s", [2, 3])
def test_box_decimate_brute_force(rng, s):
    x = rng.random((7 * s + 1, 5 * s + s - 1))   # ragged: cropped right/bottom
    y = O.box_decimate(x, s)
    assert y.shape == (7, 5)
    for i in range(7):
        for j in range(5):
            tot = 0.0
            for a in range(s):
                for b in range(s):
                    tot += x[s * i + a, s * j + b]
            assert abs(y[i, j] - tot / (s * s)) < 1e-15


@pytest.mark.parametrize("s", [2, 3])
def test_degrade_adjoint_is_matrix_transpose(rng, s):
    # Build the linear operator column by column (brute force) and compare its
    # transpose with the oracle's adjoint.
    H, W = 4 * s, 3 * s + 1
    n_in = H * W
    cols = []
    for k in range(n_in):
        e = np.zeros(n_in)
        e[k] = 1.0
        cols.append(O.degrade(e.reshape(H, W), s, 0.8).ravel())
    A = np.stack(cols, axis=1)
    y = rng.random((4, 3))
    np.testing.assert_allclose(O.degrade_adjoint(y, s, 0.8, (H, W)).ravel(), A.T @ y.ravel(), atol=1e-14)
    x = rng.random((H, W))
    lhs = (O.degrade(x, s, 0.8) * y).sum()
    rhs = (x * O.degrade_adjoint(y, s, 0.8, (H, W))).sum()
    assert abs(lhs - rhs) < 1e-12


def test_decimation_preserves_sum(rng):
    x = rng.random((12, 12))
    assert abs(O.box_decimate(x, 2).sum() * 4 - x.sum()) < 1e-12
