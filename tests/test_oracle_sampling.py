"""Pins of the oracle's training-crop sampler (Sec. 5.1, "Training Data
Generation"): a CDF over the pixels from their gradient magnitude, inverse
sampling, crop windows."""
import math

import numpy as np
import pytest

from oracle import zoom_oracle as O


def test_magnitude_of_a_ramp():
    # x = a r + b c: interior gradients (2b, 2a), magnitude 2 sqrt(a^2 + b^2)
    a, b = 0.3, -0.4
    r, c = np.meshgrid(np.arange(7), np.arange(9), indexing="ij")
    m = O.gradient_magnitude(a * r + b * c)
    np.testing.assert_allclose(m[1:-1, 1:-1], 2 * math.hypot(a, b), atol=1e-13)
    np.testing.assert_allclose(m[0, 1:-1], math.hypot(a, 2 * b), atol=1e-13)   # one-sided in y


def test_a_single_bright_pixel_splits_the_draws_four_ways():
    # one pixel of 1 in a zero image: its left, right, upper and lower
    # neighbours each carry mass 1 (one gradient component of 1), so the
    # quarters of [0, 1) fall on them in row-major order
    img = np.zeros((6, 7))
    img[3, 4] = 1.0
    u = np.array([0.0, 0.2, 0.25, 0.49, 0.5, 0.74, 0.75, 0.999])
    r, c = O.sample_crop_centers(img, u)
    expect = [(2, 4), (2, 4), (3, 3), (3, 3), (3, 5), (3, 5), (4, 4), (4, 4)]
    assert list(zip(r.tolist(), c.tolist())) == expect


def test_flat_image_draws_uniformly():
    r, c = O.sample_crop_centers(np.full((4, 5), 0.3), np.array([0.0, 0.5, 0.99]))
    assert list(zip(r.tolist(), c.tolist())) == [(0, 0), (2, 0), (3, 4)]


def test_inverse_cdf_brute_force(rng):
    # exact rational cumulative sums: the first pixel whose cumulative mass
    # exceeds u * total
    from fractions import Fraction
    img = rng.random((5, 6))
    m = O.gradient_magnitude(img).ravel()
    cum = []
    acc = Fraction(0)
    for v in m:
        acc += Fraction(v)
        cum.append(acc)
    u = rng.random(200)
    r, c = O.sample_crop_centers(img, u)
    for k in range(len(u)):
        t = Fraction(u[k]) * cum[-1]
        idx = next(i for i, v in enumerate(cum) if v > t)
        # the FP64 cumulative sum may put a draw within rounding of a step
        # on the other side of it
        if abs(float(t - (cum[idx - 1] if idx else 0))) < 1e-12 or abs(float(cum[idx] - t)) < 1e-12:
            continue
        assert r[k] * 6 + c[k] == idx


def test_frequencies_follow_the_gradient_mass(rng):
    img = rng.random((6, 6)) ** 3
    m = O.gradient_magnitude(img).ravel()
    p = m / m.sum()
    n = 200000
    r, c = O.sample_crop_centers(img, rng.random(n))
    freq = np.bincount(r * 6 + c, minlength=36) / n
    sd = np.sqrt(p * (1 - p) / n)
    assert (np.abs(freq - p) <= 5 * sd + 1e-4).all()


@pytest.mark.parametrize("ch,cw", [(4, 4), (5, 3)])
def test_crop_windows_centre_and_stay_inside(ch, cw):
    h, w = 20, 17
    rows = np.array([10, 0, 19, 1, 18])
    cols = np.array([8, 0, 16, 15, 2])
    top, left = O.crop_windows(rows, cols, h, w, ch, cw)
    for k in range(len(rows)):
        assert 0 <= top[k] <= h - ch and 0 <= left[k] <= w - cw
        if ch // 2 <= rows[k] <= h - ch + ch // 2:
            assert top[k] == rows[k] - ch // 2
        assert top[k] <= rows[k] < top[k] + ch and left[k] <= cols[k] < left[k] + cw
