"""Pins of the oracle's patch features (Sec. 4.1, "Feature representation"):
the mean-subtracted patch and the first- and second-order gradient features."""
import numpy as np
import pytest
from scipy import ndimage

import synth_inputs as S
from oracle import zoom_oracle as O


def test_gradients_equal_scipy_correlation(rng):
    # the gradient is the correlation with [-1, 0, 1] along each axis, with
    # the nearest edge pixel outside the image
    x = rng.random((11, 13))
    gx, gy = O.gradient_images(x)
    k = np.array([-1.0, 0.0, 1.0])
    np.testing.assert_allclose(gx, ndimage.correlate1d(x, k, axis=1, mode="nearest"), atol=1e-14)
    np.testing.assert_allclose(gy, ndimage.correlate1d(x, k, axis=0, mode="nearest"), atol=1e-14)


def test_gradients_of_a_ramp():
    # x(r, c) = a r + b c: twice the slope inside, the slope on the edges
    a, b, h, w = 0.3, -0.7, 6, 8
    r, c = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    gx, gy = O.gradient_images(a * r + b * c)
    ex = np.full((h, w), 2 * b)
    ex[:, 0] = ex[:, -1] = b
    ey = np.full((h, w), 2 * a)
    ey[0, :] = ey[-1, :] = a
    np.testing.assert_allclose(gx, ex, atol=1e-13)
    np.testing.assert_allclose(gy, ey, atol=1e-13)


@pytest.mark.parametrize("P", [3, 5])
def test_gradient_feature_layout_brute_force(rng, P):
    h, w = 9, 10
    x = rng.random((h, w))
    v, mu = O.patch_features(x, P, 1)
    assert v.shape == ((h - P + 1) * (w - P + 1), 2 * P * P)
    cl = lambda t, n: min(max(t, 0), n - 1)
    n = 0
    for i in range(h - P + 1):
        for j in range(w - P + 1):
            for a in range(P):
                for b in range(P):
                    r, c = i + a, j + b
                    gx = x[r, cl(c + 1, w)] - x[r, cl(c - 1, w)]
                    gy = x[cl(r + 1, h), c] - x[cl(r - 1, h), c]
                    assert abs(v[n, a * P + b] - gx) < 1e-14
                    assert abs(v[n, P * P + a * P + b] - gy) < 1e-14
            assert abs(mu[n] - x[i:i + P, j:j + P].mean()) < 1e-14
            n += 1


def test_gradient_feature_ignores_a_constant_and_transposes(rng):
    P, h, w = 3, 8, 7
    x = rng.random((h, w))
    v, _ = O.patch_features(x, P, 1)
    v2, _ = O.patch_features(x + 2.5, P, 1)
    np.testing.assert_allclose(v2, v, atol=1e-13)
    assert np.abs(O.patch_features(np.full((h, w), 0.4), P, 1)[0]).max() == 0
    # transposing the image swaps the two halves, each patch transposed
    vt, _ = O.patch_features(x.T, P, 1)
    nw, nwt = w - P + 1, h - P + 1
    for i in range(h - P + 1):
        for j in range(w - P + 1):
            a = v[i * nw + j]
            b = vt[j * nwt + i]
            gx = a[:P * P].reshape(P, P)
            gy = a[P * P:].reshape(P, P)
            np.testing.assert_allclose(b[:P * P].reshape(P, P), gy.T, atol=1e-14)
            np.testing.assert_allclose(b[P * P:].reshape(P, P), gx.T, atol=1e-14)


def test_dictionary_gradient_features_match_the_lr_image(rng):
    # the stored features are those of the (float32) LR training image, and
    # mu and the HR residuals do not depend on the feature mode
    s, P, sigma = 2, 3, 0.8
    hr = [S.make_image(3, 30, 26)]
    lr = O.degrade(hr[0], s, sigma).astype(np.float32)
    pos = np.array([(0, i, j) for i in range(lr.shape[0] - P + 1) for j in range(lr.shape[1] - P + 1)])
    d0 = O.build_dictionary(hr, pos, s, P, sigma, 0)
    d1 = O.build_dictionary(hr, pos, s, P, sigma, 1)
    v, mu = O.patch_features(lr, P, 1)
    assert d1.feature == 1 and d1.feat.shape == (len(pos), 2 * P * P)
    np.testing.assert_allclose(d1.feat, v, atol=1e-12)
    np.testing.assert_array_equal(d1.mu, d0.mu)
    np.testing.assert_array_equal(d1.hr_res, d0.hr_res)
    np.testing.assert_allclose(mu, d0.mu, atol=1e-12)


@pytest.mark.parametrize("s,P", [(2, 3), (3, 5)])
def test_own_patches_reconstruct_hr_exactly_with_gradients(s, P):
    # as with pixel features: every query finds itself at distance 0 and the
    # overlap average of the exact HR patches (each LR mean added back) is
    # the HR image
    hr = S.make_image(6, 16 * s, 14 * s).astype(np.float64)
    lr = O.degrade(hr, s, 0.8).astype(np.float32)
    d = O.dictionary_from_lr_hr(lr, hr, s, P, feature=1)
    D = 2 * P * P
    alpha, beta = S.lsh_draws(3, 4, 6, D, 8.0)
    idx = O.build_index(d, alpha, beta, 8.0, 4, 6)
    qr = O.query(lr, d, idx, 5, 1e-3)
    assert qr.feat.shape[1] == D
    assert (qr.dist[:, 0] == 0).all()
    assert (qr.nbr[:, 0] == np.arange(len(qr.nbr))).all()
    x = O.reconstruct(qr.nbr, qr.wgt, qr.mu, d, lr.shape[0], lr.shape[1])
    np.testing.assert_allclose(x, hr, atol=1e-10)


def test_second_order_equals_scipy_correlation(rng):
    x = rng.random((12, 9))
    gxx, gyy = O.second_order_images(x)
    k = np.array([-1.0, 0.0, 2.0, 0.0, -1.0])
    np.testing.assert_allclose(gxx, ndimage.correlate1d(x, k, axis=1, mode="nearest"), atol=1e-14)
    np.testing.assert_allclose(gyy, ndimage.correlate1d(x, k, axis=0, mode="nearest"), atol=1e-14)


def test_second_order_of_a_quadratic_and_a_ramp():
    # x = a r^2 + b c^2: g_xx = 2 b c^2 - b (c-2)^2 - b (c+2)^2 = -8 b away from
    # the borders; a linear ramp has none
    a, b, h, w = 0.2, -0.45, 9, 10
    r, c = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    gxx, gyy = O.second_order_images(a * r ** 2 + b * c ** 2)
    np.testing.assert_allclose(gxx[:, 2:-2], -8 * b, atol=1e-12)
    np.testing.assert_allclose(gyy[2:-2, :], -8 * a, atol=1e-12)
    lx, ly = O.second_order_images(0.3 * r - 0.7 * c)
    np.testing.assert_allclose(lx[:, 2:-2], 0, atol=1e-12)
    np.testing.assert_allclose(ly[2:-2, :], 0, atol=1e-12)


def test_second_order_is_the_first_order_applied_twice(rng):
    # [-1, 0, 2, 0, -1] = -([-1, 0, 1] * [-1, 0, 1]): away from the borders
    # the second-order response is minus the first-order filter applied to
    # the first-order response
    x = rng.random((11, 12))
    gx, gy = O.gradient_images(x)
    gxx, _ = O.second_order_images(x)
    _, gyy = O.second_order_images(x)
    np.testing.assert_allclose(gxx[:, 2:-2], -O.gradient_images(gx)[0][:, 2:-2], atol=1e-13)
    np.testing.assert_allclose(gyy[2:-2, :], -O.gradient_images(gy)[1][2:-2, :], atol=1e-13)


def test_second_order_feature_layout_brute_force(rng):
    P, h, w = 3, 8, 9
    x = rng.random((h, w))
    v, _ = O.patch_features(x, P, 2)
    assert v.shape == ((h - P + 1) * (w - P + 1), 2 * P * P)
    cl = lambda t, n: min(max(t, 0), n - 1)
    n = 0
    for i in range(h - P + 1):
        for j in range(w - P + 1):
            for a in range(P):
                for b in range(P):
                    r, c = i + a, j + b
                    exx = 2 * x[r, c] - x[r, cl(c - 2, w)] - x[r, cl(c + 2, w)]
                    eyy = 2 * x[r, c] - x[cl(r - 2, h), c] - x[cl(r + 2, h), c]
                    assert abs(v[n, a * P + b] - exx) < 1e-14
                    assert abs(v[n, P * P + a * P + b] - eyy) < 1e-14
            n += 1


def test_own_patches_reconstruct_hr_exactly_with_second_order():
    s, P = 2, 5
    hr = S.make_image(8, 16 * s, 14 * s).astype(np.float64)
    lr = O.degrade(hr, s, 0.8).astype(np.float32)
    d = O.dictionary_from_lr_hr(lr, hr, s, P, feature=2)
    alpha, beta = S.lsh_draws(4, 4, 6, 2 * P * P, 8.0)
    idx = O.build_index(d, alpha, beta, 8.0, 4, 6)
    qr = O.query(lr, d, idx, 5, 1e-3)
    assert (qr.dist[:, 0] == 0).all()
    assert (qr.nbr[:, 0] == np.arange(len(qr.nbr))).all()
    x = O.reconstruct(qr.nbr, qr.wgt, qr.mu, d, lr.shape[0], lr.shape[1])
    np.testing.assert_allclose(x, hr, atol=1e-10)
