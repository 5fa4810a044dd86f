"""Pins of the oracle's reconstruction (Eq. 14 + overlap averaging),
back-projection (Eq. 6-7, Eq. 15-17) and MAP gradients (Eq. 8-9)."""
import numpy as np
import pytest
from scipy import ndimage

import synth_inputs as S
from oracle import zoom_oracle as O


def test_overlap_add_brute_force(rng):
    h, w, s, P = 6, 7, 2, 3
    PH = s * P
    n = (h - P + 1) * (w - P + 1)
    p = rng.random((n, PH * PH))
    out = O.overlap_add(p, h, w, s, P)
    for Y in range(s * h):
        for X in range(s * w):
            vals = []
            for i in range(h - P + 1):
                for j in range(w - P + 1):
                    if s * i <= Y < s * i + PH and s * j <= X < s * j + PH:
                        vals.append(p[i * (w - P + 1) + j, (Y - s * i) * PH + X - s * j])
            assert abs(out[Y, X] - np.mean(vals)) < 1e-14


def test_overlap_add_adjoint(rng):
    h, w, s, P = 7, 6, 3, 3
    n = (h - P + 1) * (w - P + 1)
    p = rng.random((n, (s * P) ** 2))
    z = rng.random((s * h, s * w))
    lhs = (O.overlap_add(p, h, w, s, P) * z).sum()
    rhs = (p * O.overlap_add_adjoint(z, h, w, s, P)).sum()
    assert abs(lhs - rhs) < 1e-12


def test_constant_dictionary_gives_constant_image(rng):
    h, w, s, P = 9, 8, 2, 5
    n = (h - P + 1) * (w - P + 1)
    R = np.zeros((40, (s * P) ** 2))
    nbr = rng.integers(0, 40, size=(n, 4))
    wgt = rng.random((n, 4))
    wgt /= wgt.sum(1, keepdims=True)
    x = O.reconstruct(nbr, wgt, np.full(n, 0.25), O.Dictionary(s, P, None, None, None, R), h, w)
    np.testing.assert_allclose(x, 0.25, atol=1e-15)


@pytest.mark.parametrize("s,P", [(2, 3), (2, 5), (3, 5)])
def test_own_patches_reconstruct_hr_exactly(s, P):
    # Dictionary cut from the test image's own HR/LR pair: every query finds
    # itself at distance 0, gets a one-hot weight, and the overlap average of
    # the exact HR patches is the HR image itself.
    hr = S.make_image(5, 16 * s, 14 * s).astype(np.float64)
    lr = O.degrade(hr, s, 0.8).astype(np.float32)
    d = O.dictionary_from_lr_hr(lr, hr, s, P)
    alpha, beta = S.lsh_draws(3, 4, 6, P * P, 4.0)
    idx = O.build_index(d, alpha, beta, 4.0, 4, 6)
    qr = O.query(lr, d, idx, 5, 1e-3)
    assert (qr.dist[:, 0] == 0).all()
    assert (qr.nbr[:, 0] == np.arange(len(qr.nbr))).all()
    assert (qr.wgt == np.eye(5)[0]).all()
    x0 = O.reconstruct(qr.nbr, qr.wgt, qr.mu, d, lr.shape[0], lr.shape[1])
    np.testing.assert_allclose(x0, hr, atol=1e-12)


def test_window_sum_equals_scipy_correlate(rng):
    x = rng.random((11, 9))
    k = O.spatial_kernel(1.5, 3)
    np.testing.assert_allclose(O.window_sum_clamped(x, k), ndimage.correlate(x, k, mode="nearest"), atol=1e-14)


def test_bp_without_range_term_is_gaussian_step(rng):
    # sigma_r -> infinity makes the range weight 1: one step is then
    # x - C * up(D B x - y), a plain Gaussian convolution (scipy).
    s = 2
    x = rng.random((16, 20))
    y = rng.random((8, 10))
    e = O.degrade(x, s, 0.8) - y
    ref = x - ndimage.correlate(np.kron(e, np.ones((s, s))), O.spatial_kernel(1.5, 3), mode="nearest")
    got = O.back_project(x, y, s, 0.8, 1, 1.5, 1e12, 3)
    np.testing.assert_allclose(got, ref, atol=1e-13)


def test_bp_removes_constant_error_in_one_step(rng):
    s = 2
    x = rng.random((12, 12))
    y = O.degrade(x, s, 0.8) - 0.0625
    got = O.back_project(x, y, s, 0.8, 1, 1.5, 1e12, 3)
    np.testing.assert_allclose(O.degrade(got, s, 0.8), y, atol=1e-13)


def test_bp_flat_guide_has_unit_range_weight():
    s = 2
    x = np.full((10, 10), 0.4)
    y = np.full((5, 5), 0.3)
    got = O.back_project(x, y, s, 0.8, 1, 1.5, 0.1, 3)
    np.testing.assert_allclose(got, 0.3, atol=1e-14)


def test_bp_residual_non_increasing():
    s = 2
    hr = S.make_image(21, 64, 64).astype(np.float64)
    y = O.degrade(hr, s, 0.8)
    x = np.kron(y, np.ones((s, s))) + 0.02 * np.random.default_rng(3).normal(size=hr.shape)
    res = []
    for it in range(6):
        res.append(np.linalg.norm(O.degrade(x, s, 0.8) - y))
        x = O.back_project(x, y, s, 0.8, 1, 1.5, 0.1, 3)
    assert all(b <= a * (1 + 1e-12) for a, b in zip(res, res[1:]))
    assert res[-1] < 0.5 * res[0]


def _grad_case(s=2, P=3, h=7, w=8, K=3, N=25, seed=0):
    g = np.random.default_rng(seed)
    n = (h - P + 1) * (w - P + 1)
    R = g.normal(scale=0.1, size=(N, (s * P) ** 2))
    nbr = g.integers(0, N - 3, size=(n, K))        # the last 3 entries stay unused
    wgt = g.random((n, K))
    wgt /= wgt.sum(1, keepdims=True)
    mu = g.random(n)
    y = g.random((h, w))
    return R, nbr, wgt, mu, y


def test_data_gradient_matches_central_differences():
    s = 2
    g = np.random.default_rng(1)
    x = g.random((10, 12))
    y = g.random((5, 6))
    an = O.data_energy_grad(x, y, s, 0.8)
    for _ in range(25):
        i, j = g.integers(0, 10), g.integers(0, 12)
        xp, xm = x.copy(), x.copy()
        xp[i, j] += 1e-6
        xm[i, j] -= 1e-6
        fd = (O.data_energy(xp, y, s, 0.8) - O.data_energy(xm, y, s, 0.8)) / 2e-6
        assert abs(fd - an[i, j]) <= 1e-8 * max(1.0, abs(fd))


def test_dictionary_gradient_matches_central_differences():
    s, P, h, w = 2, 3, 7, 8
    R, nbr, wgt, mu, y = _grad_case(s, P, h, w)
    lam = 0.1
    an = O.map_energy_grad_dict(R, nbr, wgt, mu, y, h, w, s, P, 0.8, lam)
    g = np.random.default_rng(2)
    for _ in range(25):
        a, b = g.integers(0, R.shape[0] - 3), g.integers(0, R.shape[1])
        Rp, Rm = R.copy(), R.copy()
        Rp[a, b] += 1e-6
        Rm[a, b] -= 1e-6
        fd = (O.map_energy(Rp, nbr, wgt, mu, y, h, w, s, P, 0.8, lam)
              - O.map_energy(Rm, nbr, wgt, mu, y, h, w, s, P, 0.8, lam)) / 2e-6
        assert abs(fd - an[a, b]) <= 1e-7 * max(1.0, abs(fd))
    assert (an[-3:] == 0).all()


def test_prior_gradient_matches_central_differences():
    s, P, h, w = 3, 3, 6, 7
    n = (h - P + 1) * (w - P + 1)
    g = np.random.default_rng(4)
    p = g.random((n, (s * P) ** 2))
    an = O.overlap_prior_grad(p, h, w, s, P)
    for _ in range(25):
        a, b = g.integers(0, n), g.integers(0, p.shape[1])
        pp, pm = p.copy(), p.copy()
        pp[a, b] += 1e-6
        pm[a, b] -= 1e-6
        fd = (O.overlap_prior(pp, h, w, s, P) - O.overlap_prior(pm, h, w, s, P)) / 2e-6
        assert abs(fd - an[a, b]) <= 1e-7 * max(1.0, abs(fd))


def test_prior_brute_force():
    s, P, h, w = 2, 3, 5, 6
    n = (h - P + 1) * (w - P + 1)
    nw = w - P + 1
    PH = s * P
    p = np.random.default_rng(6).random((n, PH * PH))
    tot = 0.0
    for i in range(h - P + 1):
        for j in range(nw):
            for di, dj in ((0, 1), (1, 0)):
                i2, j2 = i + di, j + dj
                if i2 > h - P or j2 >= nw:
                    continue
                for Y in range(s * i2, s * i + PH):
                    for X in range(s * j2, s * j + PH):
                        a = p[i * nw + j, (Y - s * i) * PH + X - s * j]
                        b = p[i2 * nw + j2, (Y - s * i2) * PH + X - s * j2]
                        tot += (a - b) ** 2
    assert abs(O.overlap_prior(p, h, w, s, P) - tot) < 1e-10


def _step_edge(a, b, H=24, W=24, edge=12):
    x = np.full((H, W), a)
    x[:, edge:] = b
    return x


def _hand_range_weight(a, b, X, edge, radius, sigma_r):
    """Range weight of Eq. 15 at column X of a vertical step edge (a left of
    `edge`, b from it on), worked out by hand: the (2R+1)^2 box mean of the
    guide counts the window's columns on each side of the edge (rows do not
    matter), m = (n_a a + n_b b) / (2R+1)."""
    cols = np.arange(X - radius, X + radius + 1)
    n_b = int((cols >= edge).sum())
    n_a = 2 * radius + 1 - n_b
    m = (n_a * a + n_b * b) / (2 * radius + 1)
    xv = b if X >= edge else a
    return np.exp(-(xv - m) ** 2 / (2.0 * sigma_r ** 2))


@pytest.mark.parametrize("a,b,sigma_r", [(0.3, 0.5, 0.1), (0.7, 0.55, 0.08)])
def test_bp_range_weight_at_a_step_edge(a, b, sigma_r):
    # Eq. 15 with a non-flat guide.  The LR data is the degradation of the
    # guide minus a constant c, so the error image is c everywhere and its
    # normalised Gaussian filtering is c: one step is x - r * c, and r must
    # be exp(-(x - m)^2 / (2 sigma_r^2)) with m the 7 x 7 box mean of the
    # current HR estimate x, which at a step edge is a known mix of a and b.
    s, edge, R, c = 2, 12, 3, 0.05
    x = _step_edge(a, b, edge=edge)
    y = O.degrade(x, s, 0.8) - c
    got = O.back_project(x, y, s, 0.8, 1, 1.5, sigma_r, R)
    r_got = (x - got) / c
    for X in range(edge - 5, edge + 5):
        r_hand = _hand_range_weight(a, b, X, edge, R, sigma_r)
        np.testing.assert_allclose(r_got[:, X], r_hand, rtol=0, atol=1e-12)
    # next to the edge the weight is well below 1 (so the pin sees the term)
    assert _hand_range_weight(a, b, edge, edge, R, sigma_r) < 0.9
    # far from the edge the window is flat: weight 1
    np.testing.assert_allclose(r_got[:, :edge - 4], 1.0, atol=1e-12)
    np.testing.assert_allclose(r_got[:, edge + 4:], 1.0, atol=1e-12)
