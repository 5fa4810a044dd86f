"""Pins of the oracle's training-pair cut (Sec. 2.1; Sec. 5.1): which LR
pixels and which HR pixels a dictionary entry holds, and the mean removed
from both.  The HR image is a linear ramp, so every stored value has a
closed form in the entry's position."""
import numpy as np
import pytest

import synth_inputs as S
from oracle import zoom_oracle as O

ALPHA, BETA, GAMMA = 0.003, 0.0011, 0.1   # HR(Y, X) = ALPHA Y + BETA X + GAMMA


def _ramp(H, W):
    Y, X = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    return ALPHA * Y + BETA * X + GAMMA


@pytest.mark.parametrize("s,P", [(2, 3), (2, 5), (3, 5)])
def test_dictionary_entries_of_a_ramp_have_closed_forms(s, P):
    # A 3-tap symmetric blur keeps a ramp unchanged away from the clamped
    # first and last HR rows and columns, and the s x s block mean of a ramp
    # is its value at the block centre: LR(i, j) = ALPHA (s i + (s-1)/2) +
    # BETA (s j + (s-1)/2) + GAMMA for 1 <= i <= h-2, 1 <= j <= w-2.  The
    # entry at LR origin (i, j) must then hold
    #   mu      = the ramp at the patch centre (LR coordinates i + (P-1)/2),
    #   feature = ALPHA s (a - (P-1)/2) + BETA s (b - (P-1)/2),
    #   hr_res  = HR(s i + a, s j + b) - mu,   a, b < s P.
    h, w = 14, 13
    H, W = s * h, s * w
    hr = _ramp(H, W)
    pos = np.array([[0, i, j] for i in range(1, h - P) for j in range(1, w - P)], np.int32)
    d = O.build_dictionary([hr], pos, s, P, 0.8)
    PH = s * P
    c = (P - 1) / 2.0
    for n, (_, i, j) in enumerate(pos):
        mu = ALPHA * (s * (i + c) + (s - 1) / 2.0) + BETA * (s * (j + c) + (s - 1) / 2.0) + GAMMA
        assert abs(d.mu[n] - mu) < 1e-7
        a, b = np.meshgrid(np.arange(P), np.arange(P), indexing="ij")
        feat = (ALPHA * s * (a - c) + BETA * s * (b - c)).ravel()
        np.testing.assert_allclose(d.feat[n], feat, atol=1e-7)
        A, B = np.meshgrid(np.arange(PH), np.arange(PH), indexing="ij")
        hr_res = (ALPHA * (s * i + A) + BETA * (s * j + B) + GAMMA).ravel() - mu
        np.testing.assert_allclose(d.hr_res[n], hr_res, atol=1e-7)
        np.testing.assert_allclose(d.lr_pix[n].astype(np.float64), feat + mu, atol=1e-7)


@pytest.mark.parametrize("s,P", [(2, 5), (3, 3)])
def test_dictionary_over_every_position_equals_the_own_patch_dictionary(s, P):
    # build_dictionary at every LR origin of one training image, in row
    # order, equals the dictionary cut from that image's own LR/HR pair
    # (which reconstructs the HR image exactly: test_recon_bp)
    hr = S.make_image(41, 12 * s, 11 * s).astype(np.float64)
    h, w = hr.shape[0] // s, hr.shape[1] // s
    ii, jj = O.patch_origins(h, w, P)
    pos = np.stack([np.zeros_like(ii), ii, jj], axis=1).astype(np.int32)
    d = O.build_dictionary([hr], pos, s, P, 0.8)
    lr = O.degrade(hr, s, 0.8).astype(np.float32)
    e = O.dictionary_from_lr_hr(lr, hr, s, P)
    assert (d.lr_pix == e.lr_pix).all()
    np.testing.assert_allclose(d.mu, e.mu, atol=1e-15)
    np.testing.assert_allclose(d.feat, e.feat, atol=1e-15)
    np.testing.assert_allclose(d.hr_res, e.hr_res, atol=1e-15)
