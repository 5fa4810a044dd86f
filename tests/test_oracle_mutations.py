"""Planted mistakes: each test swaps one oracle function for a subtly wrong
version (a sign, a dropped term, a transposed operand, a wrong tie rule) and
checks that at least one of the oracle's pins then fails.  The mistakes are
planted in the oracle only, on the CPU."""
import numpy as np
import pytest

from oracle import zoom_oracle as O
from tests import test_golden as TG
from tests import test_oracle_degrade as TD
from tests import test_oracle_dictionary as TDI
from tests import test_oracle_features as TF
from tests import test_oracle_hash as TH
from tests import test_oracle_knn_lle as TK
from tests import test_oracle_random as TRN
from tests import test_oracle_recon_bp as TR
from tests import test_oracle_sampling as TS


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_wrong_bp_sign_is_caught(monkeypatch):
    # adding the filtered error (the literal sign of Eq. 7) instead of
    # subtracting it
    def bp_plus(x, y, s, blur_sigma, iters, sigma_sp, sigma_r, radius):
        x = np.asarray(x, np.float64).copy()
        ck = O.spatial_kernel(sigma_sp, radius)
        box = np.full((2 * radius + 1,) * 2, 1.0 / (2 * radius + 1) ** 2)
        for _ in range(iters):
            e = O.degrade(x, s, blur_sigma) - y
            g = O.window_sum_clamped(np.kron(e, np.ones((s, s))), ck)
            m = O.window_sum_clamped(x, box)
            x = x + np.exp(-(x - m) ** 2 / (2 * sigma_r ** 2)) * g
        return x
    monkeypatch.setattr(O, "back_project", bp_plus)
    _fails(TR.test_bp_removes_constant_error_in_one_step, np.random.default_rng(0))


def test_blur_on_one_axis_only_is_caught(monkeypatch):
    def blur_rows_only(x, taps):
        r = len(taps) // 2
        h, w = x.shape
        xp = np.pad(np.asarray(x, np.float64), ((r, r), (0, 0)), mode="edge")
        return sum(taps[u] * xp[u:u + h] for u in range(len(taps)))
    monkeypatch.setattr(O, "blur", blur_rows_only)
    _fails(TD.test_blur_equals_scipy_gaussian_filter, np.random.default_rng(0))


def test_decimation_adjoint_without_scale_is_caught(monkeypatch):
    # D^T spreading each LR value without the 1/s^2 factor of the box mean
    def adj_unscaled(y, s, sigma, hr_shape):
        z = np.zeros(hr_shape)
        h, w = y.shape
        z[:h * s, :w * s] = np.kron(y, np.ones((s, s)))
        return O.blur_adjoint(z, O.gaussian_taps(sigma))
    monkeypatch.setattr(O, "degrade_adjoint", adj_unscaled)
    _fails(TD.test_degrade_adjoint_is_matrix_transpose, np.random.default_rng(0), 2)


# without the regulariser the planted solve divides by a zero trace bound
@pytest.mark.filterwarnings("ignore::RuntimeWarning")
def test_dropped_regulariser_is_caught(monkeypatch):
    orig = O.lle_weights
    monkeypatch.setattr(O, "lle_weights", lambda q, nb, reg, d1: orig(q, nb, 0.0, d1))
    _fails(TK.test_lle_k2_closed_form, np.random.default_rng(0))


def test_descending_tie_rule_is_caught(monkeypatch):
    def top_k_desc(qv, cand, feat, K):
        d = ((feat[cand] - qv) ** 2).sum(axis=1)
        order = np.lexsort((-cand, d))[:K]
        return cand[order], d[order], 0
    monkeypatch.setattr(O, "top_k", top_k_desc)
    _fails(TK.test_top_k_is_sorted_brute_force_with_id_ties, np.random.default_rng(0))


def test_off_by_one_hash_is_caught(monkeypatch):
    orig = O.hash_values
    monkeypatch.setattr(O, "hash_values", lambda v, a, b, w: (np.ceil(orig(v, a, b, w)[0] + 0.5).astype(np.int64), orig(v, a, b, w)[1]))
    _fails(TH.test_unit_projection_reduces_to_floor, np.random.default_rng(0))


def test_key_fold_without_position_salt_is_caught(monkeypatch):
    def fold_no_salt(h, L, k):
        n = h.shape[0]
        keys = np.empty((n, L), np.uint64)
        for l in range(L):
            x = np.full(n, l, np.uint64)
            for j in range(k):
                x = O.mix64(x ^ ((h[:, l * k + j] & 0xFFFFFFFF).astype(np.uint64) + np.uint64(O.GOLDEN64)))
            keys[:, l] = x
        return keys
    monkeypatch.setattr(O, "fold_keys", fold_no_salt)
    _fails(TG.test_oracle_matches_golden_fixture)


def test_overlap_sum_instead_of_mean_is_caught(monkeypatch):
    def oa_sum(p, h, w, s, P):
        PH = s * P
        acc = np.zeros((s * h, s * w))
        ii, jj = O.patch_origins(h, w, P)
        for n in range(len(ii)):
            acc[s * ii[n]:s * ii[n] + PH, s * jj[n]:s * jj[n] + PH] += p[n].reshape(PH, PH)
        return acc
    monkeypatch.setattr(O, "overlap_add", oa_sum)
    _fails(TR.test_overlap_add_brute_force, np.random.default_rng(0))


def test_missing_prior_factor_is_caught(monkeypatch):
    orig = O.overlap_prior_grad
    monkeypatch.setattr(O, "overlap_prior_grad", lambda p, h, w, s, P: 0.5 * orig(p, h, w, s, P))
    _fails(TR.test_prior_gradient_matches_central_differences)


def test_gradient_with_wrapped_borders_is_caught(monkeypatch):
    # periodic instead of clamped borders
    def grad_wrap(img):
        x = np.asarray(img, np.float64)
        return np.roll(x, -1, axis=1) - np.roll(x, 1, axis=1), np.roll(x, -1, axis=0) - np.roll(x, 1, axis=0)
    monkeypatch.setattr(O, "gradient_images", grad_wrap)
    _fails(TF.test_gradient_feature_layout_brute_force, np.random.default_rng(0), 3)


def test_one_sided_gradient_is_caught(monkeypatch):
    # forward differences x(c+1) - x(c) in place of the centred [-1, 0, 1]
    def grad_fwd(img):
        x = np.asarray(img, np.float64)
        gx = np.concatenate([x[:, 1:] - x[:, :-1], np.zeros((x.shape[0], 1))], axis=1)
        gy = np.concatenate([x[1:] - x[:-1], np.zeros((1, x.shape[1]))], axis=0)
        return gx, gy
    monkeypatch.setattr(O, "gradient_images", grad_fwd)
    _fails(TF.test_gradients_of_a_ramp)


def test_swapped_gradient_halves_are_caught(monkeypatch):
    orig = O.gradient_images
    monkeypatch.setattr(O, "gradient_images", lambda img: orig(img)[::-1])
    _fails(TF.test_gradient_feature_layout_brute_force, np.random.default_rng(0), 5)


def test_second_order_with_unit_spacing_is_caught(monkeypatch):
    # [-1, 2, -1] (adjacent pixels) in place of [-1, 0, 2, 0, -1]
    def lap1(img):
        x = np.asarray(img, np.float64)
        h, w = x.shape
        cm, cp = np.maximum(np.arange(w) - 1, 0), np.minimum(np.arange(w) + 1, w - 1)
        rm, rp = np.maximum(np.arange(h) - 1, 0), np.minimum(np.arange(h) + 1, h - 1)
        return 2 * x - x[:, cm] - x[:, cp], 2 * x - x[rm, :] - x[rp, :]
    monkeypatch.setattr(O, "second_order_images", lap1)
    _fails(TF.test_second_order_of_a_quadratic_and_a_ramp)
    _fails(TF.test_second_order_feature_layout_brute_force, np.random.default_rng(0))


def test_horizontal_only_gradient_mass_is_caught(monkeypatch):
    # the sampling mass taken from g_x alone
    monkeypatch.setattr(O, "gradient_magnitude", lambda img: np.abs(O.gradient_images(img)[0]))
    _fails(TS.test_a_single_bright_pixel_splits_the_draws_four_ways)


def _bp_variant(range_sq, mean_kernel, guide):
    """back_project with one planted change in the range term of Eq. 15:
    range_sq(sigma_r) is the divisor of the squared difference, mean_kernel
    the window weights of the mean, guide picks the image the term reads."""
    def bp(x, y, s, blur_sigma, iters, sigma_sp, sigma_r, radius):
        x = np.asarray(x, np.float64).copy()
        ck = O.spatial_kernel(sigma_sp, radius)
        for _ in range(iters):
            e = O.degrade(x, s, blur_sigma) - y
            u = np.kron(e, np.ones((s, s)))
            g = O.window_sum_clamped(u, ck)
            gd = guide(x, u)
            m = O.window_sum_clamped(gd, mean_kernel(sigma_sp, radius))
            x = x - np.exp(-(gd - m) ** 2 / range_sq(sigma_r)) * g
        return x
    return bp


_BOX = lambda sp, R: np.full((2 * R + 1, 2 * R + 1), 1.0 / (2 * R + 1) ** 2)
_TWO_SQ = lambda sr: 2.0 * sr * sr
_GUIDE_X = lambda x, u: x


@pytest.mark.parametrize("variant", [
    _bp_variant(lambda sr: sr * sr, _BOX, _GUIDE_X),                 # sigma_r^2 instead of 2 sigma_r^2
    _bp_variant(_TWO_SQ, O.spatial_kernel, _GUIDE_X),                # Gaussian-weighted mean, not the box
    _bp_variant(_TWO_SQ, _BOX, lambda x, u: u),                      # the error image as the guide
    _bp_variant(_TWO_SQ, lambda sp, R: _BOX(sp, R - 1), _GUIDE_X),  # a 5 x 5 window for the mean
], ids=["sigma_r_squared", "gaussian_mean", "error_guide", "window_5x5"])
def test_range_weight_mistakes_are_caught(monkeypatch, variant):
    # every variant still passes the flat-guide and sigma_r -> infinity pins
    # that were all the range term had before; the step-edge pin sees each
    monkeypatch.setattr(O, "back_project", variant)
    TR.test_bp_flat_guide_has_unit_range_weight()
    TR.test_bp_without_range_term_is_gaussian_step(np.random.default_rng(0))
    _fails(TR.test_bp_range_weight_at_a_step_edge, 0.3, 0.5, 0.1)


def _dictionary_variant(hr_origin):
    """build_dictionary (feature 0) with the HR patch cut at hr_origin(s, i, j)."""
    def build(hr_images, positions, s, P, sigma, feature=0):
        hr64 = [np.asarray(x, np.float64) for x in hr_images]
        lr_imgs = [O.degrade(x, s, sigma).astype(np.float32) for x in hr64]
        PH = s * P
        lr_pix = np.stack([lr_imgs[m][i:i + P, j:j + P].ravel() for m, i, j in positions])
        hr = []
        for m, i, j in positions:
            Y, X = hr_origin(s, i, j)
            hr.append(hr64[m][Y:Y + PH, X:X + PH].ravel())
        mu = lr_pix.astype(np.float64).mean(axis=1)
        return O.Dictionary(s, P, lr_pix, lr_pix - mu[:, None], mu, np.stack(hr) - mu[:, None], 0)
    return build


@pytest.mark.parametrize("origin", [
    lambda s, i, j: (s * i + 1, s * j),     # one HR row too low
    lambda s, i, j: (s * i, s * j + 1),     # one HR column too far right
    lambda s, i, j: (s * j, s * i),         # row and column swapped
    lambda s, i, j: (i, j),                 # the LR origin used on the HR image
], ids=["row_plus_one", "col_plus_one", "swapped", "lr_origin"])
def test_hr_cut_mistakes_are_caught(monkeypatch, origin):
    monkeypatch.setattr(O, "build_dictionary", _dictionary_variant(origin))
    _fails(TDI.test_dictionary_entries_of_a_ramp_have_closed_forms, 2, 5)


@pytest.mark.parametrize("mistake", ["bump_first", "swap_hilo", "one_multiplier"])
def test_philox_mistakes_are_caught(monkeypatch, mistake):
    # the key bumped before the first round too, the high and low product
    # words swapped, one multiplier for both lanes
    def philox_bad(ctr, seed):
        c = [int(x) for x in np.asarray(ctr, np.uint64).reshape(-1, 4)[0]]
        k0, k1 = seed & 0xFFFFFFFF, seed >> 32
        m0, m1 = O.PHILOX_M if mistake != "one_multiplier" else (O.PHILOX_M[0],) * 2
        for r in range(10):
            if r > 0 or mistake == "bump_first":
                k0, k1 = (k0 + O.PHILOX_W[0]) & 0xFFFFFFFF, (k1 + O.PHILOX_W[1]) & 0xFFFFFFFF
            p0, p1 = m0 * c[0], m1 * c[2]
            hi0, lo0, hi1, lo1 = p0 >> 32, p0 & 0xFFFFFFFF, p1 >> 32, p1 & 0xFFFFFFFF
            if mistake == "swap_hilo":
                hi0, lo0, hi1, lo1 = lo0, hi0, lo1, hi1
            c = [(hi1 ^ c[1] ^ k0) & 0xFFFFFFFF, lo1, (hi0 ^ c[3] ^ k1) & 0xFFFFFFFF, lo0]
        return np.array([c], np.uint32)
    monkeypatch.setattr(O, "philox4x32_10", philox_bad)
    _fails(TRN.test_philox_known_answers, *TRN.KAT[2])
