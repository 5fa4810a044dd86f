"""Training-crop sampling (Sec. 5.1) through the C ABI against the oracle:
the drawn centre pixels (equal, except a draw within FP64 rounding of a CDF
step), the crop windows and the crop pixels (bit-exact), the special cases
(a flat image, a single bright pixel, a crop as large as the image), the
argument errors, and a dictionary built from the GPU's crops against the
oracle's dictionary built from its own."""
import numpy as np
import pytest

import synth_inputs as S
from oracle import zoom_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _images():
    imgs = [S.make_image(300 + i, h, w) for i, (h, w) in enumerate([(96, 128), (200, 150), (64, 64), (301, 257)])]
    spike = np.zeros((40, 50), np.float32)
    spike[17, 23] = 1.0
    flat = np.full((48, 40), 0.25, np.float32)
    return imgs + [spike, flat]


def _near_step(img, u, tol=1e-9):
    """Draws within tol * total of a step of the oracle's CDF."""
    cdf = np.cumsum(O.gradient_magnitude(img).ravel())
    total = cdf[-1]
    if total == 0:
        return np.zeros(len(u), bool)
    t = u * total
    i = np.searchsorted(cdf, t)
    lo = np.abs(t - cdf[np.maximum(i - 1, 0)])
    hi = np.abs(cdf[np.minimum(i, len(cdf) - 1)] - t)
    return (np.minimum(lo, hi) <= tol * total)


@pytest.fixture(scope="module")
def ctx():
    from paper_1004_3980_gb300 import build
    build.build()
    import paper_1004_3980_gb300 as Z
    return Z.Context(0)


def test_windows_and_crops_match_oracle(ctx):
    import paper_1004_3980_gb300 as Z
    imgs = _images()
    draws, ch, cw = 25, 32, 40
    u = np.random.default_rng(5).random((len(imgs), draws))
    u[:, 0] = 0.0                                  # the first pixel with mass
    u[:, 1] = np.nextafter(1.0, 0.0)               # the last
    win, crops = Z.sample_crops(ctx, [torch.from_numpy(x).cuda() for x in imgs], u, ch, cw)
    crops = crops.cpu().numpy()
    assert win.shape == (len(imgs), draws, 4) and crops.shape == (len(imgs) * draws, ch, cw)
    n_ex = 0
    for m, img in enumerate(imgs):
        h, w = img.shape
        r, c = O.sample_crop_centers(img, u[m])
        ex = _near_step(img, u[m])
        n_ex += int(ex[2:].sum())   # the two edge draws sit on a step by construction
        ok = ~ex
        assert np.array_equal(win[m, ok, 0], r[ok]) and np.array_equal(win[m, ok, 1], c[ok]), m
        top, left = O.crop_windows(win[m, :, 0], win[m, :, 1], h, w, ch, cw)
        assert np.array_equal(win[m, :, 2], top) and np.array_equal(win[m, :, 3], left)
        for j in range(draws):
            t, l = win[m, j, 2], win[m, j, 3]
            assert np.array_equal(crops[m * draws + j], img[t:t + ch, l:l + cw])
    assert n_ex <= 2
    # the bright pixel's four neighbours, and the flat image's uniform rule
    spike_centres = {(int(a), int(b)) for a, b in win[4, :, :2]}
    assert spike_centres <= {(16, 23), (17, 22), (17, 24), (18, 23)}
    np.testing.assert_array_equal(win[5, :, 0] * 40 + win[5, :, 1], np.floor(u[5] * 48 * 40).astype(int))


def test_crop_as_large_as_the_image_and_errors(ctx):
    import paper_1004_3980_gb300 as Z
    from paper_1004_3980_gb300 import capi
    img = S.make_image(9, 30, 20)
    t = [torch.from_numpy(img).cuda()]
    win, crops = Z.sample_crops(ctx, t, np.array([[0.3, 0.7]]), 30, 20)
    assert (win[0, :, 2:] == 0).all()
    assert np.array_equal(crops.cpu().numpy()[1], img)
    win2, none = Z.sample_crops(ctx, t, np.array([[0.3, 0.7]]), 30, 20, want_crops=False)
    assert none is None and np.array_equal(win2, win)
    with pytest.raises(capi.ZoomError):
        Z.sample_crops(ctx, t, np.array([[0.5]]), 31, 20)
    with pytest.raises(capi.ZoomError):
        Z.sample_crops(ctx, t, np.array([[1.0]]), 10, 10)
    with pytest.raises(capi.ZoomError):
        Z.sample_crops(ctx, t, np.array([[-0.1]]), 10, 10)


def test_dictionary_from_sampled_crops(ctx):
    # the paper's training set construction on synthetic images: crops drawn
    # by gradient mass become the HR training images of a dictionary
    import paper_1004_3980_gb300 as Z
    hr = [S.make_image(400 + i, 160, 160) for i in range(3)]
    u = np.random.default_rng(8).random((3, 6))
    ch = 50
    win, crops = Z.sample_crops(ctx, [torch.from_numpy(x).cuda() for x in hr], u, ch, ch)
    s, P = 2, 5
    lrs = ch // s
    pos = S.sample_positions(3, 18, lrs, lrs, P, 2000)
    d = Z.Dictionary(ctx, list(crops), pos, s, P, 0.8)
    ocrops = []
    for m in range(3):
        r, c = O.sample_crop_centers(hr[m], u[m])
        top, left = O.crop_windows(r, c, 160, 160, ch, ch)
        ocrops += [hr[m][t:t + ch, l:l + ch] for t, l in zip(top, left)]
    od = O.build_dictionary(ocrops, pos, s, P, 0.8)
    lr_pix, mu, hres = d.export()
    diff = lr_pix != od.lr_pix
    assert diff.mean() <= 1e-4
    np.testing.assert_array_max_ulp(lr_pix, od.lr_pix, maxulp=1)
    np.testing.assert_allclose(hres, od.hr_res, atol=2e-6)
