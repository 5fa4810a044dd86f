"""Gradient features (Sec. 4.1, feature modes 1 and 2: the first- and
second-order gradients of the LR image at the patch's pixels, D = 2 P^2)
through every search path of the C ABI, against the oracle with the same
seeded inputs: the features via the bucket keys and the neighbour
distances, the SIMT scan, the exact tensor-core filter (bit-identical to the
scan; K = 80 operands for P = 3, K = 160 for P = 5), the BF16 filter
(recall), the capped walk and the whole upscale.  Bin widths give candidate
sets of a seventh to a third of the dictionary, so LSH membership matters."""
import dataclasses

import numpy as np
import pytest

import synth_inputs as S
from oracle import zoom_oracle as O
from tests import gpu_cases as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", params=[(3, 1.5, 1), (5, 3.0, 1), (3, 2.0, 2), (5, 4.0, 2)],
                ids=["first_P3_D18", "first_P5_D50", "second_P3_D18", "second_P5_D50"])
def grad(request):
    from paper_1004_3980_gb300 import build
    build.build()
    import paper_1004_3980_gb300 as Z
    P, w, F = request.param
    wl = dataclasses.replace(S.WORKLOADS["zoom2x_64_dict20k"], patch=P, n_pairs=8000, lr_h=32, lr_w=36, w=w)
    train = S.training_images(wl, 8)
    lrs = wl.train_hr // wl.scale
    pos = S.sample_positions(wl.pos_seed, len(train), lrs, lrs, P, wl.n_pairs)
    D = 2 * P * P
    alpha, beta = S.lsh_draws(wl.proj_seed, wl.L, wl.k, D, w)
    lr = S.test_image(wl)
    odict = O.build_dictionary(train, pos, wl.scale, P, wl.blur_sigma, feature=F)
    oindex = O.build_index(odict, alpha, beta, w, wl.L, wl.k)
    oq = O.query(lr, odict, oindex, wl.K + 1, wl.reg_rel)
    ctx = Z.Context(0)
    d = Z.Dictionary(ctx, [torch.from_numpy(x).cuda() for x in train], pos, wl.scale, P, wl.blur_sigma,
                     feature=F)
    ix = Z.Index(d, wl.L, wl.k, w, alpha, beta)
    return dict(wl=wl, train=train, pos=pos, alpha=alpha, beta=beta, lr=lr, odict=odict, oindex=oindex,
                oq=oq, ctx=ctx, d=d, ix=ix, D=D, F=F)


def _q(g, **kw):
    import paper_1004_3980_gb300 as Z
    r = Z.query(g["ix"], torch.from_numpy(g["lr"]).cuda(), G.params(g["wl"], **kw))
    return {k: v.cpu().numpy() for k, v in r.items()}


def test_dictionary_and_keys(grad):
    g = grad
    assert g["d"].feature == g["F"] and g["d"].dim == g["D"]
    keys, _ = g["ix"].export_keys()
    ok = g["oindex"].margin >= 1e-5
    assert ok.mean() > 0.95
    assert np.array_equal(keys[ok], g["oindex"].keys[ok])
    # stored pixels, means and HR residuals do not depend on the feature mode
    lr_pix, mu, hr = g["d"].export()
    # the degraded LR pixel is the FP64 value rounded once; a rare last-bit
    # difference remains where the GPU's compensated sum lands on a tie
    diff = lr_pix != g["odict"].lr_pix
    assert diff.mean() <= 1e-4, diff.mean()
    np.testing.assert_array_max_ulp(lr_pix, g["odict"].lr_pix, maxulp=1)
    np.testing.assert_allclose(mu, g["odict"].mu, rtol=0, atol=1e-6)
    np.testing.assert_allclose(hr, g["odict"].hr_res, rtol=0, atol=2e-6)


def test_scan_matches_oracle(grad):
    g = grad
    wl, oq = g["wl"], g["oq"]
    r = _q(g, search=1)
    qk = r["keys"].view(np.uint64)
    ok = oq.margin >= 1e-5
    assert np.array_equal(qk[ok], oq.keys[ok])
    assert 0.05 < oq.n_cand.mean() / g["odict"].n < 0.5
    ex = G.tie_or_boundary(oq, wl.K, g["oindex"].margin)
    assert ex.mean() < 0.1
    bad = (r["nbr"] != oq.nbr[:, :wl.K]).any(axis=1) & ~ex
    assert not bad.any(), np.flatnonzero(bad)[:10]
    # FP32 difference-form distances of the gradient features against FP64
    keep = ~ex
    np.testing.assert_allclose(r["dist"][keep], oq.dist[keep, :wl.K], rtol=2e-5, atol=1e-7)
    np.testing.assert_allclose(r["mu"], oq.mu, rtol=0, atol=1e-6)


def test_exact_filter_equals_scan(grad):
    a = _q(grad, search=1)
    b = _q(grad, search=2)
    st = grad["ctx"].stats()
    assert (a["nbr"] == b["nbr"]).all() and (a["dist"] == b["dist"]).all()
    np.testing.assert_array_equal(a["wgt"], b["wgt"])
    assert st["n_filter_fallback"] < 0.2 * st["n_queries"], st


@pytest.mark.parametrize("rerank_mult", [2, 4])
def test_bf16_filter_recall(grad, rerank_mult):
    K = grad["wl"].K
    ex = _q(grad, search=1)
    pr = _q(grad, precision=1, search=2, rerank_mult=rerank_mult)
    rec = np.mean([len(set(pr["nbr"][q]) & set(ex["nbr"][q])) / K for q in range(len(ex["nbr"]))])
    assert rec >= 0.99, rec


def test_capped_walk_matches_oracle(grad):
    import paper_1004_3980_gb300 as Z
    g = grad
    wl = g["wl"]
    cap = 3 * wl.L
    ixc = Z.Index(g["d"], wl.L, wl.k, wl.w, g["alpha"], g["beta"], max_candidates=cap)
    r = Z.query(ixc, torch.from_numpy(g["lr"]).cuda(), G.params(wl))
    nbr = r["nbr"].cpu().numpy()
    oq = O.query(g["lr"], g["odict"], g["oindex"], wl.K + 1, wl.reg_rel, max_candidates=cap)
    # the capped set depends on which IDs the walk takes from each bin
    from tests.test_gpu_cap import _excluded
    ex = _excluded(oq, wl.K, g["oindex"], ixc.export_keys()[0], cap)
    assert ex.mean() < 0.15, ex.mean()
    bad = (nbr != oq.nbr[:, :wl.K]).any(axis=1) & ~ex
    assert not bad.any(), np.flatnonzero(bad)[:10]


def test_upscale_matches_oracle(grad):
    # the HR image against the oracle's, away from the queries whose
    # neighbours differ (ties and boundary cases) and their reach through
    # the overlap average and the back-projection
    import paper_1004_3980_gb300 as Z
    g = grad
    wl, oq, od = g["wl"], g["oq"], g["odict"]
    lr = g["lr"]
    P, s = wl.patch, wl.scale
    r = _q(g, search=2)
    hr = Z.upscale(g["ix"], torch.from_numpy(lr).cuda(), G.params(wl, search=2)).cpu().numpy()
    x, _, _ = O.upscale(lr, od, g["oindex"], wl.K, wl.reg_rel, wl.bp_iters, wl.blur_sigma,
                        wl.sigma_spatial, wl.sigma_range, wl.bp_radius)
    assert hr.shape == x.shape
    differ = (r["nbr"] != oq.nbr[:, :wl.K]).any(axis=1)
    nw = wl.lr_w - P + 1
    mask = np.zeros_like(x, bool)
    reach = wl.bp_iters * (wl.bp_radius + 2 * s)
    for q in np.flatnonzero(differ):
        i, j = divmod(q, nw)
        mask[max(0, s * i - reach):s * (i + P) + reach, max(0, s * j - reach):s * (j + P) + reach] = True
    assert mask.mean() < 0.25
    assert np.abs(hr - x)[~mask].max() < 1e-3


def test_weights_recomputed_by_the_backward_path(grad):
    # zoom_backward recomputes the LLE weights from the gradient features of
    # the given neighbours: with the search's own neighbours they equal the
    # search's weights, and the forward HR image is their reconstruction
    import paper_1004_3980_gb300 as Z
    g = grad
    r = Z.query(g["ix"], torch.from_numpy(g["lr"]).cuda(), G.params(g["wl"], search=1))
    h, w = g["lr"].shape
    x0 = Z.reconstruct(g["ix"], r["nbr"], r["wgt"], r["mu"], h, w).cpu().numpy()
    b = Z.map_energy_grads(g["ix"], torch.from_numpy(g["lr"]).cuda(), r["nbr"], None, lam=0.0,
                           reg_rel=g["wl"].reg_rel)
    np.testing.assert_allclose(b["hr"].cpu().numpy(), x0, rtol=0, atol=1e-5)


def test_save_and_load_keep_the_feature_mode(grad, tmp_path):
    import paper_1004_3980_gb300 as Z
    g = grad
    p = str(tmp_path / "grad.zd")
    g["d"].save(p)
    d2 = Z.Dictionary.load(g["ctx"], p)
    assert d2.feature == g["F"] and d2.dim == g["D"]
    wl = g["wl"]
    ix2 = Z.Index(d2, wl.L, wl.k, wl.w, g["alpha"], g["beta"])
    assert np.array_equal(ix2.export_keys()[0], g["ix"].export_keys()[0])
    with pytest.raises(ValueError):
        Z.Index(d2, wl.L, wl.k, wl.w, g["alpha"][:, :g["wl"].patch ** 2], g["beta"])
