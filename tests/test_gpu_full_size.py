"""The 2x zoom of a 512 x 512 LR image with the 1,000,000-pair dictionary
(5x5 LR / 10x10 HR patches, L = 16, k = 16, K = 8) in the configuration
bench.py times, with the pixel feature (w = 4) and with the first-order
gradient feature (D = 50, w = 8, as the bench's gradient line):
  * 256 sampled queries against the oracle (its features, keys, candidate
    sets -- 92 % of the dictionary -- exact K nearest and LLE weights);
  * every query's neighbours and distances equal to the SIMT scan's;
  * every HR pixel of the reconstruction (Eq. 14 + overlap average) from
    seeded injected neighbours and weights, and every pixel of the
    back-projection (Eq. 6-7, 15-17), against the oracle."""
import dataclasses

import numpy as np
import pytest

import synth_inputs as S
from oracle import zoom_oracle as O
from tests import gpu_cases as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N_SAMPLE = 256


@pytest.fixture(scope="module", params=[(0, None), (1, 8.0)], ids=["pixels", "gradients"])
def full(request):
    from paper_1004_3980_gb300 import build
    build.build()
    import paper_1004_3980_gb300 as Z
    F, w = request.param
    wl = S.WORKLOADS["zoom2x_512_dict1m"]
    if w is not None:
        wl = dataclasses.replace(wl, w=w)
    D = O.FEATURE_DIMS[F](wl.patch)
    train = S.training_images(wl)
    lrs = wl.train_hr // wl.scale
    pos = S.sample_positions(wl.pos_seed, len(train), lrs, lrs, wl.patch, wl.n_pairs)
    alpha, beta = S.lsh_draws(wl.proj_seed, wl.L, wl.k, D, wl.w)
    lr = S.test_image(wl)
    ctx = Z.Context(0)
    d = Z.Dictionary(ctx, [torch.from_numpy(x).cuda() for x in train], pos, wl.scale, wl.patch, wl.blur_sigma,
                     feature=F)
    ix = Z.Index(d, wl.L, wl.k, wl.w, alpha, beta)
    # the oracle's dictionary features: the definition of build_dictionary
    # (the feature of the float32 LR training image at each position) taken
    # image by image with patch_features; HR residuals are not needed here
    P = wl.patch
    feat = np.empty((len(pos), D))
    mu = np.empty(len(pos))
    for m, x in enumerate(train):
        lr_m = O.degrade(np.asarray(x, np.float64), wl.scale, wl.blur_sigma).astype(np.float32)
        v, mv = O.patch_features(lr_m, P, F)
        sel = np.flatnonzero(pos[:, 0] == m)
        nw = lr_m.shape[1] - P + 1
        src = pos[sel, 1] * nw + pos[sel, 2]
        feat[sel] = v[src]
        mu[sel] = mv[src]
    od = O.Dictionary(wl.scale, P, None, feat, mu, None, F)
    oix = O.build_index(od, alpha, beta, wl.w, wl.L, wl.k)
    return dict(Z=Z, wl=wl, lr=lr, ctx=ctx, d=d, ix=ix, od=od, oix=oix, train=train, pos=pos, F=F)


def test_sampled_queries_match_oracle(full):
    Z, wl, lr = full["Z"], full["wl"], full["lr"]
    nq = (wl.lr_h - wl.patch + 1) * (wl.lr_w - wl.patch + 1)
    rows = np.sort(np.random.default_rng(29).choice(nq, N_SAMPLE, replace=False))
    r = Z.query(full["ix"], torch.from_numpy(lr).cuda(), G.params(wl))
    st = full["ctx"].stats()
    nbr = r["nbr"].cpu().numpy()[rows]
    dist = r["dist"].cpu().numpy()[rows]
    wgt = r["wgt"].cpu().numpy()[rows]
    oq = G.oracle_rows(lr, full["od"], full["oix"], wl.K + 1, wl.reg_rel, rows)
    qk = r["keys"].cpu().numpy().view(np.uint64)[rows]
    ok = oq.margin >= 1e-5
    assert np.array_equal(qk[ok], oq.keys[ok])
    ex = O.neighbour_exclusions(oq.feat, oq.margin, oq.dist, full["od"], full["oix"])
    print(f"\n{full['F']=}: {ex.sum()} of {N_SAMPLE} sampled queries excluded (boundary or tie)")
    assert ex.mean() < 0.02, ex.sum()
    bad = (nbr != oq.nbr[:, :wl.K]).any(axis=1) & ~ex
    assert not bad.any(), rows[bad]
    np.testing.assert_allclose(dist[~ex], oq.dist[~ex, :wl.K], rtol=2e-5, atol=1e-7)
    # LLE weights over the K nearest (Eq. 12-13), FP32 solve at condition <= 1001
    for i in np.flatnonzero(~ex):
        w_o, _ = O.lle_weights(oq.feat[i], full["od"].feat[oq.nbr[i, :wl.K]], wl.reg_rel, oq.dist[i, 0])
        np.testing.assert_allclose(wgt[i], w_o, atol=2e-3)
    # the paper's similarity-check count: the candidate sets are most of the
    # dictionary at these bin widths, and no query lacks candidates
    assert st["n_queries"] == nq and st["n_empty"] == 0
    assert 0.8 < oq.n_cand.mean() / full["od"].n < 1.0


def test_every_query_equals_the_scan(full):
    Z, wl, lr = full["Z"], full["wl"], full["lr"]
    lr_t = torch.from_numpy(lr).cuda()
    a = Z.query(full["ix"], lr_t, G.params(wl, search=1))
    b = Z.query(full["ix"], lr_t, G.params(wl))
    assert torch.equal(a["nbr"], b["nbr"]) and torch.equal(a["dist"], b["dist"])
    c = Z.query(full["ix"], lr_t, G.params(wl, search=3))
    assert torch.equal(a["nbr"], c["nbr"]) and torch.equal(a["dist"], c["dist"])


def test_injected_neighbours_every_pixel(full):
    # Eq. 14 + the overlap average at full size: seeded neighbours (K
    # distinct IDs per query) and weights (positive, summing to 1), the
    # query means from the oracle's patch features; every HR pixel of the
    # GPU reconstruction against the oracle's, each side from its own
    # dictionary build
    if full["F"] != 0:
        pytest.skip("the reconstruction does not depend on the feature mode")
    Z, wl, lr = full["Z"], full["wl"], full["lr"]
    nq = (wl.lr_h - wl.patch + 1) * (wl.lr_w - wl.patch + 1)
    g = np.random.default_rng(53)
    nbr = np.stack([g.choice(wl.n_pairs, wl.K, replace=False) for _ in range(nq)]).astype(np.int64)
    wgt = g.dirichlet(np.ones(wl.K), size=nq).astype(np.float32)
    _, mu = O.patch_features(lr, wl.patch, 0)
    od = O.build_dictionary(full["train"], full["pos"], wl.scale, wl.patch, wl.blur_sigma)
    x_o = O.reconstruct(nbr, wgt.astype(np.float64), mu.astype(np.float32).astype(np.float64), od, wl.lr_h, wl.lr_w)
    x_g = Z.reconstruct(full["ix"], torch.from_numpy(nbr.astype(np.int32)).cuda(), torch.from_numpy(wgt).cuda(),
                        torch.from_numpy(mu.astype(np.float32)).cuda(), wl.lr_h, wl.lr_w).cpu().numpy()
    err = np.abs(x_g - x_o).max()
    print(f"\nreconstruction, every one of {x_o.size} HR pixels: max-abs {err:.2e}")
    assert err <= 1e-3


def test_backproject_every_pixel(full):
    # Eq. 6-7 with the approximate cross-bilateral filter (Eq. 15-17), the
    # workload's 5 steps on a 1024 x 1024 estimate (the LR image replicated
    # plus seeded noise): every HR pixel against the oracle
    if full["F"] != 0:
        pytest.skip("back-projection does not depend on the feature mode")
    Z, wl, lr = full["Z"], full["wl"], full["lr"]
    s = wl.scale
    x0 = (np.kron(lr.astype(np.float64), np.ones((s, s)))
          + 0.02 * np.random.default_rng(59).normal(size=(s * wl.lr_h, s * wl.lr_w))).astype(np.float32)
    x_o = O.back_project(x0.astype(np.float64), lr.astype(np.float64), s, wl.blur_sigma, wl.bp_iters,
                         wl.sigma_spatial, wl.sigma_range, wl.bp_radius)
    hr = torch.from_numpy(x0).cuda()
    Z.backproject(full["ctx"], torch.from_numpy(lr).cuda(), hr, s, G.params(wl), wl.blur_sigma)
    err = np.abs(hr.cpu().numpy() - x_o).max()
    print(f"\nback-projection, every one of {x_o.size} HR pixels: max-abs {err:.2e}")
    assert err <= 1e-3
