"""The 2x zoom of a 512 x 512 LR image with the 1,000,000-pair dictionary
(5x5 LR / 10x10 HR patches, L = 16, k = 16, K = 8) in the configuration
bench.py times, with the pixel feature (w = 4) and with the first-order
gradient feature (D = 50, w = 8, as the bench's gradient line): the
neighbours and distances of 40 sampled queries against the oracle (its
features, keys, candidate sets and exact K nearest, one query at a time),
every query's neighbours and distances equal to the SIMT scan's, and the
search statistics."""
import dataclasses

import numpy as np
import pytest

import synth_inputs as S
from oracle import zoom_oracle as O
from tests import gpu_cases as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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
    return dict(Z=Z, wl=wl, lr=lr, ctx=ctx, d=d, ix=ix, od=od, oix=oix)


def test_sampled_queries_match_oracle(full):
    Z, wl, lr = full["Z"], full["wl"], full["lr"]
    nq = (wl.lr_h - wl.patch + 1) * (wl.lr_w - wl.patch + 1)
    rows = np.random.default_rng(29).choice(nq, 40, replace=False)
    r = Z.query(full["ix"], torch.from_numpy(lr).cuda(), G.params(wl))
    st = full["ctx"].stats()
    nbr = r["nbr"].cpu().numpy()[rows]
    dist = r["dist"].cpu().numpy()[rows]
    oq = O.query(lr, full["od"], full["oix"], wl.K + 1, wl.reg_rel, rows=rows)
    qk = r["keys"].cpu().numpy().view(np.uint64)[rows]
    ok = oq.margin >= 1e-5
    assert np.array_equal(qk[ok], oq.keys[ok])
    ex = G.tie_or_boundary(oq, wl.K, full["oix"].margin)
    assert ex.mean() < 0.25, ex.mean()
    bad = (nbr != oq.nbr[:, :wl.K]).any(axis=1) & ~ex
    assert not bad.any(), rows[bad]
    np.testing.assert_allclose(dist[~ex], oq.dist[~ex, :wl.K], rtol=2e-5, atol=1e-7)
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
