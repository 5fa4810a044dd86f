"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs, stage by stage and end to end.

Tolerances (from the method's required accuracy):
  * dictionary LR pixels: equal to the oracle's FP64 degradation rounded to
    float32 (a 1-ulp difference is allowed where the FP64 value sits on a
    rounding midpoint, at most 1e-4 of the pixels);
  * bucket keys: bit-exact, except rows whose projection lies within 1e-5*w
    of a bin boundary (counted);
  * neighbour IDs: bit-exact, except boundary-affected queries and queries
    whose K+1 nearest FP64 distances are tied within 1e-6 relative (counted,
    must stay below 2% of the queries);
  * LLE weights: max-abs 2e-3 (FP32 solve of a system with condition <= 1001);
  * HR pixels: max-abs 1e-3 on the [0, 1] scale.
"""
import numpy as np
import pytest

import synth_inputs as S
from oracle import zoom_oracle as O
from tests import gpu_cases as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def built():
    from paper_1004_3980_gb300 import build
    build.build()
    case = G.small_case()
    ctx, d, ix = G.gpu_build(case)
    return case, ctx, d, ix


@pytest.fixture(scope="module")
def oracle_queries(built):
    case = built[0]
    wl = case.wl
    oq = O.query(case.lr, case.odict, case.oindex, wl.K + 1, wl.reg_rel)
    # weights over the first K (the oracle call above used K + 1 for the tie gap)
    wk = np.stack([O.lle_weights(oq.feat[q], case.odict.feat[oq.nbr[q, :wl.K]], wl.reg_rel,
                                 oq.dist[q, 0])[0] for q in range(len(oq.nbr))])
    return oq, wk


def test_dictionary_matches_oracle(built):
    case, ctx, d, ix = built
    lr_pix, mu, hr = d.export()
    od = case.odict
    diff = lr_pix != od.lr_pix
    assert diff.mean() <= 1e-4, diff.mean()
    if diff.any():
        np.testing.assert_array_max_ulp(lr_pix, od.lr_pix, maxulp=1)
    np.testing.assert_allclose(mu, od.mu, atol=1e-6)
    PH2 = (case.wl.scale * case.wl.patch) ** 2
    np.testing.assert_allclose(hr, od.hr_res[:, :PH2], atol=2e-6)


def test_dictionary_keys_bit_exact(built):
    case, ctx, d, ix = built
    keys, nbins = ix.export_keys()
    ok = case.oindex.keys
    bnd = case.oindex.margin < 1e-5
    mism = (keys != ok).any(axis=1)
    assert not (mism & ~bnd).any(), np.flatnonzero(mism & ~bnd)[:10]
    for l in range(case.wl.L):
        assert nbins[l] == len(case.oindex.buckets[l]) or bnd.any()


def test_query_stages_match_oracle(built, oracle_queries):
    case, ctx, d, ix = built
    wl = case.wl
    oq, wk = oracle_queries
    lr = torch.from_numpy(case.lr).cuda()
    r = __import__("paper_1004_3980_gb300").query(ix, lr, G.params(wl))
    torch.cuda.synchronize()
    keys = r["keys"].cpu().numpy().view(np.uint64)
    qb = oq.margin < 1e-5
    kmis = (keys != oq.keys).any(axis=1)
    assert not (kmis & ~qb).any()
    np.testing.assert_allclose(r["mu"].cpu().numpy(), oq.mu, atol=1e-6)
    # bucket sizes (the similarity-check count of the paper) where keys agree;
    # a boundary-affected dictionary entry may sit in a neighbouring bin
    nb_dict_bnd = int((case.oindex.margin < 1e-5).sum())
    bs = r["bucket_sum"].cpu().numpy()
    assert (np.abs(bs - oq.n_bucket)[~qb] <= wl.L * max(nb_dict_bnd, 0)).all()
    assert (bs[~qb] == oq.n_bucket[~qb]).mean() > 0.95
    ex = G.tie_or_boundary(oq, wl.K, case.oindex.margin)
    nbr = r["nbr"].cpu().numpy()
    bad = (nbr != oq.nbr[:, :wl.K]).any(axis=1) & ~ex
    assert not bad.any(), (np.flatnonzero(bad)[:10], ex.sum())
    assert ex.mean() < 0.02, ex.mean()
    dist = r["dist"].cpu().numpy()
    ok = ~ex
    np.testing.assert_allclose(dist[ok], oq.dist[ok, :wl.K], rtol=1e-5, atol=1e-7)
    wgt = r["wgt"].cpu().numpy()
    np.testing.assert_allclose(wgt.sum(axis=1), 1.0, atol=1e-5)
    assert np.abs(wgt[ok] - wk[ok]).max() < 2e-3
    st = ctx.stats()
    assert st["n_queries"] == len(nbr)
    assert abs(st["mean_bucket_sum"] - oq.n_bucket.mean()) <= 1e-2 * oq.n_bucket.mean()


def test_reconstruct_injected_neighbours(built, oracle_queries):
    case, ctx, d, ix = built
    wl = case.wl
    oq, wk = oracle_queries
    import paper_1004_3980_gb300 as Z
    nbr = torch.from_numpy(oq.nbr[:, :wl.K].astype(np.int32)).cuda()
    wgt = torch.from_numpy(wk.astype(np.float32)).cuda()
    mu = torch.from_numpy(oq.mu.astype(np.float32)).cuda()
    hr = Z.reconstruct(ix, nbr, wgt, mu, wl.lr_h, wl.lr_w).cpu().numpy()
    ref = O.reconstruct(oq.nbr[:, :wl.K], wgt.cpu().numpy().astype(np.float64), mu.cpu().numpy().astype(np.float64),
                        case.odict, wl.lr_h, wl.lr_w)
    assert np.abs(hr - ref).max() < 1e-3


@pytest.mark.parametrize("s", [2, 3])
def test_backproject_matches_oracle(built, s):
    case, ctx, d, ix = built
    import paper_1004_3980_gb300 as Z
    y = S.make_image(77, 40, 52)
    x0 = np.kron(y, np.ones((s, s))).astype(np.float32) + 0.01 * S.make_image(78, 40 * s, 52 * s)
    p = Z.UpscaleParams(bp_iters=4)
    hr = torch.from_numpy(x0).cuda()
    Z.backproject(ctx, torch.from_numpy(y).cuda(), hr, s, p)
    ref = O.back_project(x0, y, s, 0.8, 4, 1.5, 0.1, 3)
    assert np.abs(hr.cpu().numpy() - ref).max() < 1e-3


def test_upscale_end_to_end(built, oracle_queries):
    case, ctx, d, ix = built
    wl = case.wl
    oq, wk = oracle_queries
    import paper_1004_3980_gb300 as Z
    lr_t = torch.from_numpy(case.lr).cuda()
    hr = Z.upscale(ix, lr_t, G.params(wl)).cpu().numpy()
    x0 = O.reconstruct(oq.nbr[:, :wl.K], wk, oq.mu, case.odict, wl.lr_h, wl.lr_w)
    ref = O.back_project(x0, case.lr, wl.scale, wl.blur_sigma, wl.bp_iters, wl.sigma_spatial,
                         wl.sigma_range, wl.bp_radius)
    # queries whose neighbour list differs (allowed only where a projection is
    # on a bin boundary or distances tie) are left out together with every HR
    # pixel they reach through their patch and the back-projection windows
    nbr = Z.query(ix, lr_t, G.params(wl))["nbr"].cpu().numpy()
    ex = G.tie_or_boundary(oq, wl.K, case.oindex.margin)
    differ = (nbr != oq.nbr[:, :wl.K]).any(axis=1)
    assert not (differ & ~ex).any()
    P, s = wl.patch, wl.scale
    nw = wl.lr_w - P + 1
    mask = np.zeros_like(ref, bool)
    reach = wl.bp_iters * (wl.bp_radius + s + 1)
    for q in np.flatnonzero(differ):
        i, j = divmod(q, nw)
        mask[max(0, s * i - reach):s * i + s * P + reach, max(0, s * j - reach):s * j + s * P + reach] = True
    assert mask.mean() < 0.25, (differ.sum(), mask.mean())
    assert np.abs(hr - ref)[~mask].max() < 1e-3
    # the back-projection moves the degraded output toward the LR input
    r0 = np.linalg.norm(O.degrade(x0, s, 0.8) - case.lr)
    r1 = np.linalg.norm(O.degrade(hr.astype(np.float64), s, 0.8) - case.lr)
    assert r1 < r0


def test_own_patches_give_one_hot_and_exact_hr(built):
    # dictionary cut from the HR image of the query itself: every query finds
    # itself at distance 0 (one-hot weight) and the HR image is reproduced
    case, ctx, d, ix = built
    import paper_1004_3980_gb300 as Z
    s, P = 2, 5
    hr = S.make_image(31, 24 * s, 20 * s)
    lr = O.degrade(hr.astype(np.float64), s, 0.8).astype(np.float32)
    pos = np.array([(0, i, j) for i in range(24 - P + 1) for j in range(20 - P + 1)], np.int32)
    dd = Z.Dictionary(ctx, [torch.from_numpy(hr).cuda()], pos, s, P)
    alpha, beta = S.lsh_draws(3, 4, 6, P * P, 4.0)
    ii = Z.Index(dd, 4, 6, 4.0, alpha, beta)
    p = Z.UpscaleParams(K=4, bp_iters=0)
    lr_t = torch.from_numpy(lr).cuda()
    r = Z.query(ii, lr_t, p)
    assert (r["dist"][:, 0] == 0).all()
    nbr0 = r["nbr"][:, 0].cpu().numpy()
    assert (nbr0 == np.arange(len(pos))).all()
    assert (r["wgt"][:, 0] == 1).all() and (r["wgt"][:, 1:] == 0).all()
    out = Z.upscale(ii, lr_t, p).cpu().numpy()
    assert np.abs(out - hr).max() < 1e-6
    assert ctx.stats()["n_exact_match"] == len(pos)


def test_small_candidate_sets_are_padded(built):
    # t = L (an ID must share the bin in every table) leaves some queries with
    # fewer than K candidates; they are padded with the nearest non-members.
    case, ctx, d, _ = built
    wl = case.wl
    import paper_1004_3980_gb300 as Z
    L, k, w = 4, 4, 0.1          # fine bins: few entries share a query's bin in all tables
    alpha, beta = S.lsh_draws(23, L, k, wl.patch ** 2, w)
    ix = Z.Index(d, L, k, w, alpha, beta, min_table_hits=L)
    oindex = O.build_index(case.odict, alpha, beta, w, L, k)
    lr = case.lr[:20, :24]
    r = Z.query(ix, torch.from_numpy(np.ascontiguousarray(lr)).cuda(), G.params(wl, K=8))
    nbr = r["nbr"].cpu().numpy()
    oq = O.query(lr, case.odict, oindex, 9, wl.reg_rel, min_hits=L)
    ex = G.tie_or_boundary(oq, 8, oindex.margin)
    assert (oq.n_padded > 0).any()
    bad = (nbr != oq.nbr[:, :8]).any(axis=1) & ~ex
    assert not bad.any()
    assert ctx.stats()["n_padded_queries"] == int((oq.n_cand < 8).sum())


@pytest.mark.parametrize("K", [1, 12])
def test_other_K(built, K):
    case, ctx, d, ix = built
    wl = case.wl
    lr = np.ascontiguousarray(case.lr[:17, :29])      # ragged
    r = __import__("paper_1004_3980_gb300").query(ix, torch.from_numpy(lr).cuda(), G.params(wl, K=K))
    oq = O.query(lr, case.odict, case.oindex, K + 1, wl.reg_rel)
    ex = G.tie_or_boundary(oq, K, case.oindex.margin)
    nbr = r["nbr"].cpu().numpy()
    assert not ((nbr != oq.nbr[:, :K]).any(axis=1) & ~ex).any()
    w = r["wgt"].cpu().numpy()
    np.testing.assert_allclose(w.sum(1), 1, atol=1e-5)
    if K == 1:
        assert (w == 1).all()


def test_fp64_solve_when_condition_bound_exceeds_threshold(built, oracle_queries):
    case, ctx, d, ix = built
    wl = case.wl
    lr = np.ascontiguousarray(case.lr[:12, :12])
    import paper_1004_3980_gb300 as Z
    r = Z.query(ix, torch.from_numpy(lr).cuda(), G.params(wl, reg_rel=1e-9))
    st = ctx.stats()
    nq = (12 - wl.patch + 1) ** 2
    assert st["n_fp64_solves"] + st["n_exact_match"] == nq
    oq = O.query(lr, case.odict, case.oindex, wl.K, 1e-9)
    ex = G.tie_or_boundary(oq, wl.K - 1, case.oindex.margin)
    ok = ~ex & (r["nbr"].cpu().numpy() == oq.nbr).all(axis=1)
    w = r["wgt"].cpu().numpy()
    np.testing.assert_allclose(w[ok], oq.wgt[ok], atol=5e-3)
    np.testing.assert_allclose(w.sum(1), 1, atol=1e-5)


def test_single_patch_row_and_column(built):
    case, ctx, d, ix = built
    wl = case.wl
    import paper_1004_3980_gb300 as Z
    # an image of exactly one patch: the first patch position along the
    # diagonal whose query is clear of bin boundaries and ties (the check
    # below then always runs)
    for o in range(0, 20):
        lr = np.ascontiguousarray(case.lr[o:o + wl.patch, o:o + wl.patch])
        oq1 = O.query(lr, case.odict, case.oindex, wl.K + 1, wl.reg_rel)
        if not O.neighbour_exclusions(oq1.feat, oq1.margin, oq1.dist, case.odict, case.oindex)[0]:
            break
    else:
        pytest.fail("no clear single-patch image on the diagonal")
    out = Z.upscale(ix, torch.from_numpy(lr).cuda(), G.params(wl)).cpu().numpy()
    oq = O.query(lr, case.odict, case.oindex, wl.K, wl.reg_rel)
    x0 = O.reconstruct(oq.nbr, oq.wgt, oq.mu, case.odict, wl.patch, wl.patch)
    ref = O.back_project(x0, lr, wl.scale, 0.8, wl.bp_iters, 1.5, 0.1, 3)
    assert out.shape == (wl.scale * wl.patch,) * 2
    assert np.abs(out - ref).max() < 1e-3


def test_argument_errors(built):
    case, ctx, d, ix = built
    import paper_1004_3980_gb300 as Z
    from paper_1004_3980_gb300.capi import ZoomError
    lr = torch.from_numpy(case.lr).cuda()
    with pytest.raises(ZoomError, match="INVALID_ARG"):
        Z.upscale(ix, lr[:2, :2].contiguous(), G.params(case.wl))
    with pytest.raises(ZoomError, match="INVALID_ARG"):
        Z.upscale(ix, lr, G.params(case.wl, K=0))
    from paper_1004_3980_gb300 import capi
    import ctypes as C
    p = G.params(case.wl).c()
    out = torch.empty((3 * 64, 3 * 64), device="cuda")
    rc = capi.lib().zoom_upscale(ix.handle, C.c_void_p(lr.data_ptr()), 64, 64, 3, C.byref(p),
                                 C.c_void_p(out.data_ptr()), None)
    assert rc == 1 and b"scale" in capi.lib().zoom_last_error()
    ctx.sync_status()
