"""Tensor-core neighbour search (tcgen05): the exact form -- the single-term
FP16 filter with its proven FP32 rerank, the FP16-split filter as its
second stage, and the split filter alone -- must return exactly the
neighbours of the SIMT scan (all follow the same (member, distance, ID)
order), and the BF16 precision form must keep its recall against exact
search."""
import numpy as np
import pytest

import synth_inputs as S
from oracle import zoom_oracle as O
from tests import gpu_cases as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def small():
    from paper_1004_3980_gb300 import build
    build.build()
    case = G.small_case()
    ctx, d, ix = G.gpu_build(case)
    return case, ctx, d, ix


def _query(ix, lr, wl, **kw):
    import paper_1004_3980_gb300 as Z
    r = Z.query(ix, torch.from_numpy(np.ascontiguousarray(lr)).cuda(), G.params(wl, **kw))
    return {k: v.cpu().numpy() for k, v in r.items()}


def test_tc_tiny_runs_and_matches_scan(small):
    case, ctx, d, ix = small
    wl = case.wl
    lr = case.lr[:20, :20]
    a = _query(ix, lr, wl, search=1)
    b = _query(ix, lr, wl, search=2)
    ctx.sync_status()
    assert (a["nbr"] == b["nbr"]).all()
    assert (a["dist"] == b["dist"]).all()


def test_tc_exact_equals_scan_on_small_workload(small):
    case, ctx, d, ix = small
    wl = case.wl
    a = _query(ix, case.lr, wl, search=1)
    b = _query(ix, case.lr, wl, search=2)
    st = ctx.stats()
    ctx.sync_status()
    assert (a["nbr"] == b["nbr"]).all()
    assert (a["dist"] == b["dist"]).all()
    np.testing.assert_array_equal(a["wgt"], b["wgt"])
    # the rerank settles nearly every query without the scan
    assert st["n_filter_fallback"] < 0.05 * st["n_queries"], st


@pytest.mark.parametrize("K", [1, 5, 12, 16])
def test_tc_exact_other_K_and_ragged(small, K):
    case, ctx, d, ix = small
    wl = case.wl
    lr = case.lr[3:40, 5:58]
    a = _query(ix, lr, wl, search=1, K=K)
    b = _query(ix, lr, wl, search=2, K=K)
    assert (a["nbr"] == b["nbr"]).all() and (a["dist"] == b["dist"]).all()


def test_tc_exact_with_t_of_L(small):
    case, ctx, d, _ = small
    wl = case.wl
    import paper_1004_3980_gb300 as Z
    ix2 = Z.Index(d, wl.L, wl.k, wl.w, case.alpha, case.beta, min_table_hits=3)
    a = _query(ix2, case.lr[:30, :30], wl, search=1)
    b = _query(ix2, case.lr[:30, :30], wl, search=2)
    assert (a["nbr"] == b["nbr"]).all() and (a["dist"] == b["dist"]).all()


@pytest.mark.parametrize("rerank_mult", [2, 4])
def test_bf16_precision_form_recall_and_psnr(small, rerank_mult):
    """16- and 32-chunk lists of the BF16 filter (rerank_mult * K <= 16 or 32)."""
    case, ctx, d, ix = small
    wl = case.wl
    import paper_1004_3980_gb300 as Z
    ex = _query(ix, case.lr, wl, search=1)
    pr = _query(ix, case.lr, wl, precision=1, rerank_mult=rerank_mult)
    K = wl.K
    rec = np.mean([len(set(pr["nbr"][q]) & set(ex["nbr"][q])) / K for q in range(len(ex["nbr"]))])
    assert rec >= 0.99, rec
    # PSNR of the precision form's HR output against the FP64 oracle
    hr = Z.upscale(ix, torch.from_numpy(case.lr).cuda(),
                   G.params(wl, precision=1, rerank_mult=rerank_mult)).cpu().numpy()
    x, _, _ = O.upscale(case.lr, case.odict, case.oindex, K, wl.reg_rel, wl.bp_iters, wl.blur_sigma,
                        wl.sigma_spatial, wl.sigma_range, wl.bp_radius)
    mse = float(np.mean((hr - x) ** 2))
    psnr = 10 * np.log10(1.0 / max(mse, 1e-30))
    assert psnr >= 50.0, psnr


@pytest.mark.parametrize("K", [5, 16])
def test_split_filter_alone_equals_scan(small, K):
    case, ctx, d, ix = small
    wl = case.wl
    lr = case.lr[:45, :61]
    a = _query(ix, lr, wl, search=1, K=K)
    b = _query(ix, lr, wl, search=3, K=K)
    ctx.sync_status()
    assert (a["nbr"] == b["nbr"]).all() and (a["dist"] == b["dist"]).all()


@pytest.mark.parametrize("sigma", [0.012, 0.006], ids=["second_stage", "third_stage"])
def test_later_stages_settle_what_the_single_term_filter_cannot(sigma):
    # The dictionary is one mosaic of 32 noisy copies of the test image side
    # by side: IDs run along the mosaic's rows, so a query's 32 near
    # duplicates fall in 32 different chunks of the same dictionary split,
    # within the single-term filter's error bound of one another.  Nearly
    # every query then fails that filter's proof (CPU simulation of the
    # proof with the planner's 8 splits: 96 %, resp. 99 %) and goes to the
    # split filter; with the smaller noise 40 % fail that proof too and go to
    # the SIMT scan.  The result must be the SIMT scan's.
    import paper_1004_3980_gb300 as Z
    s, P, n_copies = 2, 5, 32
    hr = S.make_image(91, 80, 88).astype(np.float64)
    lr = O.degrade(hr, s, 0.8).astype(np.float32)
    g = np.random.default_rng(4)
    mosaic = np.concatenate([np.clip(hr + g.normal(scale=sigma, size=hr.shape), 0, 1) for _ in range(n_copies)],
                            axis=1).astype(np.float32)
    lh, lw = mosaic.shape[0] // s, mosaic.shape[1] // s
    pos = np.array([(0, i, j) for i in range(lh - P + 1) for j in range(lw - P + 1)], np.int32)
    ctx = Z.Context(0)
    d = Z.Dictionary(ctx, [torch.from_numpy(mosaic).cuda()], pos, s, P, 0.8)
    alpha, beta = S.lsh_draws(3, 8, 12, P * P, 4.0)
    ix = Z.Index(d, 8, 12, 4.0, alpha, beta)
    wl = G.small_case().wl
    a = _query(ix, lr, wl, search=1)
    b = _query(ix, lr, wl, search=2)
    st = ctx.stats()
    ctx.sync_status()
    assert st["n_filter_fallback"] > 0.5 * st["n_queries"], st
    assert (a["nbr"] == b["nbr"]).all() and (a["dist"] == b["dist"]).all()
    c = _query(ix, lr, wl, search=3)
    assert (a["nbr"] == c["nbr"]).all() and (a["dist"] == c["dist"]).all()
    # the batched form (autotuning runs the search repeatedly on one
    # workspace, and a batch runs one search per group): every later stage
    # must see only its own search's unsettled queries
    p = G.params(wl, search=2)
    hr1 = Z.upscale(ix, torch.from_numpy(lr).cuda(), p)
    lr2 = torch.from_numpy(np.ascontiguousarray(lr[:, ::-1])).cuda()
    hr2 = Z.upscale(ix, lr2, p)
    outs, _ = Z.upscale_batch([ix], [torch.from_numpy(lr).cuda(), lr2], p)
    outs, _ = Z.upscale_batch([ix], [torch.from_numpy(lr).cuda(), lr2], p, outs=outs)
    Z.batch_release(ctx)
    assert torch.equal(outs[0], hr1) and torch.equal(outs[1], hr2)
