"""The 3x zoom of a 1920 x 1080 LR image with the 4,000,000-pair dictionary
(5x5 LR / 15x15 HR patches, L = 16, k = 18, K = 8), the configuration the
default bench line times, in both forms:
  * 48 sampled queries against the oracle (keys, exact K nearest over the
    candidate sets -- most of the 4M entries -- and LLE weights); the BF16
    form's recall of the oracle's neighbours on them;
  * every query of the exact form equal to the SIMT scan;
  * the BF16 form (the best 32 chunks reranked in FP32) against the exact
    form over every query and every HR pixel: recall >= 0.99, PSNR >= 50 dB;
  * with a dictionary one entry past the packed list keys' limit, the BF16
    form's unpacked 32-chunk lists against the exact form."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import synth_inputs as S
from oracle import zoom_oracle as O
from tests import gpu_cases as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WL = S.WORKLOADS["zoom3x_1920x1080_dict4m"]
N_SAMPLE = 48


@pytest.fixture(scope="module")
def big():
    from paper_1004_3980_gb300 import build
    build.build()
    import paper_1004_3980_gb300 as Z
    wl = WL
    train = S.training_images(wl)
    lrs = wl.train_hr // wl.scale
    pos = S.sample_positions(wl.pos_seed, len(train), lrs, lrs, wl.patch, wl.n_pairs)
    alpha, beta = S.lsh_draws(wl.proj_seed, wl.L, wl.k, wl.patch ** 2, wl.w)
    lr = S.test_image(wl)
    ctx = Z.Context(0)
    d = Z.Dictionary(ctx, [torch.from_numpy(x).cuda() for x in train], pos, wl.scale, wl.patch, wl.blur_sigma)
    ix = Z.Index(d, wl.L, wl.k, wl.w, alpha, beta)
    lr_t = torch.from_numpy(lr).cuda()
    q_ex = Z.query(ix, lr_t, G.params(wl))
    q_bf = Z.query(ix, lr_t, G.params(wl, precision=1, rerank_mult=4))
    ctx.sync_status()
    return dict(Z=Z, wl=wl, lr=lr, lr_t=lr_t, ctx=ctx, d=d, ix=ix, train=train, pos=pos, alpha=alpha,
                beta=beta, q_ex=q_ex, q_bf=q_bf)


def test_sampled_queries_match_oracle_3x(big):
    wl, lr = big["wl"], big["lr"]
    od = O.build_dictionary(big["train"], big["pos"], wl.scale, wl.patch, wl.blur_sigma, with_hr=False)
    oix = O.build_index(od, big["alpha"], big["beta"], wl.w, wl.L, wl.k)
    nq = (wl.lr_h - wl.patch + 1) * (wl.lr_w - wl.patch + 1)
    rows = np.sort(np.random.default_rng(61).choice(nq, N_SAMPLE, replace=False))
    oq = G.oracle_rows(lr, od, oix, wl.K + 1, wl.reg_rel, rows)
    fn = (od.feat * od.feat).sum(axis=1)
    parts = np.array_split(np.arange(N_SAMPLE), min(N_SAMPLE, os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=len(parts)) as exe:
        exs = list(exe.map(lambda p: O.neighbour_exclusions(oq.feat[p], oq.margin[p], oq.dist[p], od, oix,
                                                            feat_norm2=fn), parts))
    ex = np.concatenate(exs)
    print(f"\n{ex.sum()} of {N_SAMPLE} sampled queries excluded (boundary or tie)")
    assert ex.sum() <= 2
    qk = big["q_ex"]["keys"].cpu().numpy().view(np.uint64)[rows]
    ok = oq.margin >= 1e-5
    assert np.array_equal(qk[ok], oq.keys[ok])
    nbr = big["q_ex"]["nbr"].cpu().numpy()[rows]
    dist = big["q_ex"]["dist"].cpu().numpy()[rows]
    wgt = big["q_ex"]["wgt"].cpu().numpy()[rows]
    bad = (nbr != oq.nbr[:, :wl.K]).any(axis=1) & ~ex
    assert not bad.any(), rows[bad]
    np.testing.assert_allclose(dist[~ex], oq.dist[~ex, :wl.K], rtol=2e-5, atol=1e-7)
    for i in np.flatnonzero(~ex):
        w_o, _ = O.lle_weights(oq.feat[i], od.feat[oq.nbr[i, :wl.K]], wl.reg_rel, oq.dist[i, 0])
        np.testing.assert_allclose(wgt[i], w_o, atol=2e-3)
    # the precision form's recall of the oracle's K nearest
    nb_bf = big["q_bf"]["nbr"].cpu().numpy()[rows]
    rec = np.mean([len(np.intersect1d(a, b)) / wl.K for a, b in zip(nb_bf[~ex], oq.nbr[~ex, :wl.K])])
    assert rec >= 0.99, rec
    assert 0.5 < oq.n_cand.mean() / od.n < 1.0


def test_every_query_equals_the_scan_3x(big):
    Z, wl = big["Z"], big["wl"]
    a = Z.query(big["ix"], big["lr_t"], G.params(wl, search=1))
    b = big["q_ex"]
    assert torch.equal(a["nbr"], b["nbr"]) and torch.equal(a["dist"], b["dist"])


def test_bf16_form_against_the_exact_form_3x(big):
    Z, wl = big["Z"], big["wl"]
    ne, nb = big["q_ex"]["nbr"], big["q_bf"]["nbr"]
    hits = torch.zeros(ne.shape[0], dtype=torch.int32, device="cuda")
    for m in range(wl.K):
        hits += (nb == ne[:, m:m + 1]).any(dim=1).int()
    recall = float(hits.double().mean()) / wl.K
    assert recall >= 0.99, recall
    x_e = Z.upscale(big["ix"], big["lr_t"], G.params(wl))
    x_b = Z.upscale(big["ix"], big["lr_t"], G.params(wl, precision=1, rerank_mult=4))
    mse = float(((x_e.double() - x_b.double()) ** 2).mean())
    psnr = 10 * np.log10(1.0 / max(mse, 1e-30))
    print(f"\nBF16 vs exact: recall {recall:.6f} over {ne.shape[0]} queries, PSNR {psnr:.1f} dB")
    assert psnr >= 50.0


def test_bf16_32_chunk_lists_past_the_packed_key_limit(big):
    # One entry past 4,194,304 the chunk numbers need 18 bits, more than the
    # packed list keys leave room for: the BF16 form keeps its 32-chunk lists
    # as (value, index) pairs there.  Same training images, a crop of the test
    # image; recall of the exact form's neighbours.
    Z, wl = big["Z"], big["wl"]
    n = 4_194_305
    lrs = wl.train_hr // wl.scale
    pos = S.sample_positions(wl.pos_seed + 1, len(big["train"]), lrs, lrs, wl.patch, n)
    d = Z.Dictionary(big["ctx"], [torch.from_numpy(x).cuda() for x in big["train"]], pos, wl.scale, wl.patch,
                     wl.blur_sigma)
    ix = Z.Index(d, wl.L, wl.k, wl.w, big["alpha"], big["beta"])
    lr_c = big["lr_t"][:96, :160].contiguous()
    q_ex = Z.query(ix, lr_c, G.params(wl))
    q_bf = Z.query(ix, lr_c, G.params(wl, precision=1, rerank_mult=4))
    scan = Z.query(ix, lr_c, G.params(wl, search=1))
    big["ctx"].sync_status()
    assert torch.equal(q_ex["nbr"], scan["nbr"]) and torch.equal(q_ex["dist"], scan["dist"])
    ne, nb = q_ex["nbr"], q_bf["nbr"]
    hits = sum((nb == ne[:, m:m + 1]).any(dim=1).int() for m in range(wl.K))
    recall = float(hits.double().mean()) / wl.K
    assert recall >= 0.99, recall
    assert int(nb.min()) >= 0 and int(nb.max()) < n
    ix.close()
    d.close()
