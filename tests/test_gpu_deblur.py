"""De-blurring (scale 1: blur only), the second workload the paper shows:
the same per-patch inference with P x P HR patches, the back-projection of a
blur-only degradation; compared with the oracle end to end."""
import dataclasses

import numpy as np
import pytest

import synth_inputs as S
from oracle import zoom_oracle as O
from tests import gpu_cases as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def deblur():
    from paper_1004_3980_gb300 import build
    build.build()
    import paper_1004_3980_gb300 as Z
    wl = dataclasses.replace(S.WORKLOADS["zoom2x_64_dict20k"], scale=1, n_pairs=8000, lr_h=40, lr_w=44)
    train = S.training_images(wl, 4)
    lrs = wl.train_hr // wl.scale
    pos = S.sample_positions(wl.pos_seed, len(train), lrs, lrs, wl.patch, wl.n_pairs)
    alpha, beta = S.lsh_draws(wl.proj_seed, wl.L, wl.k, wl.patch ** 2, wl.w)
    # the blurred observation of a sharp test image
    sharp = S.make_image(77, wl.lr_h, wl.lr_w)
    lr = O.degrade(sharp.astype(np.float64), 1, wl.blur_sigma).astype(np.float32)
    odict = O.build_dictionary(train, pos, 1, wl.patch, wl.blur_sigma)
    oindex = O.build_index(odict, alpha, beta, wl.w, wl.L, wl.k)
    ctx = Z.Context(0)
    d = Z.Dictionary(ctx, [torch.from_numpy(x).cuda() for x in train], pos, 1, wl.patch, wl.blur_sigma)
    ix = Z.Index(d, wl.L, wl.k, wl.w, alpha, beta)
    return wl, lr, sharp, odict, oindex, ctx, d, ix


def test_deblur_matches_oracle(deblur):
    import paper_1004_3980_gb300 as Z
    wl, lr, sharp, odict, oindex, ctx, d, ix = deblur
    lr_t = torch.from_numpy(lr).cuda()
    p = G.params(wl, search=1)
    r = Z.query(ix, lr_t, p)
    oq = O.query(lr, odict, oindex, wl.K + 1, wl.reg_rel)
    ex = G.tie_or_boundary(oq, wl.K, oindex.margin)
    nbr = r["nbr"].cpu().numpy()
    differ = (nbr != oq.nbr[:, :wl.K]).any(axis=1)
    assert not (differ & ~ex).any()
    # HR (same size as the input) against the oracle, away from differing queries
    hr = Z.upscale(ix, lr_t, p).cpu().numpy()
    wk = np.stack([O.lle_weights(oq.feat[q], odict.feat[oq.nbr[q, :wl.K]], wl.reg_rel, oq.dist[q, 0])[0]
                   for q in range(len(oq.nbr))])
    x0 = O.reconstruct(oq.nbr[:, :wl.K], wk, oq.mu, odict, wl.lr_h, wl.lr_w)
    ref = O.back_project(x0, lr, 1, wl.blur_sigma, wl.bp_iters, wl.sigma_spatial, wl.sigma_range,
                         wl.bp_radius)
    assert hr.shape == lr.shape == ref.shape
    P = wl.patch
    nw = wl.lr_w - P + 1
    mask = np.zeros_like(ref, bool)
    reach = wl.bp_iters * (wl.bp_radius + 2)
    for q in np.flatnonzero(differ):
        i, j = divmod(q, nw)
        mask[max(0, i - reach):i + P + reach, max(0, j - reach):j + P + reach] = True
    assert mask.mean() < 0.25
    assert np.abs(hr - ref)[~mask].max() < 1e-3
    # the restoration is closer to the sharp image than the blurred input
    assert np.abs(hr - sharp).mean() < np.abs(lr - sharp).mean()
    # the tensor-core path gives the SIMT scan's neighbours here too
    r2 = Z.query(ix, lr_t, G.params(wl, search=2))
    assert torch.equal(r2["nbr"], r["nbr"])
