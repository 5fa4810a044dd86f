"""Blend + overlap average (Eq. 14 and the averaging of overlaps) in its two
GPU forms: the two-pass form (blended patches staged in scratch, used by
zoom_reconstruct, zoom_upscale and the batch) and the one-pass gather form
(zoom_reconstruct_with) give the same bits for every scale, patch size and
neighbour count, on images whose patch rows are not a multiple of the
32-query blocks and whose HR patches take one or two shared-memory rounds;
both are checked against the oracle's FP64 average."""
import numpy as np
import pytest

import synth_inputs as S
from oracle import zoom_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_1004_3980_gb300 import build
    build.build()
    import paper_1004_3980_gb300 as Z
    return Z.Context(0)


# (s, P): HR patches of 100, 225, 144 and 36 pixels (225 and 144 take two
# 128-pixel rounds of the blend pass)
@pytest.mark.parametrize("s,P", [(2, 5), (3, 5), (4, 3), (2, 3)])
@pytest.mark.parametrize("K", [1, 8, 13, 64])
def test_two_pass_equals_one_pass_and_oracle(ctx, s, P, K):
    import paper_1004_3980_gb300 as Z
    train = [S.make_image(50 + m, 48 * s, 40 * s) for m in range(2)]
    pos = S.sample_positions(7, 2, 48, 40, P, 3000)
    d = Z.Dictionary(ctx, [torch.from_numpy(x).cuda() for x in train], pos, s, P, 0.8)
    alpha, beta = S.lsh_draws(3, 2, 4, P * P, 4.0)
    ix = Z.Index(d, 2, 4, 4.0, alpha, beta)
    h, w = 37, 3 * 32 + P + 4                 # 3 full blocks of 32 queries + a ragged 5th
    nq = (h - P + 1) * (w - P + 1)
    rng = np.random.default_rng(s * 100 + P * 10 + K)
    nbr = rng.integers(0, d.n, (nq, K)).astype(np.int32)
    wgt = (rng.random((nq, K)) / K).astype(np.float32)
    mu = rng.random(nq).astype(np.float32)
    nbr_t, wgt_t, mu_t = (torch.from_numpy(a).cuda() for a in (nbr, wgt, mu))
    two = Z.reconstruct(ix, nbr_t, wgt_t, mu_t, h, w)
    lr_pix, _, hres = d.export()
    one = Z.reconstruct_with(ix, torch.from_numpy(hres).cuda(), nbr_t, wgt_t, mu_t, h, w)
    assert two.shape == (s * h, s * w)
    assert torch.equal(two, one)
    od = O.Dictionary(s, P, lr_pix.astype(np.float64), None, None, hres.astype(np.float64))
    ref = O.reconstruct(nbr, wgt.astype(np.float64), mu.astype(np.float64), od, h, w)
    np.testing.assert_allclose(two.cpu().numpy(), ref, rtol=0, atol=2e-6)


def test_single_patch_image(ctx):
    # an image of exactly one patch: every HR pixel has one covering patch
    import paper_1004_3980_gb300 as Z
    s, P = 2, 5
    train = [S.make_image(60, 40, 40)]
    pos = S.sample_positions(8, 1, 20, 20, P, 200)
    d = Z.Dictionary(ctx, [torch.from_numpy(train[0]).cuda()], pos, s, P, 0.8)
    alpha, beta = S.lsh_draws(3, 2, 4, P * P, 4.0)
    ix = Z.Index(d, 2, 4, 4.0, alpha, beta)
    nbr = torch.tensor([[3, 7]], dtype=torch.int32).cuda()
    wgt = torch.tensor([[0.25, 0.75]], dtype=torch.float32).cuda()
    mu = torch.tensor([0.5], dtype=torch.float32).cuda()
    out = Z.reconstruct(ix, nbr, wgt, mu, P, P).cpu().numpy()
    _, _, hres = d.export()
    ref = (0.5 + 0.25 * hres[3].astype(np.float64) + 0.75 * hres[7]).reshape(s * P, s * P)
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-6)
