"""Batched zoom (zoom_upscale_batch): many LR images of uneven sizes and two
scales in one call, searched per scale by one persistent launch and replayed
from a recorded CUDA graph.  In the exact FP32 form every image must equal
its own zoom_upscale output bit for bit (batching changes no arithmetic of a
query); the BF16 form must stay within 50 dB PSNR of the exact form."""
import numpy as np
import pytest

import synth_inputs as S
from oracle import zoom_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def two_scales():
    from paper_1004_3980_gb300 import build
    build.build()
    import paper_1004_3980_gb300 as Z
    ctx = Z.Context(0)
    idx = {}
    for s, hrs in ((2, 96), (3, 144)):
        train = [S.make_image(3000 + 10 * s + i, hrs, hrs) for i in range(3)]
        pos = S.sample_positions(7, 3, hrs // s, hrs // s, 5, 5000)
        alpha, beta = S.lsh_draws(11, 8, 10, 25, 4.0)
        d = Z.Dictionary(ctx, [torch.from_numpy(x).cuda() for x in train], pos, s, 5)
        idx[s] = (Z.Index(d, 8, 10, 4.0, alpha, beta), d, train, pos, alpha, beta)
    shapes = [(2, 20, 24), (3, 31, 17), (2, 40, 56), (3, 22, 29), (2, 9, 13), (3, 35, 40)]
    imgs = [(s, S.make_image(3100 + i, h, w)) for i, (s, h, w) in enumerate(shapes)]
    return ctx, idx, imgs


def _single(ix, lr, p):
    import paper_1004_3980_gb300 as Z
    return Z.upscale(ix, torch.from_numpy(lr).cuda(), p).cpu().numpy()


def test_batch_equals_single_image_calls_exact(two_scales):
    import paper_1004_3980_gb300 as Z
    ctx, idx, imgs = two_scales
    p = Z.UpscaleParams(K=8, bp_iters=3)
    lrs = [(s, torch.from_numpy(x).cuda()) for s, x in imgs]
    indexes = [idx[2][0], idx[3][0]]
    outs, lat = Z.upscale_batch(indexes, lrs, p, want_latency=True)
    for (s, x), o in zip(imgs, outs):
        ref = _single(idx[s][0], x, p)
        assert np.array_equal(o.cpu().numpy(), ref)
    assert all(t > 0 for t in lat)
    # second call replays the recorded graph on new contents of the same buffers
    new = [S.make_image(3200 + i, *x.shape) for i, (s, x) in enumerate(imgs)]
    for (s, t), n in zip(lrs, new):
        t.copy_(torch.from_numpy(n))
    outs2, _ = Z.upscale_batch(indexes, lrs, p, outs=outs)
    for (s, _), n, o in zip(imgs, new, outs2):
        assert np.array_equal(o.cpu().numpy(), _single(idx[s][0], n, p))
    Z.batch_release(ctx)


def test_batch_bf16_close_to_exact(two_scales):
    import paper_1004_3980_gb300 as Z
    ctx, idx, imgs = two_scales
    indexes = [idx[2][0], idx[3][0]]
    lrs = [(s, torch.from_numpy(x).cuda()) for s, x in imgs]
    ex, _ = Z.upscale_batch(indexes, lrs, Z.UpscaleParams(K=8, bp_iters=3))
    ex = [o.clone() for o in ex]
    pr, _ = Z.upscale_batch(indexes, lrs, Z.UpscaleParams(K=8, bp_iters=3, precision=1, rerank_mult=2))
    for a, b in zip(ex, pr):
        mse = float(((a - b) ** 2).mean())
        assert 10 * np.log10(1.0 / max(mse, 1e-30)) >= 50.0
    Z.batch_release(ctx)


def test_batch_image_matches_oracle(two_scales):
    # one 3x image of the batch (31 x 17) against the FP64 oracle end to end
    import paper_1004_3980_gb300 as Z
    ctx, idx, imgs = two_scales
    ix, d, train, pos, alpha, beta = idx[3]
    s, lr = imgs[1]
    p = Z.UpscaleParams(K=8, bp_iters=3)
    outs, _ = Z.upscale_batch([idx[2][0], ix], [(s2, torch.from_numpy(x).cuda()) for s2, x in imgs], p)
    od = O.build_dictionary(train, pos, 3, 5, 0.8)
    oi = O.build_index(od, alpha, beta, 4.0, 8, 10)
    x, oq, _ = O.upscale(lr, od, oi, 8, 1e-3, 3, 0.8, 1.5, 0.1, 3)
    # max-abs on every HR pixel no excluded query (bin boundary or tie) can
    # reach: each one's patch footprint, grown by what 3 back-projection
    # steps spread (7 x 7 window, 3-tap blur, 3 x 3 blocks: 3 * (3 + 1 + 3))
    oq9 = O.query(lr, od, oi, 9, 1e-3)
    ex = O.neighbour_exclusions(oq9.feat, oq9.margin, oq9.dist, od, oi)
    assert ex.mean() < 0.02, ex.sum()
    s, PH, nw = 3, 15, lr.shape[1] - 4
    reach = np.zeros((s * lr.shape[0], s * lr.shape[1]), bool)
    g = 3 * (3 + 1 + 3)
    for n in np.flatnonzero(ex):
        i, j = divmod(int(n), nw)
        reach[max(0, s * i - g):s * i + PH + g, max(0, s * j - g):s * j + PH + g] = True
    out = outs[1].cpu().numpy()
    assert (~reach).mean() > 0.5
    assert np.abs(out - x)[~reach].max() < 1e-3
    mse = float(np.mean((out - x) ** 2))
    assert 10 * np.log10(1.0 / mse) >= 50.0
    Z.batch_release(ctx)
