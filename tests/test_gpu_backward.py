"""Differentiation: the hand-written adjoint kernels (zoom_backward,
zoom_reconstruct_adjoint, zoom_degrade_adjoint) against the FP64 oracle's
MAP energy (Sec. 4, Eq. 5-9) and its analytic gradients, and against FP64
central finite differences (step 1e-6; the energy is quadratic, so the
differences are exact up to rounding).

Neighbours are held fixed.  Both sides use the same LLE weights: the
oracle's FP64 weights rounded to float32 (given to the GPU as input).
Gradient tolerance: |g - g_ref| <= 1e-4 * max(|g_ref|, 1e-3 * max|g_ref|)
+ a floor for the FP32 arithmetic: the GPU forms the HR image x with at
most K + 1 rounded operations per pixel and the residual D B x - y with one
more, so every gradient element carries an absolute error up to about
2 (K + 2) 2^-24 max|x| (the adjoint maps have unit row sums).
"""
import numpy as np
import pytest

import synth_inputs as S
from oracle import zoom_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LAM = 0.1


def fp32_floor(K, xmax=1.0):
    return 2.0 * (K + 2) * 2.0 ** -24 * xmax


def _close(g, ref, rel=1e-4, K=8):
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    tol = rel * np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max()) + fp32_floor(K)
    bad = np.abs(g - ref) > tol
    return not bad.any(), (int(bad.sum()), float(np.abs(g - ref).max()))


def _setup(train, pos, lr, s, P, nbr, L=4, k=4):
    import paper_1004_3980_gb300 as Z
    ctx = Z.Context(0)
    d = Z.Dictionary(ctx, [torch.from_numpy(x).cuda() for x in train], pos, s, P)
    alpha, beta = S.lsh_draws(5, L, k, P * P, 4.0)
    ix = Z.Index(d, L, k, 4.0, alpha, beta)
    od = O.build_dictionary(train, pos, s, P, 0.8)
    v, mu = O.patch_features(lr, P)
    K = nbr.shape[1]
    w64 = np.stack([O.lle_weights(v[q], od.feat[nbr[q]], 1e-3, 1.0)[0] for q in range(len(nbr))])
    w32 = w64.astype(np.float32)
    return ctx, d, ix, od, mu, w32, K


@pytest.fixture(scope="module")
def small():
    from paper_1004_3980_gb300 import build
    build.build()
    s, P = 2, 5
    train = [S.make_image(2000 + i, 96, 96) for i in range(3)]
    pos = S.sample_positions(7, 3, 48, 48, P, 3000)
    lr = S.make_image(2100, 18, 16)
    nq = (18 - P + 1) * (16 - P + 1)
    nbr = np.random.default_rng(3).integers(0, 2900, size=(nq, 8))   # the last 100 entries stay unused
    ctx, d, ix, od, mu, w32, K = _setup(train, pos, lr, s, P, nbr)
    return dict(s=s, P=P, lr=lr, nbr=nbr, ctx=ctx, d=d, ix=ix, od=od, mu=mu, w32=w32, K=K)


def _gpu(c, wgt=True, lam=LAM):
    import paper_1004_3980_gb300 as Z
    r = Z.map_energy_grads(c["ix"], torch.from_numpy(c["lr"]).cuda(),
                           torch.from_numpy(c["nbr"].astype(np.int32)).cuda(),
                           torch.from_numpy(c["w32"]).cuda() if wgt else None, lam=lam)
    return r["energy"], r["grad_x"].cpu().numpy(), r["grad_dict"].cpu().numpy(), r["hr"].cpu().numpy()


def _oracle(c, lam=LAM):
    s, P, lr, nbr, od = c["s"], c["P"], c["lr"], c["nbr"], c["od"]
    h, w = lr.shape
    w64 = c["w32"].astype(np.float64)
    x = O.reconstruct(nbr, w64, c["mu"], od, h, w)
    E = O.map_energy(od.hr_res, nbr, w64, c["mu"], lr, h, w, s, P, 0.8, lam)
    gx = O.data_energy_grad(x, lr, s, 0.8)
    gR = O.map_energy_grad_dict(od.hr_res, nbr, w64, c["mu"], lr, h, w, s, P, 0.8, lam)
    return E, gx, gR, x


def test_energy_and_gradients_match_oracle(small):
    E, gx, gR, x = _gpu(small)
    Eo, gxo, gRo, xo = _oracle(small)
    assert abs(E - Eo) <= 1e-5 * abs(Eo)
    assert np.abs(x - xo).max() < 1e-5
    ok, info = _close(gx, gxo)
    assert ok, info
    ok, info = _close(gR, gRo)
    assert ok, info
    assert (gR[2900:] == 0).all()          # entries no patch uses


def test_gradients_match_central_differences(small):
    c = small
    s, P, lr, nbr, od = c["s"], c["P"], c["lr"], c["nbr"], c["od"]
    h, w = lr.shape
    w64 = c["w32"].astype(np.float64)
    E, gx, gR, x = _gpu(c)
    xo = O.reconstruct(nbr, w64, c["mu"], od, h, w)
    g = np.random.default_rng(9)
    for _ in range(100):   # 100 HR-image coordinates
        i, j = g.integers(0, s * h), g.integers(0, s * w)
        xp, xm = xo.copy(), xo.copy()
        xp[i, j] += 1e-6
        xm[i, j] -= 1e-6
        fd = (O.data_energy(xp, lr, s, 0.8) - O.data_energy(xm, lr, s, 0.8)) / 2e-6
        assert abs(gx[i, j] - fd) <= 1e-4 * max(abs(fd), 1e-3 * np.abs(gx).max()) + fp32_floor(8), (i, j, gx[i, j], fd)
    used = np.unique(nbr)
    for _ in range(100):   # 100 HR-dictionary coordinates of entries in use
        a, b = int(g.choice(used)), int(g.integers(0, (s * P) ** 2))
        Rp, Rm = od.hr_res.copy(), od.hr_res.copy()
        Rp[a, b] += 1e-6
        Rm[a, b] -= 1e-6
        fd = (O.map_energy(Rp, nbr, w64, c["mu"], lr, h, w, s, P, 0.8, LAM)
              - O.map_energy(Rm, nbr, w64, c["mu"], lr, h, w, s, P, 0.8, LAM)) / 2e-6
        assert abs(gR[a, b] - fd) <= 1e-4 * max(abs(fd), 1e-3 * np.abs(gR).max()) + fp32_floor(8), (a, b, gR[a, b], fd)


def test_recomputed_weights(small):
    # weights recomputed on the GPU in FP32 from the LR features (the Gram
    # factors are rebuilt, not stored): gradients agree with the oracle's
    # FP64-weight gradients to the FP32 solve's accuracy
    E, gx, gR, _ = _gpu(small, wgt=False)
    Eo, gxo, gRo, _ = _oracle(small)
    assert abs(E - Eo) <= 1e-3 * abs(Eo)
    ok, info = _close(gR, gRo, rel=2e-2)
    assert ok, info


def test_autograd_functions_match_fused_backward(small):
    import paper_1004_3980_gb300 as Z
    c = small
    s = c["s"]
    h, w = c["lr"].shape
    R = Z.dictionary_hr(c["d"]).requires_grad_(True)
    nbr = torch.from_numpy(c["nbr"].astype(np.int32)).cuda()
    wgt = torch.from_numpy(c["w32"]).cuda()
    mu = torch.from_numpy(c["mu"].astype(np.float32)).cuda()
    y = torch.from_numpy(c["lr"]).cuda()
    x = Z.ReconstructFunction.apply(R, c["ix"], nbr, wgt, mu, h, w)
    yh = Z.DegradeFunction.apply(x, c["ctx"], s, 0.8)
    loss = ((yh - y) ** 2).sum()
    loss.backward()
    _, _, gR, _ = _gpu(c, lam=0.0)
    _, _, gRo, _ = _oracle(c, lam=0.0)
    ok, info = _close(R.grad.cpu().numpy(), gRo)
    assert ok, info
    assert np.abs(R.grad.cpu().numpy() - gR).max() <= 1e-5 * np.abs(gR).max()


def test_degrade_adjoint_identity(small):
    import paper_1004_3980_gb300 as Z
    ctx = small["ctx"]
    g = np.random.default_rng(4)
    for s in (2, 3):
        x = torch.from_numpy(g.random((12 * s, 10 * s)).astype(np.float32)).cuda()
        yv = torch.from_numpy(g.random((12, 10)).astype(np.float32)).cuda()
        lhs = float((Z.degrade(ctx, x, s) * yv).double().sum())
        rhs = float((x * Z.degrade_adjoint(ctx, yv, s)).double().sum())
        assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
        ref = O.degrade(x.cpu().numpy().astype(np.float64), s, 0.8)
        assert np.abs(Z.degrade(ctx, x, s).cpu().numpy() - ref).max() < 1e-6


def test_full_size_sampled_coordinates():
    """2x zoom of a 256 x 256 LR image with a 65,536-pair dictionary
    (5x5 LR / 10x10 HR), K = 8 fixed neighbours (seeded), lambda = 0.1:
    GPU gradients against the oracle's analytic gradients at 100 HR-image
    and 100 dictionary coordinates."""
    wl = S.WORKLOADS["zoom2x_256_dict64k"]
    train = S.training_images(wl)
    pos = S.sample_positions(wl.pos_seed, len(train), wl.train_hr // 2, wl.train_hr // 2, wl.patch, wl.n_pairs)
    lr = S.test_image(wl)
    nq = (wl.lr_h - wl.patch + 1) * (wl.lr_w - wl.patch + 1)
    nbr = np.random.default_rng(17).integers(0, wl.n_pairs, size=(nq, wl.K))
    ctx, d, ix, od, mu, w32, K = _setup(train, pos, lr, 2, wl.patch, nbr)
    c = dict(s=2, P=wl.patch, lr=lr, nbr=nbr, ctx=ctx, d=d, ix=ix, od=od, mu=mu, w32=w32, K=K)
    E, gx, gR, _ = _gpu(c)
    Eo, gxo, gRo, _ = _oracle(c)
    assert abs(E - Eo) <= 1e-5 * abs(Eo)
    g = np.random.default_rng(23)
    ii, jj = g.integers(0, gx.shape[0], 100), g.integers(0, gx.shape[1], 100)
    ok, info = _close(gx[ii, jj], gxo[ii, jj])
    assert ok, info
    used = np.unique(nbr)
    rows, cols = g.choice(used, 100), g.integers(0, gR.shape[1], 100)
    ok, info = _close(gR[rows, cols], gRo[rows, cols])
    assert ok, info
    unused = np.setdiff1d(np.arange(wl.n_pairs), used)
    assert (gR[unused] == 0).all()
