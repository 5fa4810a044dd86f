"""The paper's own hash: Cauchy projections (Eq. 11; the random draws are
inputs, so the library path is the same).  Bucket keys and neighbours of the
GPU path against the oracle with Cauchy draws.  The heavy-tailed projections
make FP32 dot products less exact than with Gaussian draws, so a projection
counts as boundary-affected when it lies within its FP32 rounding bound of a
bin edge."""
import numpy as np
import pytest

import synth_inputs as S
from oracle import zoom_oracle as O
from tests import gpu_cases as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _near_edge(v, alpha, beta, w):
    """[n] True where some projection (alpha . v + beta) / w lies within the
    FP32 rounding bound of the dot product (d + 2 ulps of sum |alpha_i v_i|)
    of an integer."""
    a = alpha.astype(np.float64)
    t = (v @ a.T + beta.astype(np.float64)) / w
    err = (np.abs(v) @ np.abs(a).T + np.abs(beta)) * (v.shape[1] + 2) * 2.0 ** -24 / w
    return (np.abs(t - np.round(t)) <= err + 1e-6).any(axis=1)


def test_cauchy_keys_and_neighbours(tmp_path):
    from paper_1004_3980_gb300 import build
    build.build()
    import paper_1004_3980_gb300 as Z
    case = G.small_case()
    wl = case.wl
    ctx, d, _ = G.gpu_build(case)
    alpha, beta = S.lsh_draws_cauchy(41, wl.L, wl.k, wl.patch ** 2, wl.w)
    ix = Z.Index(d, wl.L, wl.k, wl.w, alpha, beta)
    oindex = O.build_index(case.odict, alpha, beta, wl.w, wl.L, wl.k)
    # dictionary keys
    keys, _ = ix.export_keys()
    dict_edge = _near_edge(case.odict.feat, alpha, beta, wl.w)
    assert dict_edge.mean() < 0.05
    assert np.array_equal(keys[~dict_edge], oindex.keys[~dict_edge])
    # query keys and neighbours (exact search over the Cauchy candidate sets)
    lr = np.ascontiguousarray(case.lr[:32, :36])
    r = Z.query(ix, torch.from_numpy(lr).cuda(), G.params(wl, search=2))
    oq = O.query(lr, case.odict, oindex, wl.K + 1, wl.reg_rel)
    q_edge = _near_edge(oq.feat, alpha, beta, wl.w)
    qkeys = r["keys"].cpu().numpy().view(np.uint64)
    assert np.array_equal(qkeys[~q_edge], oq.keys[~q_edge])
    # Cauchy bins are finer than the Gaussian ones at this width
    assert oq.n_cand.mean() < len(case.odict.feat)
    ex = G.tie_or_boundary(oq, wl.K, np.where(dict_edge, 0.0, 1.0)) | q_edge
    nbr = r["nbr"].cpu().numpy()
    bad = (nbr != oq.nbr[:, :wl.K]).any(axis=1) & ~ex
    assert not bad.any(), (np.flatnonzero(bad)[:10], ex.mean())
    assert ex.mean() < 0.1
    # the SIMT scan agrees with the tensor-core path bit for bit
    r1 = Z.query(ix, torch.from_numpy(lr).cuda(), G.params(wl, search=1))
    assert torch.equal(r1["nbr"], r["nbr"]) and torch.equal(r1["dist"], r["dist"])
