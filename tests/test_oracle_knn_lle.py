"""Pins of the oracle's nearest-neighbour selection (Sec. 3.1 step 1a,
Sec. 4.2) and LLE weights (Eq. 12-13)."""
import numpy as np
import pytest
from scipy.spatial.distance import cdist

from oracle import zoom_oracle as O


def test_top_k_is_sorted_brute_force_with_id_ties(rng):
    feat = rng.normal(size=(200, 9))
    feat[50] = feat[10]          # exact duplicate rows: tie broken by id
    feat[120] = feat[10]
    for _ in range(20):
        q = rng.normal(size=9)
        cand = np.sort(rng.choice(200, size=80, replace=False))
        cand = np.union1d(cand, [10, 50, 120])
        ids, dist, npad = O.top_k(q, cand, feat, 7)
        brute = sorted((float(((feat[c] - q) ** 2).sum()), int(c)) for c in cand)[:7]
        assert ids.tolist() == [c for _, c in brute]
        np.testing.assert_allclose(dist, [d for d, _ in brute], rtol=1e-14)
        assert npad == 0
    q = feat[10]
    ids, dist, _ = O.top_k(q, np.array([120, 50, 10, 3]), feat, 3)
    assert ids.tolist() == [10, 50, 120] and dist.tolist() == [0.0, 0.0, 0.0]


def test_top_k_full_dictionary_equals_cdist(rng):
    feat = rng.normal(size=(500, 25))
    Q = rng.normal(size=(30, 25))
    D = cdist(Q, feat, "sqeuclidean")
    for n in range(30):
        ids, dist, _ = O.top_k(Q[n], np.arange(500), feat, 8)
        assert ids.tolist() == np.argsort(D[n], kind="stable")[:8].tolist()
        np.testing.assert_allclose(dist, np.sort(D[n])[:8], rtol=1e-12)


def test_top_k_pads_with_nearest_outside(rng):
    feat = rng.normal(size=(60, 4))
    q = rng.normal(size=4)
    cand = np.array([3, 17])
    ids, dist, npad = O.top_k(q, cand, feat, 5)
    assert npad == 3
    inside = sorted(cand, key=lambda c: (((feat[c] - q) ** 2).sum(), c))
    rest = [c for c in range(60) if c not in cand]
    outside = sorted(rest, key=lambda c: (((feat[c] - q) ** 2).sum(), c))[:3]
    assert ids.tolist() == inside + outside


def _problem(rng, K=8, d=25):
    q = rng.normal(size=d)
    nb = q + rng.normal(scale=0.2, size=(K, d))
    return q, nb


def _kkt_weights(q, nb, reg):
    # Textbook equality-constrained quadratic program: minimise w^T C w
    # subject to 1^T w = 1 via the KKT system [[2C, 1], [1^T, 0]].
    Z = q[None] - nb
    G = Z @ Z.T
    K = len(nb)
    C = G + reg * np.trace(G) * np.eye(K)
    A = np.zeros((K + 1, K + 1))
    A[:K, :K] = 2 * C
    A[:K, K] = 1
    A[K, :K] = 1
    b = np.zeros(K + 1)
    b[K] = 1
    return np.linalg.solve(A, b)[:K], C


@pytest.mark.parametrize("K", [2, 5, 8, 16])
def test_lle_matches_kkt_solution_and_sums_to_one(rng, K):
    q, nb = _problem(rng, K)
    w, cond = O.lle_weights(q, nb, 1e-3, 1.0)
    wk, C = _kkt_weights(q, nb, 1e-3)
    np.testing.assert_allclose(w, wk, atol=1e-10)
    assert abs(w.sum() - 1) < 1e-12
    assert np.linalg.cond(C) <= cond * (1 + 1e-9)
    assert cond <= 1001.0 + 1e-9


def test_lle_is_minimal_on_constraint_set(rng):
    q, nb = _problem(rng, 8)
    w, _ = O.lle_weights(q, nb, 1e-3, 1.0)
    _, C = _kkt_weights(q, nb, 1e-3)
    f0 = w @ C @ w
    for _ in range(50):
        dlt = rng.normal(size=8)
        dlt -= dlt.mean()
        assert (w + 1e-3 * dlt) @ C @ (w + 1e-3 * dlt) >= f0


def test_lle_k2_closed_form(rng):
    q, nb = _problem(rng, 2)
    w, _ = O.lle_weights(q, nb, 1e-3, 1.0)
    Z = q[None] - nb
    G = Z @ Z.T
    C = G + 1e-3 * np.trace(G) * np.eye(2)
    w1 = (C[1, 1] - C[0, 1]) / (C[0, 0] + C[1, 1] - 2 * C[0, 1])
    np.testing.assert_allclose(w, [w1, 1 - w1], atol=1e-12)


def test_lle_k1_and_exact_match(rng):
    q, nb = _problem(rng, 1)
    assert O.lle_weights(q, nb, 1e-3, 0.5)[0].tolist() == [1.0]
    q, nb = _problem(rng, 6)
    nb[0] = q
    w, _ = O.lle_weights(q, nb, 1e-3, 0.0)
    assert w.tolist() == [1, 0, 0, 0, 0, 0]


def test_lle_permutation_invariant(rng):
    q, nb = _problem(rng, 8)
    w, _ = O.lle_weights(q, nb, 1e-3, 1.0)
    p = rng.permutation(8)
    wp, _ = O.lle_weights(q, nb[p], 1e-3, 1.0)
    np.testing.assert_allclose(wp, w[p], atol=1e-12)


def test_neighbour_exclusions_flag_ties_boundaries_and_uncertain_members():
    # tiny dictionary: the exclusion rule agrees with a brute-force reading
    # of its three conditions
    import synth_inputs as S
    g = np.random.default_rng(4)
    N, D, L, k, K = 400, 9, 3, 4, 3
    feat = g.normal(scale=0.4, size=(N, D))
    feat[7] = feat[3]                                     # an exact duplicate: a distance tie
    d = O.Dictionary(2, 3, None, feat, None, None)
    a, b = S.lsh_draws(6, L, k, D, 1.0)
    ix = O.build_index(d, a, b, 1.0, L, k)
    q = np.vstack([feat[3] + 1e-3, g.normal(scale=0.4, size=(40, D))])
    hq, qm = O.hash_values(q, a, b, 1.0)
    nb = np.zeros((len(q), K + 1), np.int64)
    dist = np.zeros((len(q), K + 1))
    for i in range(len(q)):
        keys = O.fold_keys(hq[i:i + 1], L, k)[0]
        nb[i], dist[i], _ = O.top_k(q[i], O.candidate_set(ix, keys), feat, K + 1)
    ex = O.neighbour_exclusions(q, qm, dist, d, ix)
    assert ex[0]                                          # the tie
    # brute force of condition (b) with a loose boundary (1e-2): more entries
    # become uncertain, never fewer queries
    ex_loose = O.neighbour_exclusions(q, qm, dist, d, ix, bnd=1e-2)
    assert (ex_loose >= ex).all() and ex_loose.sum() > ex.sum()
    for i in np.flatnonzero(ex_loose & ~ex):
        dd = ((feat - q[i]) ** 2).sum(axis=1)
        close = np.flatnonzero(dd <= dist[i, -1])
        he, _ = O.hash_values(feat[close], a, b, 1.0)
        me = O.hash_margins(feat[close], a, b, 1.0)
        assert qm[i] < 1e-2 or any(not O.membership_is_certain(hq[i], he[j], me[j], L, k, 1e-2)
                                   for j in range(len(close)))
