"""Pins of the oracle's hashing and candidate collection (Sec. 3.2; Sec. 4.1,
Eq. 10; Sec. 4.2)."""
import math

import numpy as np
import pytest

import synth_inputs as S
from oracle import zoom_oracle as O


def test_mix64_matches_published_splitmix64_sequence():
    # SplitMix64 (Steele, Lea, Flood 2014; Vigna's reference splitmix64.c)
    # seeded with 1234567 yields this sequence.  The generator is
    # state += 0x9E3779B97F4A7C15; output = variant-13 mix of the state.
    expected = [6457827717110365317, 3203168211198807973, 9817491932198370423,
                4593380528125082431, 16408922859458223821]
    s, got = 1234567, []
    for _ in range(5):
        s = (s + 0x9E3779B97F4A7C15) & ((1 << 64) - 1)
        got.append(int(O.mix64(np.uint64(s))))
    assert got == expected


def test_unit_projection_reduces_to_floor(rng):
    # alpha = e_i, beta = 0  =>  h = floor(v_i / w)
    d, w = 9, 0.37
    v = rng.normal(size=(50, d))
    alpha = np.eye(d, dtype=np.float32)
    beta = np.zeros(d, np.float32)
    h, _ = O.hash_values(v, alpha, beta, w)
    for n in range(50):
        for i in range(d):
            assert h[n, i] == math.floor(v[n, i] / w)


def test_offset_shifts_bins(rng):
    v = rng.normal(size=(40, 4))
    alpha = rng.normal(size=(3, 4)).astype(np.float32)
    w = 1.5
    h0, _ = O.hash_values(v, alpha, np.zeros(3, np.float32), w)
    h1, _ = O.hash_values(v, alpha, np.full(3, w, np.float32), w)
    assert np.array_equal(h1, h0 + 1)


def test_margin_is_distance_to_integer():
    v = np.array([[0.999999, 0.0], [0.5, 0.0]])
    alpha = np.array([[1.0, 0.0]], np.float32)
    h, m = O.hash_values(v, alpha, np.zeros(1, np.float32), 1.0)
    assert h[:, 0].tolist() == [0, 0]
    assert abs(m[0] - 1e-6) < 1e-12 and abs(m[1] - 0.5) < 1e-12


@pytest.mark.parametrize("ratio", [0.5, 1.0, 2.0, 4.0])
def test_collision_rate_follows_pstable_law(ratio):
    # Datar et al.: a Gaussian projection hash of width w makes two points at
    # distance c collide with probability p(c).  Empirical frequency over many
    # independent projections must agree within 5 binomial standard errors.
    d, w = 6, 1.0
    c = w / ratio
    g = np.random.default_rng(int(ratio * 100))
    n = 40000
    alpha = g.normal(size=(n, d)).astype(np.float32)
    beta = (g.random(n) * w).astype(np.float32)
    u = g.normal(size=d)
    u /= np.linalg.norm(u)
    a = g.normal(size=d)
    pts = np.stack([a, a + c * u])
    h, _ = O.hash_values(pts, alpha, beta, w)
    freq = np.mean(h[0] == h[1])
    p = O.gaussian_collision_probability(c, w)
    assert abs(freq - p) < 5 * math.sqrt(p * (1 - p) / n) + 1e-3


@pytest.mark.parametrize("ratio", [0.5, 1.0, 2.0, 4.0])
def test_cauchy_collision_rate_follows_1stable_law(ratio):
    # Eq. 11 draws alpha_i = a / b (a, b ~ N(0, 1), |b| >= eps): Cauchy
    # projections, under which two points at l1 distance c collide with the
    # 1-stable probability p(c) (Datar et al.).  The |b| >= eps rejection
    # only removes projections beyond 1/eps, immaterial at this sample size.
    import synth_inputs as S
    d, w = 6, 1.0
    c = w / ratio
    n = 40000
    alpha, beta = S.lsh_draws_cauchy(int(ratio * 100) + 7, n, 1, d, w)
    g = np.random.default_rng(int(ratio * 100) + 1)
    u = g.normal(size=d)
    u /= np.abs(u).sum()                      # unit l1 norm
    a = g.normal(size=d)
    pts = np.stack([a, a + c * u])
    h, _ = O.hash_values(pts, alpha, beta, w)
    freq = np.mean(h[0] == h[1])
    p = O.cauchy_collision_probability(c, w)
    assert abs(freq - p) < 5 * math.sqrt(p * (1 - p) / n) + 1e-3
    # and it differs from the Gaussian law at the same l2 distance
    assert abs(O.gaussian_collision_probability(np.linalg.norm(c * u), w) - p) > 0.01


def test_fold_keys_equal_iff_tuples_equal(rng):
    L, k = 3, 4
    base = rng.integers(-3, 3, size=(30, L * k))
    h = np.concatenate([base, base[:10]])          # exact repeats
    keys = O.fold_keys(h, L, k)
    for l in range(L):
        tup = [tuple(r) for r in h[:, l * k:(l + 1) * k]]
        for a in range(len(h)):
            for b in range(len(h)):
                assert (keys[a, l] == keys[b, l]) == (tup[a] == tup[b])
    # the same tuple in different tables gives different keys
    same = np.tile(base[:1, :k], (1, L))
    kk = O.fold_keys(same, L, k)
    assert len(set(kk[0].tolist())) == L


def _tiny_index(rng, N=300, d=9, L=4, k=3, w=0.6):
    feat = rng.normal(scale=0.3, size=(N, d))
    feat -= feat.mean(axis=1, keepdims=True)
    dct = O.Dictionary(2, 3, feat.astype(np.float32), feat, np.zeros(N), np.zeros((N, 36)))
    alpha = rng.normal(size=(L * k, d)).astype(np.float32)
    beta = (rng.random(L * k) * w).astype(np.float32)
    return dct, O.build_index(dct, alpha, beta, w, L, k)


def test_buckets_group_identical_tuples(rng):
    dct, idx = _tiny_index(rng)
    h, _ = O.hash_values(dct.feat, idx.alpha, idx.beta, idx.w)
    for l in range(idx.L):
        tup = [tuple(r) for r in h[:, l * idx.k:(l + 1) * idx.k]]
        for n in range(dct.n):
            members = idx.buckets[l][int(idx.keys[n, l])]
            brute = [m for m in range(dct.n) if tup[m] == tup[n]]
            assert members.tolist() == brute


def test_candidate_set_brute_force(rng):
    dct, idx = _tiny_index(rng)
    q = rng.normal(scale=0.3, size=(20, 9))
    hq, _ = O.hash_values(q, idx.alpha, idx.beta, idx.w)
    hd, _ = O.hash_values(dct.feat, idx.alpha, idx.beta, idx.w)
    qk = O.fold_keys(hq, idx.L, idx.k)
    for t in (1, 2):
        for n in range(20):
            hits = np.zeros(dct.n, int)
            for l in range(idx.L):
                sl = slice(l * idx.k, (l + 1) * idx.k)
                hits += np.all(hd[:, sl] == hq[n, sl], axis=1)
            brute = np.flatnonzero(hits >= t)
            assert O.candidate_set(idx, qk[n], min_hits=t).tolist() == brute.tolist()


def test_candidate_cap_takes_tables_in_order():
    # Two tables; bins {5, 1, 9} and {1, 7, 3}: a cap of 4 collects 1, 5, 9
    # from table 0 (ascending IDs) and then 3 from table 1.
    idx = O.LshIndex(2, 1, 1.0, None, None, None, None,
                     [{11: np.array([1, 5, 9])}, {22: np.array([1, 3, 7])}])
    qk = np.array([11, 22], np.uint64)
    assert O.candidate_set(idx, qk, max_candidates=4).tolist() == [1, 3, 5, 9]
    assert O.candidate_set(idx, qk, max_candidates=2).tolist() == [1, 5]
    assert O.candidate_set(idx, qk).tolist() == [1, 3, 5, 7, 9]


def test_membership_certainty_of_boundary_entries():
    # L = 2 tables of k = 3 values; the entry matches the query's bin in
    # table 0 only where a near-boundary value flips
    L, k = 2, 3
    hq = np.array([1, 2, 3, 7, 7, 7])
    far = np.ones(6)
    # equal in table 0, no near values: a certain member
    assert O.membership_is_certain(hq, np.array([1, 2, 3, 0, 0, 0]), far, L, k)
    # differs everywhere by a clear value: certainly not a member
    assert O.membership_is_certain(hq, np.array([1, 2, 4, 0, 7, 7]), far, L, k)
    # differs in table 0 only at a near-boundary value: may flip in
    m = far.copy()
    m[2] = 1e-7
    assert not O.membership_is_certain(hq, np.array([1, 2, 4, 0, 7, 7]), m, L, k)
    # equal in table 0 with a near value, but a certain member via table 1
    m = far.copy()
    m[0] = 1e-7
    assert O.membership_is_certain(hq, np.array([1, 2, 3, 7, 7, 7]), m, L, k)
    # equal in table 0 only, with a near value: may flip out
    assert not O.membership_is_certain(hq, np.array([1, 2, 3, 7, 7, 6]), m, L, k)


def test_hash_margins_agree_with_hash_values(rng):
    v = rng.normal(size=(50, 9))
    a, b = S.lsh_draws(5, 3, 4, 9, 4.0)
    h, margin = O.hash_values(v, a, b, 4.0)
    mm = O.hash_margins(v, a, b, 4.0)
    np.testing.assert_array_equal(mm.min(axis=1), margin)
