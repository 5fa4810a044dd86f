"""Pins of the oracle's seeded draws: Philox4x32-10 against the published
known-answer vectors of its authors (Salmon et al., SC 2011, the Random123
test vectors), and the laws of the projection and position draws."""
import math

import numpy as np
import pytest

from oracle import zoom_oracle as O

# Published known-answer vectors of Philox4x32-10: (counter, key) -> output
KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,out", KAT)
def test_philox_known_answers(ctr, key, out):
    got = O.philox4x32_10(np.array([ctr], np.uint32), key[0] | (key[1] << 32))
    assert tuple(int(x) for x in got[0]) == out


def test_gaussian_projections_follow_their_law():
    a, b = O.projection_draws(11, 16, 18, 25, 4.0, dist=0)
    assert a.shape == (288, 25) and b.shape == (288,) and a.dtype == np.float32
    x = a.ravel().astype(np.float64)
    n = x.size
    assert abs(x.mean()) < 4 / math.sqrt(n)
    assert abs(x.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    # the fraction within one standard deviation: 0.6827 (binomial 5 sigma)
    f = np.mean(np.abs(x) < 1.0)
    assert abs(f - 0.682689) < 5 * math.sqrt(0.6827 * 0.3173 / n)
    assert (b >= 0).all() and (b < 4.0).all()
    assert abs(b.mean() - 2.0) < 5 * 4.0 / math.sqrt(12 * b.size)
    # another seed: other draws; the same seed: the same draws
    assert not np.array_equal(O.projection_draws(12, 16, 18, 25, 4.0)[0], a)
    assert np.array_equal(O.projection_draws(11, 16, 18, 25, 4.0)[0], a)


def test_cauchy_projections_follow_eq_11():
    a, _ = O.projection_draws(3, 8, 16, 25, 4.0, dist=1)
    x = a.ravel().astype(np.float64)
    n = x.size
    # a / b of independent standard normals is standard Cauchy: quartiles
    # at -1 and +1, median 0 (binomial 5 sigma on the counts)
    for q, v in ((0.25, -1.0), (0.5, 0.0), (0.75, 1.0)):
        assert abs(np.mean(x <= v) - q) < 5 * math.sqrt(q * (1 - q) / n)


def test_rejection_keeps_b_away_from_zero():
    # a tiny seed sweep with a large eps: every b used has |b| >= eps, so
    # |alpha| <= |a| / eps
    a0, _ = O.projection_draws(5, 2, 4, 9, 1.0, dist=0)
    a1, _ = O.projection_draws(5, 2, 4, 9, 1.0, dist=1, eps=0.8)
    assert (np.abs(a1) <= np.abs(a0) / 0.8 + 1e-6).all()


def test_seeded_positions_are_a_uniform_sorted_subset():
    sizes = [(20, 30), (15, 40), (25, 25)]
    P = 5
    counts = [(h - P + 1) * (w - P + 1) for h, w in sizes]
    pos = O.sample_positions_seeded(7, sizes, P, 600)
    assert pos.shape == (600, 3)
    # valid origins, strictly ascending in (image, row, col): unique IDs
    for m, i, j in pos:
        assert 0 <= i <= sizes[m][0] - P and 0 <= j <= sizes[m][1] - P
    key = pos[:, 0].astype(np.int64) * 10 ** 6 + pos[:, 1] * 1000 + pos[:, 2]
    assert (np.diff(key) > 0).all()
    # uniform: each image's share within 5 sigma of the hypergeometric mean
    tot = sum(counts)
    for m, c in enumerate(counts):
        k = np.sum(pos[:, 0] == m)
        mean = 600 * c / tot
        var = 600 * (c / tot) * (1 - c / tot) * (tot - 600) / (tot - 1)
        assert abs(k - mean) < 5 * math.sqrt(var)
    # all origins: the whole grid in order
    allp = O.sample_positions_seeded(7, sizes, P, tot)
    assert len(allp) == tot and (np.diff(allp[:, 0] * 10 ** 6 + allp[:, 1] * 1000 + allp[:, 2]) > 0).all()
    with pytest.raises(ValueError):
        O.sample_positions_seeded(7, sizes, P, tot + 1)
