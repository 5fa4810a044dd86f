"""The library's seeded draws (zoom_lsh_draws, zoom_sample_positions: host
code behind the C ABI, no GPU needed) against the oracle's generator, which
is written separately from the same published definition of
Philox4x32-10: the same projections, offsets and positions."""
import numpy as np
import pytest

from oracle import zoom_oracle as O


@pytest.fixture(scope="module")
def Z():
    from paper_1004_3980_gb300 import build
    build.build()
    import paper_1004_3980_gb300 as Zm
    return Zm


def _ulps(a, b):
    ai = a.view(np.int32).astype(np.int64)
    bi = b.view(np.int32).astype(np.int64)
    return np.abs(ai - bi)


@pytest.mark.parametrize("L,k,D,w,dist,seed", [(16, 18, 25, 4.0, 0, 11), (16, 16, 50, 8.0, 0, 11),
                                               (8, 12, 9, 4.0, 1, 3), (4, 6, 25, 1.5, 1, 2 ** 40 + 5)])
def test_library_draws_equal_the_oracle(Z, L, k, D, w, dist, seed):
    a, b = Z.lsh_draws(L, k, D, w, seed, dist)
    oa, ob = O.projection_draws(seed, L, k, D, w, dist)
    # both sides round one FP64 Box-Muller value to float32; their libm
    # log and cos may differ in the last FP64 bit, which can move a float32
    # rounding only when the value sits on a rounding boundary
    u = _ulps(a.ravel(), oa.ravel())
    assert u.max() <= 1 and (u > 0).mean() < 1e-3
    assert np.array_equal(b, ob)
    assert (b < w).all() and (b >= 0).all()


def test_library_positions_equal_the_oracle(Z):
    sizes = [(128, 128)] * 6 + [(96, 160)] * 3
    for seed, n in ((7, 5000), (123, 40000), (1, 1)):
        got = Z.sample_positions(seed, sizes, 5, n)
        ref = O.sample_positions_seeded(seed, sizes, 5, n)
        assert np.array_equal(got, ref)


def test_library_draws_reject_bad_arguments(Z):
    from paper_1004_3980_gb300.capi import ZoomError
    with pytest.raises(ZoomError, match="INVALID_ARG"):
        Z.lsh_draws(16, 16, 25, 4.0, 1, proj_dist=2)
    with pytest.raises(ZoomError, match="INVALID_ARG"):
        Z.sample_positions(1, [(4, 4)], 5, 1)
    with pytest.raises(ZoomError, match="INVALID_ARG"):
        Z.sample_positions(1, [(8, 8)], 5, 17)
