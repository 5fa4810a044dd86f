"""Dictionary and index files: a saved and reloaded dictionary holds the
same arrays bit for bit, a reloaded index the same keys and bins and
projections, and both give the same HR output; malformed files are refused
with the documented status."""
import os

import numpy as np
import pytest

from tests import gpu_cases as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def built():
    from paper_1004_3980_gb300 import build
    build.build()
    case = G.small_case()
    ctx, d, ix = G.gpu_build(case)
    return case, ctx, d, ix


def test_save_load_roundtrip(built, tmp_path):
    import paper_1004_3980_gb300 as Z
    case, ctx, d, ix = built
    pd, pi = str(tmp_path / "dict.zd"), str(tmp_path / "index.zi")
    d.save(pd)
    ix.save(pi)
    d2 = Z.Dictionary.load(ctx, pd)
    assert (d2.n, d2.patch, d2.scale, d2.blur_sigma) == (d.n, d.patch, d.scale, d.blur_sigma)
    for a, b in zip(d.export(), d2.export()):
        assert np.array_equal(a, b)
    ix2 = Z.Index.load(d2, pi)
    assert (ix2.L, ix2.k, ix2.w, ix2.min_table_hits) == (ix.L, ix.k, ix.w, ix.min_table_hits)
    k1, n1 = ix.export_keys()
    k2, n2 = ix2.export_keys()
    assert np.array_equal(k1, k2) and np.array_equal(n1, n2)
    a2, b2 = ix2.params()
    assert np.array_equal(a2, case.alpha) and np.array_equal(b2, case.beta)
    lr = torch.from_numpy(case.lr).cuda()
    p = G.params(case.wl)
    assert torch.equal(Z.upscale(ix, lr, p), Z.upscale(ix2, lr, p))


def test_load_errors(built, tmp_path):
    import paper_1004_3980_gb300 as Z
    from paper_1004_3980_gb300 import capi
    case, ctx, d, ix = built
    with pytest.raises(capi.ZoomError) as e:
        Z.Dictionary.load(ctx, str(tmp_path / "missing.zd"))
    assert capi.STATUS_NAMES[e.value.status] == "ZOOM_ERR_IO"
    bad = tmp_path / "bad.zd"
    bad.write_bytes(b"NOTADICT" + bytes(64))
    with pytest.raises(capi.ZoomError) as e:
        Z.Dictionary.load(ctx, str(bad))
    assert capi.STATUS_NAMES[e.value.status] == "ZOOM_ERR_INVALID_ARG"
    pd = tmp_path / "dict.zd"
    d.save(str(pd))
    cut = tmp_path / "cut.zd"
    cut.write_bytes(pd.read_bytes()[: os.path.getsize(pd) // 2])
    with pytest.raises(capi.ZoomError) as e:
        Z.Dictionary.load(ctx, str(cut))
    assert capi.STATUS_NAMES[e.value.status] == "ZOOM_ERR_IO"
    # an index file of another dictionary
    pi = tmp_path / "index.zi"
    ix.save(str(pi))
    small = G.make_case("zoom2x_64_dict20k", n_train=2, n_pairs=500, with_oracle=False)
    _, d_small, _ = G.gpu_build(small, ctx)
    with pytest.raises(capi.ZoomError) as e:
        Z.Index.load(d_small, str(pi))
    assert capi.STATUS_NAMES[e.value.status] == "ZOOM_ERR_INVALID_ARG"
