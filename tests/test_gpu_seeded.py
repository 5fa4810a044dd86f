"""Dictionary and index built from seeds instead of caller arrays: with
positions NULL the dictionary equals the one built from the library's drawn
positions (zoom_sample_positions, equal to the oracle's generator), and with
alpha and beta NULL the index's projections (zoom_export_params) are the
library's draws (zoom_lsh_draws) and its keys and search equal those of the
index built from those arrays."""
import numpy as np
import pytest

import synth_inputs as S
from oracle import zoom_oracle as O
from tests import gpu_cases as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_seeded_dictionary_and_index():
    from paper_1004_3980_gb300 import build
    build.build()
    import paper_1004_3980_gb300 as Z
    wl = S.WORKLOADS["zoom2x_64_dict20k"]
    train = S.training_images(wl, 8)
    lrs = wl.train_hr // wl.scale
    ctx = Z.Context(0)
    imgs = [torch.from_numpy(x).cuda() for x in train]
    pos = Z.sample_positions(17, [(lrs, lrs)] * len(train), wl.patch, 12000)
    assert np.array_equal(pos, O.sample_positions_seeded(17, [(lrs, lrs)] * len(train), wl.patch, 12000))
    d_seed = Z.Dictionary(ctx, imgs, None, wl.scale, wl.patch, n_pairs=12000, seed=17)
    d_arr = Z.Dictionary(ctx, imgs, pos, wl.scale, wl.patch)
    for a, b in zip(d_seed.export(), d_arr.export()):
        assert np.array_equal(a, b)
    for dist in (0, 1):
        ix_seed = Z.Index(d_seed, wl.L, wl.k, wl.w, proj_dist=dist, seed=29)
        a, b = Z.lsh_draws(wl.L, wl.k, wl.patch ** 2, wl.w, 29, dist)
        ea, eb = ix_seed.params()
        assert np.array_equal(ea, a) and np.array_equal(eb, b)
        ix_arr = Z.Index(d_arr, wl.L, wl.k, wl.w, a, b)
        assert np.array_equal(ix_seed.export_keys()[0], ix_arr.export_keys()[0])
        lr = torch.from_numpy(S.test_image(wl)).cuda()
        r1 = Z.query(ix_seed, lr, G.params(wl))
        r2 = Z.query(ix_arr, lr, G.params(wl))
        assert torch.equal(r1["nbr"], r2["nbr"]) and torch.equal(r1["dist"], r2["dist"])
        ix_seed.close()
        ix_arr.close()
    ctx.sync_status()
