"""Shared builders for the GPU parity tests: one seeded workload, built once
on the GPU (through the C ABI) and once in the oracle, from the same
synthetic inputs."""
from __future__ import annotations

import dataclasses
import functools
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import synth_inputs as S
from oracle import zoom_oracle as O


@dataclasses.dataclass
class Case:
    wl: S.Workload
    train: list
    positions: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray
    lr: np.ndarray
    odict: O.Dictionary | None = None
    oindex: O.LshIndex | None = None


def make_case(name: str, n_train: int | None = None, n_pairs: int | None = None,
              lr_shape=None, with_oracle: bool = True) -> Case:
    wl = S.WORKLOADS[name]
    if n_pairs is not None:
        wl = dataclasses.replace(wl, n_pairs=n_pairs)
    if lr_shape is not None:
        wl = dataclasses.replace(wl, lr_h=lr_shape[0], lr_w=lr_shape[1])
    train = S.training_images(wl, n_train)
    lrs = wl.train_hr // wl.scale
    pos = S.sample_positions(wl.pos_seed, len(train), lrs, lrs, wl.patch, wl.n_pairs)
    alpha, beta = S.lsh_draws(wl.proj_seed, wl.L, wl.k, wl.patch ** 2, wl.w)
    lr = S.test_image(wl)
    c = Case(wl, train, pos, alpha, beta, lr)
    if with_oracle:
        c.odict = O.build_dictionary(train, pos, wl.scale, wl.patch, wl.blur_sigma)
        c.oindex = O.build_index(c.odict, alpha, beta, wl.w, wl.L, wl.k)
    return c


@functools.lru_cache(maxsize=None)
def small_case():
    """The 2x zoom of a 64 x 64 LR image with a 20,000-pair dictionary of
    3x3 LR / 6x6 HR patches (L=8, k=12, K=5, 3 back-projection steps)."""
    return make_case("zoom2x_64_dict20k")


def gpu_build(case: Case, ctx=None, min_table_hits: int = 1):
    import torch

    import paper_1004_3980_gb300 as Z
    ctx = ctx or Z.Context(0)
    imgs = [torch.from_numpy(x).cuda() for x in case.train]
    d = Z.Dictionary(ctx, imgs, case.positions, case.wl.scale, case.wl.patch, case.wl.blur_sigma)
    ix = Z.Index(d, case.wl.L, case.wl.k, case.wl.w, case.alpha, case.beta, min_table_hits=min_table_hits)
    return ctx, d, ix


def params(wl: S.Workload, **kw):
    import paper_1004_3980_gb300 as Z
    p = Z.UpscaleParams(K=wl.K, reg_rel=wl.reg_rel, bp_iters=wl.bp_iters, sigma_spatial=wl.sigma_spatial,
                        sigma_range=wl.sigma_range, bp_radius=wl.bp_radius)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def tie_or_boundary(oq: O.QueryResult, K: int, dict_margin: np.ndarray, rel: float = 1e-6,
                    bnd: float = 1e-5) -> np.ndarray:
    """Queries excluded from the bit-exact neighbour check: the query's own
    projections, or those of any of its K+1 nearest oracle neighbours, lie
    within bnd (in units of w) of a bin boundary; or two of its K+1 nearest
    FP64 distances differ by less than rel (relative)."""
    n = len(oq.nbr)
    ex = oq.margin < bnd
    ex |= (dict_margin[oq.nbr] < bnd).any(axis=1)
    d = oq.dist
    gaps = np.diff(d, axis=1)
    scale = np.maximum(d[:, 1:], 1e-30)
    ex |= (gaps <= rel * scale).any(axis=1)
    assert ex.shape == (n,)
    return ex


def oracle_rows(lr, od, oix, K, reg_rel, rows):
    """O.query on the given query rows, split over the host threads."""
    parts = np.array_split(np.asarray(rows), max(1, min(len(rows), os.cpu_count() or 1)))
    with ThreadPoolExecutor(max_workers=len(parts)) as ex:
        res = list(ex.map(lambda r: O.query(lr, od, oix, K, reg_rel, rows=r), parts))
    cat = lambda f: np.concatenate([getattr(q, f) for q in res])
    return O.QueryResult(*(cat(f.name) for f in dataclasses.fields(O.QueryResult)))
