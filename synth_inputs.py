"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the zoom method itself: it only draws
images, dictionary sample positions and the random numbers the method
consumes (LSH projection vectors and offsets), all from numpy PCG64 streams
with fixed seeds.  Both the CUDA path and the CPU oracle receive these
arrays as inputs.

Image recipe (stand-in for the paper's natural-image training set and test
images, which are not available here):
  * canvas at grey level 128;
  * plus 6 oriented sinusoids, period U[4, 32] px, angle U[0, pi),
    phase U[0, 2 pi), amplitude U[8, 24] grey levels;
  * plus 8 ellipses, each adding a constant level U[-48, 48] inside; centre
    uniform over the canvas, semi-axes U[n/16, n/4] with n = min(h, w),
    angle U[0, pi);
  * plus Gaussian noise sigma = 2 grey levels;
  * clip to [0, 255], round half-to-even to uint8, divide by 255 -> float32.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def make_image(seed: int, h: int, w: int) -> np.ndarray:
    """One synthetic grey image, float32 [h][w] on the [0, 1] scale."""
    rng = _rng(seed)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    img = np.full((h, w), 128.0)
    for _ in range(6):
        period = rng.uniform(4.0, 32.0)
        angle = rng.uniform(0.0, math.pi)
        phase = rng.uniform(0.0, 2.0 * math.pi)
        amp = rng.uniform(8.0, 24.0)
        u = xx * math.cos(angle) + yy * math.sin(angle)
        img += amp * np.sin(2.0 * math.pi * u / period + phase)
    n = min(h, w)
    for _ in range(8):
        level = rng.uniform(-48.0, 48.0)
        cy = rng.uniform(0.0, h)
        cx = rng.uniform(0.0, w)
        ay = rng.uniform(n / 16.0, n / 4.0)
        ax = rng.uniform(n / 16.0, n / 4.0)
        ang = rng.uniform(0.0, math.pi)
        dx = xx - cx
        dy = yy - cy
        u = dx * math.cos(ang) + dy * math.sin(ang)
        v = -dx * math.sin(ang) + dy * math.cos(ang)
        img[(u / ax) ** 2 + (v / ay) ** 2 <= 1.0] += level
    img += rng.normal(0.0, 2.0, size=(h, w))
    img = np.rint(np.clip(img, 0.0, 255.0)).astype(np.uint8)
    return (img.astype(np.float32) / np.float32(255.0)).astype(np.float32)


def sample_positions(seed: int, n_images: int, lr_h: int, lr_w: int, patch: int,
                     n_pairs: int) -> np.ndarray:
    """Dictionary sample positions: int32 [n_pairs][3] = (image, lr_row, lr_col).

    Drawn uniformly without replacement over every valid LR patch origin of
    every training image, then sorted by (image, row, col), so that the row
    index of a position is the unique integer ID of its patch pair.
    """
    ph, pw = lr_h - patch + 1, lr_w - patch + 1
    per = ph * pw
    total = n_images * per
    if n_pairs > total:
        raise ValueError(f"n_pairs={n_pairs} exceeds the {total} patch origins")
    flat = np.sort(_rng(seed).choice(total, size=n_pairs, replace=False))
    img = flat // per
    rem = flat % per
    return np.stack([img, rem // pw, rem % pw], axis=1).astype(np.int32)


def lsh_draws(seed: int, L: int, k: int, d: int, w: float):
    """Random draws of the p-stable hash: alpha float32 [L*k][d] ~ N(0, 1)
    and beta float32 [L*k] ~ U[0, w)."""
    rng = _rng(seed)
    alpha = rng.standard_normal((L * k, d)).astype(np.float32)
    beta = (rng.uniform(0.0, 1.0, size=L * k) * w).astype(np.float32)
    beta = np.minimum(beta, np.nextafter(np.float32(w), np.float32(0.0)))
    return alpha, beta


def lsh_draws_cauchy(seed: int, L: int, k: int, d: int, w: float, eps: float = 1e-3):
    """Cauchy draws alpha = a / b, a, b ~ N(0, 1) with |b| >= eps (rejection),
    and beta ~ U[0, w); float32."""
    rng = _rng(seed)
    a = rng.standard_normal((L * k, d))
    b = rng.standard_normal((L * k, d))
    bad = np.abs(b) < eps
    while bad.any():
        b[bad] = rng.standard_normal(int(bad.sum()))
        bad = np.abs(b) < eps
    alpha = (a / b).astype(np.float32)
    beta = (rng.uniform(0.0, 1.0, size=L * k) * w).astype(np.float32)
    beta = np.minimum(beta, np.nextafter(np.float32(w), np.float32(0.0)))
    return alpha, beta


@dataclasses.dataclass(frozen=True)
class Workload:
    """One named workload: test image, training set and method parameters."""
    name: str
    lr_h: int
    lr_w: int
    scale: int
    patch: int
    n_train: int
    train_hr: int          # training HR images are train_hr x train_hr
    n_pairs: int
    L: int
    k: int
    K: int
    bp_iters: int
    w: float = 4.0
    reg_rel: float = 1e-3
    sigma_spatial: float = 1.5
    sigma_range: float = 0.1
    bp_radius: int = 3
    blur_sigma: float = 0.8
    test_seed: int = 1
    train_seed0: int = 1000
    pos_seed: int = 7
    proj_seed: int = 11


# The workloads' sizes and parameters (LR size, zoom, dictionary size, L, k, K,
# back-projection iterations).  Training-image counts are chosen so the
# dictionary is a sample of a few million patch origins.
WORKLOADS = {
    "zoom2x_64_dict20k": Workload("zoom2x_64_dict20k", 64, 64, 2, 3, 16, 256, 20_000,
                                  L=8, k=12, K=5, bp_iters=3),
    "zoom2x_512_dict1m": Workload("zoom2x_512_dict1m", 512, 512, 2, 5, 64, 512, 1_000_000,
                                  L=16, k=16, K=8, bp_iters=5),
    "zoom3x_1920x1080_dict4m": Workload("zoom3x_1920x1080_dict4m", 1080, 1920, 3, 5, 128, 768,
                                        4_000_000, L=16, k=18, K=8, bp_iters=5),
    "zoom2x_256_dict64k": Workload("zoom2x_256_dict64k", 256, 256, 2, 5, 16, 512, 65_536,
                                   L=16, k=16, K=8, bp_iters=0),
}


def training_images(wl: Workload, count: int | None = None):
    n = wl.n_train if count is None else count
    return [make_image(wl.train_seed0 + i, wl.train_hr, wl.train_hr) for i in range(n)]


def test_image(wl: Workload) -> np.ndarray:
    return make_image(wl.test_seed, wl.lr_h, wl.lr_w)


def batch_shapes(n_images: int = 64, seed0: int = 100, perm_seed: int = 99):
    """Batched workload: per-image (seed, h, w, scale); h ~ U{96..768},
    w ~ U{128..1024}; a seeded permutation gives half the images scale 3."""
    out = []
    for i in range(n_images):
        r = _rng(seed0 + i)
        h = int(r.integers(96, 769))
        w = int(r.integers(128, 1025))
        out.append([seed0 + i, h, w, 2])
    perm = _rng(perm_seed).permutation(n_images)
    for i in perm[: n_images // 2]:
        out[int(i)][3] = 3
    return [tuple(x) for x in out]
