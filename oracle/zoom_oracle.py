"""Plain, slow FP64 oracle of "Hashing Image Patches for Zooming" (Das Gupta).

TEST INFRASTRUCTURE.  Only tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may use this module; the product path never does.

Every function follows one passage of the paper (cited in its docstring) in
the paper's order and notation.  Numbers are FP64 numpy arrays unless stated.
Library primitives used as single steps: matrix products, sorting,
``np.linalg.cholesky``.  Readings of passages the paper leaves open are stated
where they are applied.

Pins: every function here is pinned by at least one CPU test in ``tests/``
against a closed form, an invariant, a brute-force computation or a library
routine (see the test files named ``test_oracle_*.py``).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GOLDEN64 = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1

# ---------------------------------------------------------------------------
# Degradation (Sec. 2.1 "Notations"; smoothing kernel g of Eq. 6)
# ---------------------------------------------------------------------------


def gaussian_taps(sigma: float, radius: int = 1) -> np.ndarray:
    """Normalised 1-D Gaussian taps exp(-t^2 / (2 sigma^2)), |t| <= radius.

    Sec. 2.1: the LR image is the HR image blurred by a Gaussian kernel
    K(sigma^2) and then down-sampled.  The kernel is 3 taps wide (radius 1).
    """
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    g = np.exp(-t * t / (2.0 * sigma * sigma))
    return g / g.sum()


def blur(x: np.ndarray, taps: np.ndarray) -> np.ndarray:
    """Separable blur with clamp-to-edge borders (reading: the paper states no
    border rule; pixels outside the image take the value of the nearest edge
    pixel)."""
    r = len(taps) // 2
    h, w = x.shape
    xp = np.pad(np.asarray(x, dtype=np.float64), r, mode="edge")
    rows = sum(taps[u] * xp[u:u + h, r:r + w] for u in range(len(taps)))
    rp = np.pad(rows, ((0, 0), (r, r)), mode="edge")
    return sum(taps[u] * rp[:, u:u + w] for u in range(len(taps)))


def box_decimate(x: np.ndarray, s: int) -> np.ndarray:
    """Down-sampling by s: the mean of each s x s block (reading: the paper
    names only the factor; sizes not divisible by s are cropped)."""
    h, w = x.shape[0] // s, x.shape[1] // s
    return x[:h * s, :w * s].reshape(h, s, w, s).mean(axis=(1, 3))


def degrade(x: np.ndarray, s: int, sigma: float) -> np.ndarray:
    """y = D_s(B x): Gaussian blur, then s x s box down-sampling (Sec. 2.1)."""
    return box_decimate(blur(x, gaussian_taps(sigma)), s)


def blur_adjoint(z: np.ndarray, taps: np.ndarray) -> np.ndarray:
    """Adjoint of ``blur``: each output value sends taps back to the (clamped)
    input pixels it read."""
    r = len(taps) // 2
    h, w = z.shape
    t1 = np.zeros((h, w))
    cols = np.arange(w)
    for u in range(len(taps)):
        src = np.clip(cols + u - r, 0, w - 1)
        np.add.at(t1, (slice(None), src), taps[u] * z)
    out = np.zeros((h, w))
    rows = np.arange(h)
    for u in range(len(taps)):
        src = np.clip(rows + u - r, 0, h - 1)
        np.add.at(out, src, taps[u] * t1)
    return out


def degrade_adjoint(y: np.ndarray, s: int, sigma: float, hr_shape) -> np.ndarray:
    """B^T D^T y: spread each LR value / s^2 over its s x s block (zero in a
    cropped margin), then the blur adjoint."""
    z = np.zeros(hr_shape)
    h, w = y.shape
    z[:h * s, :w * s] = np.kron(y, np.ones((s, s))) / (s * s)
    return blur_adjoint(z, gaussian_taps(sigma))


# ---------------------------------------------------------------------------
# Patches and the dictionary (Sec. 2.1; Sec. 5.1 "Training Data Generation")
# ---------------------------------------------------------------------------


def patch_origins(h: int, w: int, P: int):
    """All P x P patch origins (i, j) at stride 1, numbered in row order
    (Sec. 2.1: patches are numbered row by row)."""
    ii, jj = np.meshgrid(np.arange(h - P + 1), np.arange(w - P + 1), indexing="ij")
    return ii.ravel(), jj.ravel()


def gradient_images(img: np.ndarray):
    """First-order gradients of an image (Sec. 4.1, "Feature representation":
    convolution with [-1, 0, 1] and its transpose), as the central differences
    g_x(r, c) = x(r, c+1) - x(r, c-1), g_y(r, c) = x(r+1, c) - x(r-1, c).
    Readings: borders clamp to the edge (as the blur); the sign is that of
    the correlation with [-1, 0, 1] (a sign flip changes no distance)."""
    x = np.asarray(img, dtype=np.float64)
    h, w = x.shape
    cm, cp = np.maximum(np.arange(w) - 1, 0), np.minimum(np.arange(w) + 1, w - 1)
    rm, rp = np.maximum(np.arange(h) - 1, 0), np.minimum(np.arange(h) + 1, h - 1)
    return x[:, cp] - x[:, cm], x[rp, :] - x[rm, :]


def second_order_images(img: np.ndarray):
    """Second-order gradients of an image (Sec. 4.1, "Feature representation":
    convolution with [-1, 0, 2, 0, -1] and its transpose):
    g_xx(r, c) = 2 x(r, c) - x(r, c-2) - x(r, c+2), and g_yy likewise along
    the rows.  Readings: borders clamp to the edge, as for the first order."""
    x = np.asarray(img, dtype=np.float64)
    h, w = x.shape
    cm, cp = np.maximum(np.arange(w) - 2, 0), np.minimum(np.arange(w) + 2, w - 1)
    rm, rp = np.maximum(np.arange(h) - 2, 0), np.minimum(np.arange(h) + 2, h - 1)
    return 2.0 * x - x[:, cm] - x[:, cp], 2.0 * x - x[rm, :] - x[rp, :]


# Feature modes of a dictionary (Sec. 4.1): 0 = the LR patch minus its mean
# (P*P values); 1 = the first-order gradients of the LR image at the patch's
# pixels (g_x row-major, then g_y: 2*P*P values); 2 = the second-order
# gradients, laid out the same way (g_xx, then g_yy).
FEATURE_DIMS = {0: lambda P: P * P, 1: lambda P: 2 * P * P, 2: lambda P: 2 * P * P}


def gradient_fn(feature: int):
    """The gradient filter pair of a gradient feature mode (1 or 2)."""
    if feature == 1:
        return gradient_images
    if feature == 2:
        return second_order_images
    raise ValueError("feature must be 0, 1 or 2")


def patch_features(img: np.ndarray, P: int, feature: int = 0):
    """Feature of every overlapping P x P patch and its pixel mean mu.

    Sec. 4.1 ("Feature representation") hashes a feature of the LR patch:
    feature 0 is the mean-subtracted patch, feature 1 the first-order
    gradients of the image at the patch's pixels (``gradient_images``),
    feature 2 the second-order ones (``second_order_images``)."""
    x = np.asarray(img, dtype=np.float64)
    ii, jj = patch_origins(x.shape[0], x.shape[1], P)
    n = len(ii)
    px = np.empty((n, P * P))
    for a in range(P):
        for b in range(P):
            px[:, a * P + b] = x[ii + a, jj + b]
    mu = px.mean(axis=1)
    if feature == 0:
        return px - mu[:, None], mu
    gx, gy = gradient_fn(feature)(x)
    v = np.empty((n, 2 * P * P))
    for a in range(P):
        for b in range(P):
            v[:, a * P + b] = gx[ii + a, jj + b]
            v[:, P * P + a * P + b] = gy[ii + a, jj + b]
    return v, mu


@dataclasses.dataclass
class Dictionary:
    """N LR/HR patch pairs with integer IDs 0..N-1 (Sec. 2.1).

    lr_pix  float32 [N][P*P]   stored LR patch pixels
    feat    float64 [N][D]     LR feature (D = P*P pixels minus mean, or
                               D = 2*P*P gradients: see patch_features)
    mu      float64 [N]        LR patch mean
    hr_res  float64 [N][PH*PH] HR patch minus the LR patch mean
    """
    scale: int
    patch: int
    lr_pix: np.ndarray
    feat: np.ndarray
    mu: np.ndarray
    hr_res: np.ndarray
    feature: int = 0      # feature mode (see patch_features)

    @property
    def n(self) -> int:
        return self.feat.shape[0]

    @property
    def hr_patch(self) -> int:
        return self.scale * self.patch


def build_dictionary(hr_images, positions, s: int, P: int, sigma: float, feature: int = 0,
                     with_hr: bool = True) -> Dictionary:
    """Training pairs (Sec. 2.1, Sec. 5.1): every HR training image is blurred
    and down-sampled; at each position (image, i, j) the LR patch at (i, j) is
    paired with the HR patch of side s*P at (s*i, s*j).

    Readings: the LR training image is stored at float32, the precision of the
    test LR image; the LR patch mean is subtracted from both patches and is
    added back at reconstruction time.  Position k in ``positions`` (sorted by
    image, row, column) is the unique ID k.  Features 1 and 2: the gradients
    of the whole (float32) LR training image at the patch's pixels.
    with_hr=False leaves hr_res out (None): the search needs only the LR side,
    and an entry's HR residual depends on its own position alone, so a
    dictionary built from a subset of the positions gives those entries'."""
    hr64 = [np.asarray(x, np.float64) for x in hr_images]
    lr_imgs = [degrade(x, s, sigma).astype(np.float32) for x in hr64]
    PH = s * P
    N = len(positions)
    lr_pix = np.empty((N, P * P), np.float32)
    hr = np.empty((N, PH * PH)) if with_hr else None
    for n, (m, i, j) in enumerate(np.asarray(positions)):
        lr_pix[n] = lr_imgs[m][i:i + P, j:j + P].ravel()
        if with_hr:
            hr[n] = hr64[m][s * i:s * i + PH, s * j:s * j + PH].ravel()
    lr64 = lr_pix.astype(np.float64)
    mu = lr64.mean(axis=1)
    if feature == 0:
        feat = lr64 - mu[:, None]
    else:
        grads = [gradient_fn(feature)(x) for x in lr_imgs]
        feat = np.empty((N, 2 * P * P))
        for n, (m, i, j) in enumerate(np.asarray(positions)):
            gx, gy = grads[m]
            feat[n, :P * P] = gx[i:i + P, j:j + P].ravel()
            feat[n, P * P:] = gy[i:i + P, j:j + P].ravel()
    return Dictionary(s, P, lr_pix, feat, mu, hr - mu[:, None] if with_hr else None, feature)


def dictionary_from_lr_hr(lr_img, hr_img, s: int, P: int, feature: int = 0) -> Dictionary:
    """Every patch pair of one given LR/HR image pair (used for the
    exact-reconstruction pins: the test image's own patches in the dictionary,
    as in the girl-image experiment of Sec. 5.2)."""
    lr = np.asarray(lr_img, np.float32)
    hr = np.asarray(hr_img, np.float64)
    ii, jj = patch_origins(lr.shape[0], lr.shape[1], P)
    PH = s * P
    lr_pix = np.stack([lr[i:i + P, j:j + P].ravel() for i, j in zip(ii, jj)])
    hrp = np.stack([hr[s * i:s * i + PH, s * j:s * j + PH].ravel() for i, j in zip(ii, jj)])
    feat, mu = patch_features(lr, P, feature)
    return Dictionary(s, P, lr_pix, feat, mu, hrp - mu[:, None], feature)


# ---------------------------------------------------------------------------
# Training-crop sampling (Sec. 5.1 "Training Data Generation")
# ---------------------------------------------------------------------------


def gradient_magnitude(img: np.ndarray) -> np.ndarray:
    """Sec. 5.1: the horizontal and vertical first-order gradients at every
    pixel (``gradient_images``), combined per pixel.  Reading: the Euclidean
    magnitude sqrt(g_x^2 + g_y^2), in FP64."""
    gx, gy = gradient_images(img)
    return np.sqrt(gx * gx + gy * gy)


def sample_crop_centers(img: np.ndarray, u: np.ndarray):
    """Sec. 5.1: a CDF over the pixels from their gradient values, and the
    centre pixel of a crop drawn from it, for each uniform draw u in [0, 1)
    (the draws are inputs).  Readings: pixels in row-major order, mass =
    gradient magnitude; the drawn pixel is the first whose cumulative mass
    exceeds u * total (so a pixel without mass is never drawn); a flat image
    (no mass) draws uniformly, pixel floor(u * n).  Returns int64 rows and
    columns."""
    x = np.asarray(img, dtype=np.float64)
    h, w = x.shape
    n = h * w
    u = np.asarray(u, dtype=np.float64)
    cdf = np.cumsum(gradient_magnitude(x).ravel())
    total = cdf[-1]
    if total > 0:
        idx = np.searchsorted(cdf, u * total, side="right")
    else:
        idx = np.floor(u * n).astype(np.int64)
    idx = np.minimum(idx, n - 1)
    return idx // w, idx % w


def crop_windows(rows, cols, h: int, w: int, ch: int, cw: int):
    """Top-left corners of ch x cw crops centred at (rows, cols) (Sec. 5.1:
    a crop centred at the drawn pixel).  Reading: the centre of an even side
    is the pixel after the middle (top = row - ch // 2), and a window that
    would leave the image is shifted inside it."""
    top = np.clip(np.asarray(rows) - ch // 2, 0, h - ch)
    left = np.clip(np.asarray(cols) - cw // 2, 0, w - cw)
    return top, left


# ---------------------------------------------------------------------------
# Seeded random draws: projections (Eq. 10-11) and dictionary positions
# (Sec. 5.1), from the counter-based generator Philox4x32-10 of Salmon,
# Moraes, Dror and Shaw ("Parallel random numbers: as easy as 1, 2, 3", SC
# 2011), written from its published definition.
# ---------------------------------------------------------------------------

PHILOX_M = (0xD2511F53, 0xCD9E8D57)     # round multipliers
PHILOX_W = (0x9E3779B9, 0xBB67AE85)     # key schedule (Weyl) increments
CAUCHY_EPS = 1e-3                       # |b| >= eps in Eq. 11 (the paper gives no value)


def philox4x32_10(ctr: np.ndarray, seed: int) -> np.ndarray:
    """Philox4x32 with 10 rounds for counters ctr uint32 [n][4] under the
    64-bit key `seed` (low word first).  One round maps (c0, c1, c2, c3) to
    (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key
    gains the Weyl increments before every round but the first.  Returns
    uint32 [n][4]."""
    c = np.asarray(ctr, np.uint64).reshape(-1, 4).copy()
    k0, k1 = np.uint64(seed & 0xFFFFFFFF), np.uint64((seed >> 32) & 0xFFFFFFFF)
    m0, m1 = np.uint64(PHILOX_M[0]), np.uint64(PHILOX_M[1])
    lo32 = np.uint64(0xFFFFFFFF)
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(PHILOX_W[0])) & lo32
            k1 = (k1 + np.uint64(PHILOX_W[1])) & lo32
        p0 = m0 * c[:, 0]
        p1 = m1 * c[:, 2]
        c = np.stack([(p1 >> np.uint64(32)) ^ c[:, 1] ^ k0, p1 & lo32,
                      (p0 >> np.uint64(32)) ^ c[:, 3] ^ k1, p0 & lo32], axis=1)
    return c.astype(np.uint32)


def _unit(x: np.ndarray) -> np.ndarray:
    """A 32-bit word to a uniform value in (0, 1): (x + 1/2) / 2^32."""
    return (np.asarray(x, np.float64) + 0.5) * 2.0 ** -32


def _normal(words: np.ndarray) -> np.ndarray:
    """Box-Muller (cosine branch) from the first two words of each counter's
    output, in FP64: sqrt(-2 ln u1) cos(2 pi u2)."""
    u1, u2 = _unit(words[:, 0]), _unit(words[:, 1])
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def _ctr(n, c1=0, c2=0, c3=0) -> np.ndarray:
    n = np.asarray(n, np.uint64)
    out = np.zeros((n.size, 4), np.uint64)
    out[:, 0] = n & np.uint64(0xFFFFFFFF)
    out[:, 1] = (n >> np.uint64(32)) + np.uint64(c1)
    out[:, 2] = c2
    out[:, 3] = c3
    return out


def projection_draws(seed: int, L: int, k: int, D: int, w: float, dist: int = 0, eps: float = CAUCHY_EPS):
    """The random draws of Eq. 10 from `seed`: alpha float32 [L*k][D] and beta
    float32 [L*k].  Element n (row-major) of alpha: dist 0 (Gaussian, the
    workloads') the normal of counter (n, 0, 0, 0); dist 1 (Cauchy, Eq. 11)
    a / b, a that normal and b the normal of counter (n, t, 1, 0) for the
    first t = 0, 1, ... with |b| >= eps.  beta_j = u w, u from counter
    (j, 0, 0, 1), kept below w after rounding to float32."""
    n = L * k * D
    a = _normal(philox4x32_10(_ctr(np.arange(n)), seed))
    if dist == 1:
        b = np.empty(n)
        todo = np.arange(n)
        t = 0
        while todo.size:
            bt = _normal(philox4x32_10(_ctr(todo, c1=t, c2=1), seed))
            ok = np.abs(bt) >= eps
            b[todo[ok]] = bt[ok]
            todo = todo[~ok]
            t += 1
        a = a / b
    elif dist != 0:
        raise ValueError("dist must be 0 (Gaussian) or 1 (Cauchy)")
    alpha = a.astype(np.float32).reshape(L * k, D)
    beta = (_unit(philox4x32_10(_ctr(np.arange(L * k), c3=1), seed)[:, 0]) * w).astype(np.float32)
    beta = np.minimum(beta, np.nextafter(np.float32(w), np.float32(0.0)))
    return alpha, beta


def sample_positions_seeded(seed: int, lr_sizes, P: int, n_pairs: int) -> np.ndarray:
    """Dictionary positions (Sec. 2.1, Sec. 5.1), uniform without replacement
    over every P x P patch origin of every LR training image (origins numbered
    image by image, row by row): origin o draws the 64-bit key (w0, w1) of
    counter (o, 0, 0, 2); the n_pairs origins with the smallest (key, o) are
    kept, in origin order, so that a position's rank is its ID.  lr_sizes:
    (h, w) per image.  Returns int32 [n_pairs][3] = (image, row, col)."""
    counts = [(h - P + 1) * (w - P + 1) for h, w in lr_sizes]
    total = int(sum(counts))
    if not 0 < n_pairs <= total:
        raise ValueError("n_pairs must be in 1..number of origins")
    words = philox4x32_10(_ctr(np.arange(total), c3=2), seed).astype(np.uint64)
    key = (words[:, 0] << np.uint64(32)) | words[:, 1]
    order = np.lexsort((np.arange(total), key))
    chosen = np.sort(order[:n_pairs])
    starts = np.cumsum([0] + counts)
    img = np.searchsorted(starts, chosen, side="right") - 1
    rem = chosen - starts[img]
    nw = np.array([w - P + 1 for _, w in lr_sizes])[img]
    return np.stack([img, rem // nw, rem % nw], axis=1).astype(np.int32)


# ---------------------------------------------------------------------------
# Hashing (Sec. 3.2; Sec. 4.1, Eq. 10)
# ---------------------------------------------------------------------------


def hash_values(v: np.ndarray, alpha: np.ndarray, beta: np.ndarray, w: float):
    """Eq. 10: h(v) = floor((alpha . v + beta) / r) for every projection.

    alpha float32 [L*k][d], beta float32 [L*k] (drawn outside, passed in);
    r is the bucket width w.  Returns int64 h [n][L*k] and, per row, the
    distance of the nearest ratio (alpha.v + beta)/w to an integer (a row
    with a value below 1e-5 is "boundary-affected")."""
    t = np.asarray(v, np.float64) @ np.asarray(alpha, np.float64).T + np.asarray(beta, np.float64)
    ratio = t / w
    h = np.floor(ratio).astype(np.int64)
    margin = np.abs(ratio - np.rint(ratio)).min(axis=1)
    return h, margin


def hash_margins(v: np.ndarray, alpha: np.ndarray, beta: np.ndarray, w: float) -> np.ndarray:
    """Distance of every ratio (alpha.v + beta)/w of Eq. 10 to the nearest
    integer, per projection: [n][L*k].  A value below 1e-5 marks a projection
    whose floor an FP32 evaluation may place in the neighbouring bin."""
    t = np.asarray(v, np.float64) @ np.asarray(alpha, np.float64).T + np.asarray(beta, np.float64)
    ratio = t / w
    return np.abs(ratio - np.rint(ratio))


def membership_is_certain(hq: np.ndarray, he: np.ndarray, me: np.ndarray, L: int, k: int,
                          bnd: float = 1e-5) -> bool:
    """Whether an entry's membership in a query's candidate set (the union of
    the query's bins over the L tables, Sec. 3.2) survives moving any of the
    entry's boundary-affected projections (margin me < bnd) to the
    neighbouring bin.  hq, he: the k*L hash values of the query and the entry;
    the query's own projections are assumed clear of boundaries."""
    certain_in = possible_in = False
    for l in range(L):
        sl = slice(l * k, (l + 1) * k)
        eq = hq[sl] == he[sl]
        near = me[sl] < bnd
        if eq.all() and not near.any():
            certain_in = True
        if (eq | near).all():
            possible_in = True
    return certain_in == possible_in


def mix64(z):
    """Stafford's variant-13 64-bit finaliser (the SplitMix64 output mixer),
    applied elementwise to uint64 arrays with wrap-around arithmetic."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def fold_keys(h: np.ndarray, L: int, k: int) -> np.ndarray:
    """Bucket key of each table: g_l(v) = (h_1, ..., h_k) (Sec. 3.2) folded
    into one 64-bit integer, x = l; x = mix64(x XOR (uint32(h_j) + G*(j+1)))
    for j = 0..k-1, G = 0x9E3779B97F4A7C15 (reading: the paper's bin is the
    k-tuple itself; equal tuples give equal keys)."""
    n = h.shape[0]
    keys = np.empty((n, L), np.uint64)
    with np.errstate(over="ignore"):
        for l in range(L):
            x = np.full(n, l, np.uint64)
            for j in range(k):
                hj = (h[:, l * k + j] & 0xFFFFFFFF).astype(np.uint64)
                x = mix64(x ^ (hj + np.uint64((GOLDEN64 * (j + 1)) & MASK64)))
            keys[:, l] = x
    return keys


@dataclasses.dataclass
class LshIndex:
    """L hash tables of bins holding patch IDs (Sec. 3.2, Sec. 4.1).

    keys     uint64 [N][L]      bucket key of every dictionary entry
    margin   float64 [N]        boundary margin of every entry's projections
    buckets  list of L dicts    key -> int64 array of IDs, ascending
    """
    L: int
    k: int
    w: float
    alpha: np.ndarray
    beta: np.ndarray
    keys: np.ndarray
    margin: np.ndarray
    buckets: list


def build_index(d: Dictionary, alpha, beta, w: float, L: int, k: int) -> LshIndex:
    """Hash every dictionary feature into L tables (Sec. 4.1: the ID of each
    training patch is stored in the bin of its k hash values, per table).
    Entries are hashed in blocks of rows (each row's values depend on that
    row alone) to bound the memory of the projections."""
    n = d.feat.shape[0]
    keys = np.empty((n, L), np.uint64)
    margin = np.empty(n)
    for r0 in range(0, n, 1 << 18):
        h, margin[r0:r0 + (1 << 18)] = hash_values(d.feat[r0:r0 + (1 << 18)], alpha, beta, w)
        keys[r0:r0 + (1 << 18)] = fold_keys(h, L, k)
    buckets = []
    for l in range(L):
        order = np.argsort(keys[:, l], kind="stable")
        ks = keys[order, l]
        cut = np.flatnonzero(ks[1:] != ks[:-1]) + 1
        starts = np.concatenate([[0], cut])
        ends = np.concatenate([cut, [len(ks)]])
        buckets.append({int(ks[a]): np.sort(order[a:b]) for a, b in zip(starts, ends)})
    return LshIndex(L, k, w, np.asarray(alpha), np.asarray(beta), keys, margin, buckets)


def candidate_set(index: LshIndex, qkeys: np.ndarray, min_hits: int = 1,
                  max_candidates: int = 0) -> np.ndarray:
    """Candidate IDs of one query (Sec. 3.2; Sec. 4.2): the union of the bins
    the query falls in, over the L tables.

    ``min_hits`` t: an ID must be found in at least t of the L tables (the
    hash-match criterion of Sec. 4.1).  ``max_candidates``: if > 0, tables
    are visited in order l = 0..L-1, each bin in ascending ID, and the
    search stops once that many distinct IDs were collected (the early stop
    of Sec. 4.2; reading: the stop is exact at the cap).  Returns ascending
    unique IDs (collection order is only used for the cap)."""
    found = [index.buckets[l].get(int(qkeys[l]), np.empty(0, np.int64)) for l in range(index.L)]
    if max_candidates > 0:
        seen, order = set(), []
        for ids in found:
            for c in ids:
                c = int(c)
                if c not in seen:
                    seen.add(c)
                    order.append(c)
                    if len(order) == max_candidates:
                        return np.sort(np.array(order, np.int64))
        return np.sort(np.array(order, np.int64))
    if not found:
        return np.empty(0, np.int64)
    n = int(max((f.max() for f in found if len(f)), default=-1)) + 1
    hits = np.zeros(max(n, 1), np.int32)
    for ids in found:
        hits[ids] += 1
    return np.flatnonzero(hits >= max(min_hits, 1)).astype(np.int64)


def neighbour_exclusions(qv: np.ndarray, q_margin: np.ndarray, dist: np.ndarray, d: "Dictionary",
                         index: "LshIndex", rel: float = 1e-6, bnd: float = 1e-5, feat_norm2=None) -> np.ndarray:
    """Queries whose K nearest another exact implementation (FP32 keys and
    distances) may select or order differently, for comparisons with this
    oracle: (a) a projection of the query within bnd of a bin boundary (its
    own bins are uncertain, Eq. 10); (b) an entry of the whole dictionary at
    distance <= the query's (K+1)-th nearest candidate whose membership in the
    candidate set (Sec. 3.2) is uncertain (``membership_is_certain``); (c) two
    of the K+1 nearest FP64 distances within rel of each other (the tie rule
    then decides).  qv [n][D] features, q_margin [n], dist [n][K+1] from
    ``query`` with K+1 neighbours.  Returns bool [n]."""
    qv = np.asarray(qv, np.float64)
    n = qv.shape[0]
    ex = np.asarray(q_margin) < bnd
    gaps = np.diff(dist, axis=1)
    ex |= (gaps <= rel * np.maximum(dist[:, 1:], 1e-30)).any(axis=1)
    fn = (d.feat * d.feat).sum(axis=1) if feat_norm2 is None else feat_norm2
    hq_all, _ = hash_values(qv, index.alpha, index.beta, index.w)
    for i in range(n):
        if ex[i]:
            continue
        D = dist[i, -1]
        approx = fn - 2.0 * (d.feat @ qv[i]) + qv[i] @ qv[i]
        idx = np.flatnonzero(approx <= D + 1e-9 * (1.0 + D))
        exact = ((d.feat[idx] - qv[i]) ** 2).sum(axis=1)
        idx = idx[exact <= D]
        if len(idx) == 0:
            continue
        he, _ = hash_values(d.feat[idx], index.alpha, index.beta, index.w)
        me = hash_margins(d.feat[idx], index.alpha, index.beta, index.w)
        for j in range(len(idx)):
            if not membership_is_certain(hq_all[i], he[j], me[j], index.L, index.k, bnd):
                ex[i] = True
                break
    return ex


def top_k(qv: np.ndarray, cand: np.ndarray, feat: np.ndarray, K: int):
    """The K nearest candidates of one query (Sec. 3.1, step 1a; Sec. 4.2).

    Distance: squared Euclidean, sum_i (q_i - c_i)^2, in FP64.  Order: by
    distance, ties by ascending ID (reading: the paper gives no tie rule).
    If fewer than K candidates exist, the list is padded with the nearest
    dictionary entries outside the candidate set, in the same order
    (reading: the paper does not treat this case).
    Returns (ids int64 [K], dist float64 [K], n_padded)."""
    qv = np.asarray(qv, np.float64)
    d = ((feat[cand] - qv) ** 2).sum(axis=1)
    order = np.lexsort((cand, d))
    ids = cand[order[:K]]
    dist = d[order[:K]]
    npad = 0
    if len(ids) < K:
        rest = np.setdiff1d(np.arange(feat.shape[0]), cand)
        dr = ((feat[rest] - qv) ** 2).sum(axis=1)
        o2 = np.lexsort((rest, dr))[:K - len(ids)]
        npad = len(o2)
        ids = np.concatenate([ids, rest[o2]])
        dist = np.concatenate([dist, dr[o2]])
    return ids.astype(np.int64), dist, npad


def lle_weights(qv: np.ndarray, nbr_feat: np.ndarray, reg_rel: float, d_first: float):
    """Eq. 12-13: min || y - sum_m w_m y_m ||^2 subject to sum_m w_m = 1, over
    the K selected neighbours.

    With Z = y - y_m (rows), the local Gram matrix is G = Z Z^T; it is
    regularised as C = G + eps I, eps = reg_rel * trace(G) (reading: the
    paper states no regulariser); C z = 1 is solved by Cholesky and
    w = z / sum(z).  If the nearest distance is exactly 0 the query equals
    a dictionary entry and w is one-hot on it (this also covers trace(G)=0).
    Returns (w [K], condition bound (tr G + eps)/eps)."""
    K = nbr_feat.shape[0]
    if d_first == 0.0:
        w = np.zeros(K)
        w[0] = 1.0
        return w, 1.0
    Z = np.asarray(qv, np.float64)[None, :] - nbr_feat
    G = Z @ Z.T
    eps = reg_rel * np.trace(G)
    C = G + eps * np.eye(K)
    Lc = np.linalg.cholesky(C)
    # forward substitution L u = 1, then back substitution L^T z = u
    u = np.zeros(K)
    for i in range(K):
        u[i] = (1.0 - Lc[i, :i] @ u[:i]) / Lc[i, i]
    z = np.zeros(K)
    for i in range(K - 1, -1, -1):
        z[i] = (u[i] - Lc[i + 1:, i] @ z[i + 1:]) / Lc[i, i]
    return z / z.sum(), (np.trace(G) + eps) / eps


def blend_patches(nbr: np.ndarray, wgt: np.ndarray, mu: np.ndarray, hr_res: np.ndarray) -> np.ndarray:
    """Eq. 14: x^t = sum_m w_m x^m, applied to the HR residual patches, plus the
    query's LR mean mu (reading of the mean handling).  Returns [n][PH*PH]."""
    return mu[:, None] + np.einsum("nm,nmp->np", wgt, hr_res[nbr])


def overlap_add(patches: np.ndarray, h: int, w: int, s: int, P: int) -> np.ndarray:
    """Place every blended HR patch at (s*i, s*j) and average where patches
    overlap (the simple averaging of overlaps, Sec. 1; the prior of Eq. 9
    only penalises their disagreement).  Output (s*h) x (s*w)."""
    PH = s * P
    acc = np.zeros((s * h, s * w))
    cnt = np.zeros((s * h, s * w))
    ii, jj = patch_origins(h, w, P)
    for n in range(len(ii)):
        Y, X = s * ii[n], s * jj[n]
        acc[Y:Y + PH, X:X + PH] += patches[n].reshape(PH, PH)
        cnt[Y:Y + PH, X:X + PH] += 1.0
    return acc / cnt


def overlap_add_adjoint(z: np.ndarray, h: int, w: int, s: int, P: int) -> np.ndarray:
    """Adjoint of ``overlap_add``: patch n receives z / n_cov over its
    footprint."""
    PH = s * P
    cnt = np.zeros_like(z)
    ii, jj = patch_origins(h, w, P)
    for n in range(len(ii)):
        cnt[s * ii[n]:s * ii[n] + PH, s * jj[n]:s * jj[n] + PH] += 1.0
    zc = z / cnt
    out = np.empty((len(ii), PH * PH))
    for n in range(len(ii)):
        out[n] = zc[s * ii[n]:s * ii[n] + PH, s * jj[n]:s * jj[n] + PH].ravel()
    return out


# ---------------------------------------------------------------------------
# Back-projection with the approximate cross-bilateral filter
# (Sec. 4, Eq. 6-7; Sec. 4.3, Eq. 15-17)
# ---------------------------------------------------------------------------


def spatial_kernel(sigma_sp: float, radius: int) -> np.ndarray:
    """Eq. 3: c(x, y) = exp(-||x - y||^2 / (2 sigma_c^2)) on the
    (2R+1)^2 window, normalised to sum 1 (the normalised filter C of Eq. 17)."""
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    c = np.exp(-(t[:, None] ** 2 + t[None, :] ** 2) / (2.0 * sigma_sp * sigma_sp))
    return c / c.sum()


def window_sum_clamped(x: np.ndarray, kern: np.ndarray) -> np.ndarray:
    """sum over the window of kern(delta) * x(clamp(p + delta))."""
    r = kern.shape[0] // 2
    h, w = x.shape
    xp = np.pad(x, r, mode="edge")
    out = np.zeros((h, w))
    for a in range(2 * r + 1):
        for b in range(2 * r + 1):
            out += kern[a, b] * xp[a:a + h, b:b + w]
    return out


def back_project(x: np.ndarray, y: np.ndarray, s: int, blur_sigma: float, iters: int,
                 sigma_sp: float, sigma_r: float, radius: int) -> np.ndarray:
    """Error back-projection (Sec. 4), ``iters`` times:

    e = (x * g) down - y                               (Eq. 6)
    u = e up           (each LR value copied to its s x s block)
    G = C * u          (normalised spatial Gaussian, Eq. 3 / Eq. 17)
    m = mean of x over the same window Gamma          (Eq. 15)
    r = exp(-(x - m)^2 / (2 sigma_r^2))                (Eq. 15)
    x <- x - r * G                                     (Eq. 7, Eq. 16-17)

    Readings: the update subtracts the filtered error (Eq. 6 defines e as
    simulated minus observed, so adding it would move away from the data);
    the range term's guide is the current HR estimate; the window Gamma is
    the (2R+1)^2 square for both the spatial filter and the mean; borders
    are clamped."""
    x = np.asarray(x, np.float64).copy()
    y = np.asarray(y, np.float64)
    ck = spatial_kernel(sigma_sp, radius)
    box = np.full((2 * radius + 1, 2 * radius + 1), 1.0 / (2 * radius + 1) ** 2)
    for _ in range(iters):
        e = degrade(x, s, blur_sigma) - y
        u = np.kron(e, np.ones((s, s)))
        g = window_sum_clamped(u, ck)
        m = window_sum_clamped(x, box)
        r = np.exp(-(x - m) ** 2 / (2.0 * sigma_r * sigma_r))
        x = x - r * g
    return x


# ---------------------------------------------------------------------------
# The whole inference (Sec. 4: Eq. 10, Eq. 12-14, Eq. 6-7)
# ---------------------------------------------------------------------------


@dataclasses.dataclass
class QueryResult:
    keys: np.ndarray        # uint64 [n][L]
    margin: np.ndarray      # float64 [n] boundary margin of the query's projections
    n_cand: np.ndarray      # int64 [n] |C(q)|
    n_bucket: np.ndarray    # int64 [n] sum over tables of the bin sizes
    nbr: np.ndarray         # int64 [n][K]
    dist: np.ndarray        # float64 [n][K]
    n_padded: np.ndarray    # int64 [n]
    wgt: np.ndarray         # float64 [n][K]
    mu: np.ndarray          # float64 [n]
    feat: np.ndarray        # float64 [n][d]


def query(lr: np.ndarray, d: Dictionary, index: LshIndex, K: int, reg_rel: float,
          rows=None, min_hits: int = 1, max_candidates: int = 0) -> QueryResult:
    """Per-patch inference of Sec. 4.2 for the queries numbered ``rows``
    (default: all, row order): hash, collect the candidates, K nearest,
    LLE weights."""
    v, mu = patch_features(lr, d.patch, d.feature)
    if rows is None:
        rows = np.arange(v.shape[0])
    rows = np.asarray(rows)
    v, mu = v[rows], mu[rows]
    h, margin = hash_values(v, index.alpha, index.beta, index.w)
    keys = fold_keys(h, index.L, index.k)
    n = len(rows)
    nbr = np.zeros((n, K), np.int64)
    dist = np.zeros((n, K))
    wgt = np.zeros((n, K))
    ncand = np.zeros(n, np.int64)
    nbuck = np.zeros(n, np.int64)
    npad = np.zeros(n, np.int64)
    for q in range(n):
        cand = candidate_set(index, keys[q], min_hits, max_candidates)
        ncand[q] = len(cand)
        nbuck[q] = sum(len(index.buckets[l].get(int(keys[q, l]), ())) for l in range(index.L))
        nbr[q], dist[q], npad[q] = top_k(v[q], cand, d.feat, K)
        wgt[q], _ = lle_weights(v[q], d.feat[nbr[q]], reg_rel, dist[q, 0])
    return QueryResult(keys, margin, ncand, nbuck, nbr, dist, npad, wgt, mu, v)


def reconstruct(nbr, wgt, mu, d: Dictionary, h: int, w: int) -> np.ndarray:
    """Eq. 14 for every query, then the overlap average: the HR estimate before
    back-projection."""
    return overlap_add(blend_patches(nbr, wgt, mu, d.hr_res), h, w, d.scale, d.patch)


def upscale(lr, d: Dictionary, index: LshIndex, K: int, reg_rel: float, bp_iters: int,
            blur_sigma: float, sigma_sp: float, sigma_r: float, radius: int):
    """Full inference: every query, reconstruction, back-projection.
    Returns (HR image, QueryResult, HR before back-projection)."""
    lr = np.asarray(lr, np.float32)
    h, w = lr.shape
    qr = query(lr, d, index, K, reg_rel)
    x0 = reconstruct(qr.nbr, qr.wgt, qr.mu, d, h, w)
    x = back_project(x0, lr, d.scale, blur_sigma, bp_iters, sigma_sp, sigma_r, radius)
    return x, qr, x0


# ---------------------------------------------------------------------------
# MAP energy and its gradients (Sec. 4: Eq. 5, Eq. 8-9)
# ---------------------------------------------------------------------------


def overlap_prior(patches: np.ndarray, h: int, w: int, s: int, P: int) -> float:
    """Eq. 9 (without the constant 1/(2 sigma_o^2), folded into lambda):
    sum over 4-connected neighbour patches (right, down) of the squared
    difference of the two HR patches on the intersection of their HR
    footprints (reading: neighbours are the LR-grid neighbours)."""
    PH = s * P
    nh, nw = h - P + 1, w - P + 1
    pt = patches.reshape(nh, nw, PH, PH)
    ov = PH - s
    if ov <= 0:
        return 0.0
    right = pt[:, :-1, :, s:] - pt[:, 1:, :, :ov]
    down = pt[:-1, :, s:, :] - pt[1:, :, :ov, :]
    return float((right ** 2).sum() + (down ** 2).sum())


def overlap_prior_grad(patches: np.ndarray, h: int, w: int, s: int, P: int) -> np.ndarray:
    """Gradient of ``overlap_prior`` with respect to every patch."""
    PH = s * P
    nh, nw = h - P + 1, w - P + 1
    pt = patches.reshape(nh, nw, PH, PH)
    g = np.zeros_like(pt)
    ov = PH - s
    if ov > 0:
        right = pt[:, :-1, :, s:] - pt[:, 1:, :, :ov]
        g[:, :-1, :, s:] += 2.0 * right
        g[:, 1:, :, :ov] -= 2.0 * right
        down = pt[:-1, :, s:, :] - pt[1:, :, :ov, :]
        g[:-1, :, s:, :] += 2.0 * down
        g[1:, :, :ov, :] -= 2.0 * down
    return g.reshape(patches.shape)


def data_energy(x, y, s: int, blur_sigma: float) -> float:
    """Data term ||D B x - y||^2 (Gaussian noise model of Sec. 4, Eq. 6)."""
    r = degrade(x, s, blur_sigma) - y
    return float((r * r).sum())


def data_energy_grad(x, y, s: int, blur_sigma: float) -> np.ndarray:
    """d/dx ||D B x - y||^2 = 2 B^T D^T (D B x - y)."""
    r = degrade(x, s, blur_sigma) - y
    return 2.0 * degrade_adjoint(r, s, blur_sigma, np.shape(x))


def map_energy(hr_res, nbr, wgt, mu, y, h: int, w: int, s: int, P: int, blur_sigma: float,
               lam: float) -> float:
    """E(R) = ||D B x - y||^2 + lambda * prior(patches), x = overlap average of
    the patches, patches = mu + sum_m w R[nbr] (Eq. 8-9, Eq. 14), with the
    neighbour IDs and weights held fixed."""
    p = blend_patches(nbr, wgt, mu, hr_res)
    x = overlap_add(p, h, w, s, P)
    return data_energy(x, y, s, blur_sigma) + lam * overlap_prior(p, h, w, s, P)


def map_energy_grad_dict(hr_res, nbr, wgt, mu, y, h: int, w: int, s: int, P: int,
                         blur_sigma: float, lam: float) -> np.ndarray:
    """dE/dR_j = sum over uses (n, m) with nbr[n, m] = j of w[n, m] dE/dPatch_n,
    dE/dPatch_n = OA^T(dE/dx) + lambda * d prior / d Patch_n."""
    p = blend_patches(nbr, wgt, mu, hr_res)
    x = overlap_add(p, h, w, s, P)
    gx = data_energy_grad(x, y, s, blur_sigma)
    gp = overlap_add_adjoint(gx, h, w, s, P) + lam * overlap_prior_grad(p, h, w, s, P)
    gR = np.zeros_like(hr_res)
    for m in range(nbr.shape[1]):
        np.add.at(gR, nbr[:, m], wgt[:, m:m + 1] * gp)
    return gR


# ---------------------------------------------------------------------------
# Collision law of p-stable LSH (Sec. 3.2, Def. 1; used as a test pin)
# ---------------------------------------------------------------------------


def gaussian_collision_probability(c: float, w: float) -> float:
    """Probability that two points at Euclidean distance c share one
    Gaussian-projection hash value floor((a.v + b)/w), b ~ U[0, w):
    p(c) = 1 - 2 Phi(-w/c) - 2 / (sqrt(2 pi) (w/c)) (1 - exp(-(w/c)^2 / 2))."""
    r = w / c
    phi = 0.5 * math.erfc(r / math.sqrt(2.0))
    return 1.0 - 2.0 * phi - 2.0 / (math.sqrt(2.0 * math.pi) * r) * (1.0 - math.exp(-r * r / 2.0))


def cauchy_collision_probability(c: float, w: float) -> float:
    """Probability that two points at l1 distance c share one Cauchy-projection
    hash value floor((a.v + b)/w), b ~ U[0, w) (the 1-stable case of the
    p-stable scheme the paper cites for its Cauchy projections, Eq. 11):
    p(c) = 2 atan(w/c) / pi - ln(1 + (w/c)^2) / (pi w/c)."""
    r = w / c
    return 2.0 * math.atan(r) / math.pi - math.log1p(r * r) / (math.pi * r)


__all__ = [n for n in dir() if not n.startswith("_")]
