"""Python front end of the C ABI: torch CUDA tensors in, torch CUDA tensors
out.  PyTorch supplies device memory (its caching allocator, handed to the
library as the context allocator) and the current stream; every step of the
method runs in the library's CUDA kernels."""
from __future__ import annotations

import atexit
import ctypes as C
import dataclasses
import os
import sys
import weakref

import numpy as np
import torch

from . import capi

# Live handles, closed at exit in dependency order (indexes, dictionaries,
# contexts) while the CUDA runtime and torch are still up.
_LIVE = {"index": weakref.WeakSet(), "dict": weakref.WeakSet(), "ctx": weakref.WeakSet()}


@atexit.register
def _close_all():
    for kind in ("index", "dict", "ctx"):
        for h in list(_LIVE[kind]):
            try:
                h.close()
            except Exception:
                pass


def _finalizing() -> bool:
    return sys.is_finalizing()


STAGES = ("features", "hash", "lookup", "knn", "lle", "overlap_add", "backproject", "knn_filter_kernel")


def _stream(stream=None) -> C.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(0 if t is None else t.data_ptr())


def _need(t: torch.Tensor, dtype, name: str):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")


@dataclasses.dataclass
class UpscaleParams:
    """Inference parameters (see zoom_upscale_params in include/zoom.h)."""
    K: int = 8
    reg_rel: float = 1e-3
    bp_iters: int = 5
    sigma_spatial: float = 1.5
    sigma_range: float = 0.1
    bp_radius: int = 3
    precision: int = 0
    rerank_mult: int = 2
    fp64_cond_threshold: float = 1e6
    search: int = 0

    def c(self) -> capi.UpscaleParams:
        return capi.UpscaleParams(self.K, self.reg_rel, self.bp_iters, self.sigma_spatial,
                                  self.sigma_range, self.bp_radius, self.precision,
                                  self.rerank_mult, self.fp64_cond_threshold, self.search)


class Context:
    """A library context on one CUDA device; device scratch memory comes from
    PyTorch's caching allocator, or from `allocator` (an object with methods
    alloc(nbytes, stream, user) -> device pointer or None, and
    free(ptr, nbytes, stream, user)), or -- torch_allocator=False and no
    allocator -- from cudaMallocAsync inside the library."""

    def __init__(self, device: int = 0, torch_allocator: bool = True, allocator=None):
        self.device = device
        alloc = None
        if allocator is not None:
            self._cb = (capi.ALLOC_FN(allocator.alloc), capi.FREE_FN(allocator.free))
            alloc = capi.Allocator(self._cb[0], self._cb[1], None)
        elif torch_allocator:
            def _a(nbytes, stream, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
                except Exception:  # the library reports ZOOM_ERR_OOM
                    return None

            def _f(ptr, nbytes, stream, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._cb = (capi.ALLOC_FN(_a), capi.FREE_FN(_f))
            alloc = capi.Allocator(self._cb[0], self._cb[1], None)
        self._alloc = alloc
        h = C.c_void_p()
        capi.call("zoom_ctx_create", device, C.byref(alloc) if alloc is not None else None,
                  C.byref(h))
        self.handle = h
        _LIVE["ctx"].add(self)

    def stats(self, stream=None) -> dict:
        st = capi.Stats()
        capi.call("zoom_get_stats", self.handle, _stream(stream), C.byref(st))
        out = {f: getattr(st, f) for f, _ in capi.Stats._fields_ if f != "ms_stage"}
        out["ms_stage"] = dict(zip(STAGES, list(st.ms_stage)[:len(STAGES)]))
        return out

    def set_stage_timing(self, enable: bool) -> None:
        capi.call("zoom_set_stage_timing", self.handle, 1 if enable else 0)

    def sync_status(self, stream=None) -> None:
        capi.call("zoom_sync_status", self.handle, _stream(stream))

    def set_fault_injection(self, mode: int, wait_limit_ns: int = 0) -> None:
        """Testing aid (zoom_set_fault_injection): mode 1 makes the
        tensor-core filter's bounded waits run out; wait_limit_ns bounds them
        (0: the default 2 s)."""
        capi.call("zoom_set_fault_injection", self.handle, int(mode), int(wait_limit_ns))

    def close(self):
        if getattr(self, "handle", None):
            torch.cuda.synchronize(self.device)
            capi.lib().zoom_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        if _finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


class Dictionary:
    """LR/HR patch-pair dictionary built on the device (zoom_build_dictionary)."""

    def __init__(self, ctx: Context, hr_images, positions, scale: int, patch: int,
                 blur_sigma: float = 0.8, stream=None, feature: int = 0, n_pairs: int | None = None,
                 seed: int = 7):
        """feature: 0 = LR pixels minus their mean, 1 / 2 = first / second-
        order gradients of the LR image at the patch's pixels (Sec. 4.1).
        positions: int32 [n][3] (image, LR row, LR col), or None to let the
        library draw n_pairs of them from `seed` (zoom_sample_positions)."""
        self.ctx = ctx
        for t in hr_images:
            _need(t, torch.float32, "hr image")
        n = len(hr_images)
        ptrs = (C.c_void_p * n)(*[t.data_ptr() for t in hr_images])
        hs = (C.c_int32 * n)(*[t.shape[0] for t in hr_images])
        ws = (C.c_int32 * n)(*[t.shape[1] for t in hr_images])
        degr = capi.Degradation(scale, patch, blur_sigma, feature)
        h = C.c_void_p()
        if positions is None:
            if n_pairs is None:
                raise ValueError("n_pairs is needed when the library draws the positions")
            npos, pptr = int(n_pairs), None
        else:
            pos = np.ascontiguousarray(positions, dtype=np.int32)
            npos, pptr = len(pos), pos.ctypes.data_as(C.POINTER(C.c_int32))
        capi.call("zoom_build_dictionary", ctx.handle, ptrs, hs, ws, n, C.byref(degr), npos, pptr, int(seed),
                  _stream(stream), C.byref(h))
        self._adopt(h)

    def _adopt(self, h):
        self.handle = h
        _LIVE["dict"].add(self)
        n, P, s, sig = C.c_int64(), C.c_int32(), C.c_int32(), C.c_double()
        f, dim = C.c_int32(), C.c_int32()
        capi.call("zoom_dict_info", h, C.byref(n), C.byref(P), C.byref(s), C.byref(sig), C.byref(f),
                  C.byref(dim))
        self.n, self.patch, self.scale, self.blur_sigma = n.value, P.value, s.value, sig.value
        self.feature, self.dim = f.value, dim.value

    def save(self, path: str, stream=None) -> None:
        """Writes every stored array to a file (zoom_dict_save)."""
        capi.call("zoom_dict_save", self.handle, os.fsencode(path), _stream(stream))

    @classmethod
    def load(cls, ctx: Context, path: str, stream=None) -> "Dictionary":
        """A dictionary read from a file written by save (zoom_dict_load)."""
        self = cls.__new__(cls)
        self.ctx = ctx
        h = C.c_void_p()
        capi.call("zoom_dict_load", ctx.handle, os.fsencode(path), _stream(stream), C.byref(h))
        self._adopt(h)
        return self

    def export(self, stream=None):
        d, ph = self.patch ** 2, (self.scale * self.patch) ** 2
        lr = np.empty((self.n, d), np.float32)
        mu = np.empty(self.n, np.float32)
        hr = np.empty((self.n, ph), np.float32)
        capi.call("zoom_dict_export", self.handle, lr.ctypes.data, mu.ctypes.data, hr.ctypes.data,
                  _stream(stream))
        return lr, mu, hr

    def close(self):
        # a dictionary outlives its context only by mistake; then it leaks
        if getattr(self, "handle", None) and getattr(self.ctx, "handle", None):
            torch.cuda.synchronize(self.ctx.device)
            capi.lib().zoom_dict_destroy(self.handle)
        self.handle = None

    def __del__(self):
        if _finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def sample_crops(ctx: Context, images, u, crop_h: int, crop_w: int, want_crops: bool = True, stream=None):
    """Training crops drawn where the HR images have structure (Sec. 5.1,
    zoom_sample_crops): images are CUDA float32 h x w tensors, u a numpy
    [n_images][draws] array of uniform draws in [0, 1).  Returns the windows
    (numpy int32 [n_images][draws][4]: centre row, centre column, top, left)
    and the crops (CUDA float32 [n_images * draws][crop_h][crop_w], or None)."""
    for t in images:
        _need(t, torch.float32, "image")
    u = np.ascontiguousarray(u, dtype=np.float64)
    n = len(images)
    if u.ndim != 2 or u.shape[0] != n:
        raise ValueError("u must be [n_images][draws]")
    ptrs = (C.c_void_p * n)(*[t.data_ptr() for t in images])
    hs = (C.c_int32 * n)(*[t.shape[0] for t in images])
    ws = (C.c_int32 * n)(*[t.shape[1] for t in images])
    win = np.empty((n, u.shape[1], 4), np.int32)
    crops = (torch.empty((n * u.shape[1], crop_h, crop_w), dtype=torch.float32, device=images[0].device)
             if want_crops else None)
    capi.call("zoom_sample_crops", ctx.handle, ptrs, hs, ws, n, u.ctypes.data, u.shape[1], crop_h, crop_w,
              win.ctypes.data, crops.data_ptr() if crops is not None else None, _stream(stream))
    return win, crops


class Index:
    """L-table p-stable LSH index over a dictionary (zoom_build_index)."""

    def __init__(self, dictionary: Dictionary, L: int, k: int, w: float, alpha=None, beta=None,
                 min_table_hits: int = 1, max_candidates: int = 0, stream=None, proj_dist: int = 0,
                 seed: int = 11):
        """alpha float32 [L*k][D], beta float32 [L*k] (Eq. 10), or both None
        to let the library draw them from `seed` (proj_dist 0 Gaussian, 1
        Cauchy by Eq. 11; zoom_lsh_draws)."""
        self.dictionary = dictionary
        prm = capi.LshParams(L, k, w, min_table_hits, max_candidates, proj_dist, int(seed))
        if alpha is None and beta is None:
            a = b = None
        else:
            a = np.ascontiguousarray(alpha, np.float32)
            b = np.ascontiguousarray(beta, np.float32)
            if a.shape != (L * k, dictionary.dim) or b.shape != (L * k,):
                raise ValueError(f"alpha must be [{L * k}][{dictionary.dim}] and beta [{L * k}]")
        h = C.c_void_p()
        capi.call("zoom_build_index", dictionary.handle, C.byref(prm), None if a is None else a.ctypes.data,
                  None if b is None else b.ctypes.data, _stream(stream), C.byref(h))
        self._adopt(h)

    def _adopt(self, h):
        self.handle = h
        _LIVE["index"].add(self)
        prm = capi.LshParams()
        capi.call("zoom_index_info", h, C.byref(prm))
        self.L, self.k, self.w = prm.L, prm.k, prm.w
        self.min_table_hits, self.max_candidates = prm.min_table_hits, prm.max_candidates

    def save(self, path: str, stream=None) -> None:
        """Writes the LSH parameters and projections to a file (zoom_index_save)."""
        capi.call("zoom_index_save", self.handle, os.fsencode(path), _stream(stream))

    @classmethod
    def load(cls, dictionary: Dictionary, path: str, stream=None) -> "Index":
        """The index of a file written by save, rebuilt on `dictionary` (zoom_index_load)."""
        self = cls.__new__(cls)
        self.dictionary = dictionary
        h = C.c_void_p()
        capi.call("zoom_index_load", dictionary.handle, os.fsencode(path), _stream(stream), C.byref(h))
        self._adopt(h)
        return self

    def params(self, stream=None):
        """The random draws (alpha [L*k][D], beta [L*k]) as numpy float32 (zoom_export_params)."""
        d = self.dictionary.dim
        alpha = np.empty((self.L * self.k, d), np.float32)
        beta = np.empty(self.L * self.k, np.float32)
        capi.call("zoom_export_params", self.handle, alpha.ctypes.data, beta.ctypes.data, _stream(stream))
        return alpha, beta

    def export_keys(self, stream=None):
        keys = np.empty((self.dictionary.n, self.L), np.uint64)
        nb = np.empty(self.L, np.int32)
        capi.call("zoom_index_export", self.handle, keys.ctypes.data, nb.ctypes.data, _stream(stream))
        return keys, nb

    def close(self):
        if getattr(self, "handle", None) and getattr(self.dictionary, "handle", None):
            torch.cuda.synchronize(self.dictionary.ctx.device)
            capi.lib().zoom_index_destroy(self.handle)
        self.handle = None

    def __del__(self):
        if _finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def upscale(index: Index, lr: torch.Tensor, params: UpscaleParams | None = None,
            out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Zoom one LR image (CUDA float32 h x w) by the dictionary's scale."""
    p = params or UpscaleParams()
    _need(lr, torch.float32, "lr")
    h, w = lr.shape
    s = index.dictionary.scale
    if out is None:
        out = torch.empty((s * h, s * w), dtype=torch.float32, device=lr.device)
    _need(out, torch.float32, "out")
    cp = p.c()
    capi.call("zoom_upscale", index.handle, _ptr(lr), h, w, s, C.byref(cp), _ptr(out), _stream(stream))
    return out


def query(index: Index, lr: torch.Tensor, params: UpscaleParams | None = None, stream=None) -> dict:
    """Per-patch steps only: keys, neighbours, distances, weights, means."""
    p = params or UpscaleParams()
    _need(lr, torch.float32, "lr")
    h, w = lr.shape
    P = index.dictionary.patch
    nq = (h - P + 1) * (w - P + 1)
    dev = lr.device
    keys = torch.empty((nq, index.L), dtype=torch.int64, device=dev)
    nbr = torch.empty((nq, p.K), dtype=torch.int32, device=dev)
    dist = torch.empty((nq, p.K), dtype=torch.float32, device=dev)
    wgt = torch.empty((nq, p.K), dtype=torch.float32, device=dev)
    mu = torch.empty(nq, dtype=torch.float32, device=dev)
    bsum = torch.empty(nq, dtype=torch.int32, device=dev)
    cp = p.c()
    capi.call("zoom_query", index.handle, _ptr(lr), h, w, C.byref(cp), _ptr(keys), _ptr(nbr),
              _ptr(dist), _ptr(wgt), _ptr(mu), _ptr(bsum), _stream(stream))
    return {"keys": keys, "nbr": nbr, "dist": dist, "wgt": wgt, "mu": mu, "bucket_sum": bsum}


def reconstruct(index: Index, nbr: torch.Tensor, wgt: torch.Tensor, mu: torch.Tensor, h: int, w: int,
                stream=None) -> torch.Tensor:
    """Eq. 14 blend + overlap average for given neighbours (no back-projection)."""
    _need(nbr, torch.int32, "nbr")
    _need(wgt, torch.float32, "wgt")
    _need(mu, torch.float32, "mu")
    s = index.dictionary.scale
    out = torch.empty((s * h, s * w), dtype=torch.float32, device=nbr.device)
    capi.call("zoom_reconstruct", index.handle, _ptr(nbr), _ptr(wgt), _ptr(mu), h, w, nbr.shape[1],
              _ptr(out), _stream(stream))
    return out


def backproject(ctx: Context, lr: torch.Tensor, hr: torch.Tensor, scale: int,
                params: UpscaleParams | None = None, blur_sigma: float = 0.8, stream=None) -> torch.Tensor:
    """Back-projection iterations on hr (in place) against lr."""
    p = params or UpscaleParams()
    _need(lr, torch.float32, "lr")
    _need(hr, torch.float32, "hr")
    h, w = lr.shape
    if hr.shape != (scale * h, scale * w):
        raise ValueError("hr must be (scale*h, scale*w)")
    degr = capi.Degradation(scale, 1, blur_sigma)
    cp = p.c()
    capi.call("zoom_backproject", ctx.handle, C.byref(degr), _ptr(lr), h, w, C.byref(cp), _ptr(hr),
              _stream(stream))
    return hr


# ---------------------------------------------------------------------------
# differentiation
# ---------------------------------------------------------------------------


def dictionary_hr(dictionary: Dictionary, stream=None) -> torch.Tensor:
    """The HR residual patches R of a dictionary as a CUDA tensor [N][(s*P)^2]."""
    _, _, hr = dictionary.export(stream)
    return torch.from_numpy(hr).cuda(dictionary.ctx.device)


def degrade(ctx: Context, hr: torch.Tensor, scale: int, blur_sigma: float = 0.8, stream=None) -> torch.Tensor:
    """lr = D_s(B hr) (blur + s x s box down-sampling) on the GPU."""
    _need(hr, torch.float32, "hr")
    H, W = hr.shape
    out = torch.empty((H // scale, W // scale), dtype=torch.float32, device=hr.device)
    degr = capi.Degradation(scale, 1, blur_sigma)
    capi.call("zoom_degrade", ctx.handle, C.byref(degr), _ptr(hr), H, W, _ptr(out), _stream(stream))
    return out


def degrade_adjoint(ctx: Context, g_lr: torch.Tensor, scale: int, blur_sigma: float = 0.8,
                    stream=None) -> torch.Tensor:
    """B^T D^T g_lr, the adjoint of `degrade`."""
    _need(g_lr, torch.float32, "g_lr")
    h, w = g_lr.shape
    out = torch.empty((scale * h, scale * w), dtype=torch.float32, device=g_lr.device)
    degr = capi.Degradation(scale, 1, blur_sigma)
    capi.call("zoom_degrade_adjoint", ctx.handle, C.byref(degr), _ptr(g_lr), h, w, _ptr(out), _stream(stream))
    return out


def reconstruct_with(index: Index, hr_dict: torch.Tensor, nbr, wgt, mu, h: int, w: int,
                     stream=None) -> torch.Tensor:
    """Eq. 14 blend + overlap average with a given HR dictionary [N][(s*P)^2]."""
    for t, dt, nm in ((hr_dict, torch.float32, "hr_dict"), (nbr, torch.int32, "nbr"),
                      (wgt, torch.float32, "wgt"), (mu, torch.float32, "mu")):
        _need(t, dt, nm)
    s = index.dictionary.scale
    out = torch.empty((s * h, s * w), dtype=torch.float32, device=nbr.device)
    capi.call("zoom_reconstruct_with", index.handle, _ptr(hr_dict), hr_dict.shape[1], _ptr(nbr), _ptr(wgt),
              _ptr(mu), h, w, nbr.shape[1], _ptr(out), _stream(stream))
    return out


def reconstruct_adjoint(index: Index, nbr, wgt, h: int, w: int, grad_hr: torch.Tensor,
                        want_mu: bool = False, stream=None):
    """dL/dR (and optionally dL/dmu) from dL/d(HR image), neighbours fixed."""
    _need(grad_hr, torch.float32, "grad_hr")
    d = index.dictionary
    ph2 = (d.scale * d.patch) ** 2
    gd = torch.empty((d.n, ph2), dtype=torch.float32, device=nbr.device)
    gmu = torch.empty(nbr.shape[0], dtype=torch.float32, device=nbr.device) if want_mu else None
    capi.call("zoom_reconstruct_adjoint", index.handle, _ptr(nbr), _ptr(wgt), h, w, nbr.shape[1],
              _ptr(grad_hr), _ptr(gd), ph2, _ptr(gmu), _stream(stream))
    return gd, gmu


class ReconstructFunction(torch.autograd.Function):
    """x = overlap average of mu_n + sum_m w_nm R[nbr_nm] as a differentiable
    function of the HR dictionary R (neighbours and weights fixed); the
    backward is the library's adjoint kernel."""

    @staticmethod
    def forward(fctx, hr_dict, index, nbr, wgt, mu, h, w):
        fctx.save_for_backward(nbr, wgt)
        fctx.index, fctx.hw = index, (h, w)
        return reconstruct_with(index, hr_dict.contiguous(), nbr, wgt, mu, h, w)

    @staticmethod
    def backward(fctx, g):
        nbr, wgt = fctx.saved_tensors
        gd, _ = reconstruct_adjoint(fctx.index, nbr, wgt, *fctx.hw, g.contiguous())
        return gd, None, None, None, None, None, None


class DegradeFunction(torch.autograd.Function):
    """lr = D_s(B x) as a differentiable function of x; backward B^T D^T."""

    @staticmethod
    def forward(fctx, x, ctx, scale, blur_sigma):
        fctx.ctx, fctx.scale, fctx.sigma = ctx, scale, blur_sigma
        return degrade(ctx, x.contiguous(), scale, blur_sigma)

    @staticmethod
    def backward(fctx, g):
        return degrade_adjoint(fctx.ctx, g.contiguous(), fctx.scale, fctx.sigma), None, None, None


def map_energy_grads(index: Index, lr: torch.Tensor, nbr: torch.Tensor, wgt: torch.Tensor | None = None,
                     lam: float = 0.1, reg_rel: float = 1e-3, stream=None) -> dict:
    """MAP energy E(R) = ||D B x - y||^2 + lam * overlap prior and its
    gradients dE/dx (data term at x) and dE/dR, neighbours fixed (zoom_backward)."""
    _need(lr, torch.float32, "lr")
    _need(nbr, torch.int32, "nbr")
    if wgt is not None:
        _need(wgt, torch.float32, "wgt")
    d = index.dictionary
    h, w = lr.shape
    s, ph2 = d.scale, (d.scale * d.patch) ** 2
    gx = torch.empty((s * h, s * w), dtype=torch.float32, device=lr.device)
    gd = torch.empty((d.n, ph2), dtype=torch.float32, device=lr.device)
    x = torch.empty((s * h, s * w), dtype=torch.float32, device=lr.device)
    e = C.c_double()
    capi.call("zoom_backward", index.handle, _ptr(lr), h, w, _ptr(nbr), _ptr(wgt), nbr.shape[1], reg_rel, lam,
              _ptr(gx), _ptr(gd), ph2, _ptr(x), C.byref(e), _stream(stream))
    return {"energy": e.value, "grad_x": gx, "grad_dict": gd, "hr": x}


# ---------------------------------------------------------------------------
# seeded draws (host; the library's generator)
# ---------------------------------------------------------------------------


def lsh_draws(L: int, k: int, dim: int, w: float, seed: int, proj_dist: int = 0):
    """The projections and offsets zoom_build_index draws from a seed
    (zoom_lsh_draws): alpha float32 [L*k][dim], beta float32 [L*k]."""
    prm = capi.LshParams(L, k, w, 1, 0, proj_dist, int(seed))
    a = np.empty((L * k, dim), np.float32)
    b = np.empty(L * k, np.float32)
    capi.call("zoom_lsh_draws", C.byref(prm), dim, a.ctypes.data, b.ctypes.data)
    return a, b


def sample_positions(seed: int, lr_sizes, patch: int, n_pairs: int) -> np.ndarray:
    """Dictionary positions drawn from a seed (zoom_sample_positions): int32
    [n_pairs][3] (image, LR row, LR col) over the LR images of lr_sizes."""
    n = len(lr_sizes)
    hs = (C.c_int32 * n)(*[int(h) for h, _ in lr_sizes])
    ws = (C.c_int32 * n)(*[int(w) for _, w in lr_sizes])
    out = np.empty((n_pairs, 3), np.int32)
    capi.call("zoom_sample_positions", int(seed), n, hs, ws, patch, n_pairs, out.ctypes.data)
    return out


# ---------------------------------------------------------------------------
# batched zoom
# ---------------------------------------------------------------------------


def upscale_batch(indexes, lrs, params: UpscaleParams | None = None, outs=None, want_latency: bool = False,
                  stream=None):
    """Zoom many LR images (CUDA float32, any sizes) in one call.  `lrs` is a
    list of (scale, lr) pairs (or plain tensors, all at the scale of
    indexes[0]); each image uses the index whose dictionary has its scale.
    Returns (outputs, per-image device ms from the batch start, or None)."""
    p = params or UpscaleParams()
    if isinstance(lrs[0], tuple):
        scales = [s for s, _ in lrs]
        lrs = [x for _, x in lrs]
    else:
        scales = [indexes[0].dictionary.scale] * len(lrs)
    by_scale = {ix.dictionary.scale: ix for ix in indexes}
    if outs is None:
        outs = [torch.empty((s * x.shape[0], s * x.shape[1]), dtype=torch.float32, device=x.device)
                for s, x in zip(scales, lrs)]
    for x in lrs:
        _need(x, torch.float32, "lr")
    n = len(lrs)
    ix_arr = (C.c_void_p * len(indexes))(*[ix.handle.value for ix in indexes])
    lr_arr = (C.c_void_p * n)(*[x.data_ptr() for x in lrs])
    hr_arr = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    hs = (C.c_int32 * n)(*[x.shape[0] for x in lrs])
    ws = (C.c_int32 * n)(*[x.shape[1] for x in lrs])
    ss = (C.c_int32 * n)(*scales)
    lat = (C.c_float * n)() if want_latency else None
    if any(s not in by_scale for s in scales):
        raise ValueError("no index for some image's scale")
    cp = p.c()
    capi.call("zoom_upscale_batch", ix_arr, len(indexes), n, lr_arr, hs, ws, ss, C.byref(cp), hr_arr,
              _stream(stream), lat)
    return outs, (list(lat) if want_latency else None)


def batch_release(ctx: Context) -> None:
    capi.call("zoom_batch_release", ctx.handle)
