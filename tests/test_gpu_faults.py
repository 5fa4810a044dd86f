"""Failure paths, exercised without a GPU fault:
  * a bounded wait inside the tensor-core filter that runs out (the
    filter's CTAs withhold their accumulator releases, a flag nothing else
    sets: zoom_set_fault_injection) is reported as ZOOM_ERR_TIMEOUT by
    zoom_sync_status, and the next call on the same context gives the SIMT
    scan's neighbours again;
  * the lists of a filter that gave up are never written; the rerank
    reads them (random bytes, from an allocator that fills every block)
    without following a chunk number outside the dictionary;
  * an allocation the context's allocator refuses makes the call return
    ZOOM_ERR_OOM with every allocation it made freed (the counts balance),
    except the blended-patch scratch of the overlap average, whose refusal
    falls back to the one-pass average with the same bits."""
import ctypes as C

import numpy as np
import pytest

from tests import gpu_cases as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


class CountingAllocator:
    """Device memory from PyTorch's caching allocator, with every live
    allocation recorded; fails the fail_at-th call (1-based) and every
    request of refuse_bytes bytes."""

    def __init__(self):
        self.live = {}
        self.calls = 0
        self.fail_at = None
        self.refuse_bytes = None
        self.refused = 0

    def alloc(self, nbytes, stream, user):
        self.calls += 1
        if self.calls == self.fail_at or nbytes == self.refuse_bytes:
            self.refused += 1
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), 0, int(stream or 0))
        self.live[p] = int(nbytes)
        return p

    def free(self, ptr, nbytes, stream, user):
        assert self.live.pop(ptr) == nbytes
        torch.cuda.caching_allocator_delete(ptr)


class GarbageAllocator:
    """Device memory as PyTorch byte tensors filled with seeded random bytes:
    whatever a kernel reads without having written it first is garbage, the
    same garbage in every run."""

    def __init__(self, seed: int = 5):
        self.live = {}
        self.gen = torch.Generator(device="cuda")
        self.gen.manual_seed(seed)

    def alloc(self, nbytes, stream, user):
        t = torch.randint(0, 256, (int(nbytes),), dtype=torch.uint8, device="cuda", generator=self.gen)
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def free(self, ptr, nbytes, stream, user):
        self.live.pop(ptr)


@pytest.fixture(scope="module")
def small():
    from paper_1004_3980_gb300 import build
    build.build()
    case = G.small_case()
    ctx, d, ix = G.gpu_build(case)
    return case, ctx, d, ix


@pytest.mark.parametrize("prm", [dict(search=2), dict(precision=1, rerank_mult=2)], ids=["exact", "bf16"])
def test_filter_wait_timeout_is_reported_and_the_context_recovers(small, prm):
    import paper_1004_3980_gb300 as Z
    from paper_1004_3980_gb300.capi import ZoomError
    case, ctx, d, ix = small
    wl = case.wl
    lr = torch.from_numpy(case.lr).cuda()
    ref = Z.query(ix, lr, G.params(wl, search=1))
    ctx.sync_status()
    ctx.set_fault_injection(1, 20_000_000)    # waits give up after 20 ms
    try:
        Z.query(ix, lr, G.params(wl, **prm))
        with pytest.raises(ZoomError, match="TIMEOUT"):
            ctx.sync_status()
    finally:
        ctx.set_fault_injection(0, 0)
    ctx.sync_status()                          # read and cleared: the context is usable
    r = Z.query(ix, lr, G.params(wl, **prm))
    ctx.sync_status()
    if prm.get("precision", 0) == 0:
        assert torch.equal(r["nbr"], ref["nbr"]) and torch.equal(r["dist"], ref["dist"])
    else:
        hits = sum((r["nbr"] == ref["nbr"][:, m:m + 1]).any(dim=1).int() for m in range(wl.K))
        assert float(hits.double().mean()) / wl.K >= 0.99


@pytest.mark.parametrize("prm", [dict(search=2), dict(precision=1, rerank_mult=2)], ids=["exact", "bf16"])
def test_a_filter_that_gave_up_leaves_lists_the_rerank_never_follows(small, prm):
    # The filter's waits run out before it writes any list, so the chunk
    # lists the rerank reads are the random bytes of the scratch memory:
    # chunk numbers outside the dictionary must count as "none" (never an
    # address), and every neighbour returned is still a dictionary entry.
    import paper_1004_3980_gb300 as Z
    from paper_1004_3980_gb300.capi import ZoomError
    case = small[0]
    wl = case.wl
    A = GarbageAllocator()
    ctx, d, ix = G.gpu_build(case, Z.Context(0, allocator=A))
    lr = torch.from_numpy(case.lr).cuda()
    ref = Z.query(ix, lr, G.params(wl, search=1))
    ctx.sync_status()
    ctx.set_fault_injection(1, 20_000_000)
    try:
        r = Z.query(ix, lr, G.params(wl, **prm))
        with pytest.raises(ZoomError, match="TIMEOUT"):
            ctx.sync_status()
    finally:
        ctx.set_fault_injection(0, 0)
    ctx.sync_status()
    n = len(case.positions)
    assert int(r["nbr"].min()) >= 0 and int(r["nbr"].max()) < n
    r = Z.query(ix, lr, G.params(wl, **prm))
    ctx.sync_status()
    if prm.get("precision", 0) == 0:
        assert torch.equal(r["nbr"], ref["nbr"]) and torch.equal(r["dist"], ref["dist"])


def test_fault_injection_rejects_bad_arguments(small):
    from paper_1004_3980_gb300.capi import ZoomError
    ctx = small[1]
    with pytest.raises(ZoomError, match="INVALID_ARG"):
        ctx.set_fault_injection(2, 0)
    with pytest.raises(ZoomError, match="INVALID_ARG"):
        ctx.set_fault_injection(1, 61_000_000_000)
    ctx.set_fault_injection(0, 0)


def test_refused_allocations_return_oom_and_free_everything(small):
    import paper_1004_3980_gb300 as Z
    from paper_1004_3980_gb300 import capi
    case = small[0]
    wl = case.wl
    A = CountingAllocator()
    ctx = Z.Context(0, allocator=A)
    lib = capi.lib()
    # the dictionary and index builds: refuse each of their allocations in turn
    for k in range(1, 10):
        A.calls, A.fail_at = 0, k
        try:
            G.gpu_build(case, ctx)
            built = True
        except capi.ZoomError as e:
            assert "OOM" in str(e)
            built = False
        torch.cuda.synchronize()
        A.fail_at = None
        if built:
            break
        assert not A.live, "a refused build left memory behind"
    assert built and k > 1
    _, d, ix = G.gpu_build(case, ctx)
    held = dict(A.live)                        # the dictionary's and the index's arrays
    lr = torch.from_numpy(case.lr).cuda()
    out = torch.empty((wl.scale * wl.lr_h, wl.scale * wl.lr_w), device="cuda")
    p = G.params(wl).c()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def upscale():
        return lib.zoom_upscale(ix.handle, C.c_void_p(lr.data_ptr()), wl.lr_h, wl.lr_w, wl.scale, C.byref(p),
                                C.c_void_p(out.data_ptr()), stream)

    A.calls = 0
    assert upscale() == 0
    torch.cuda.synchronize()
    n_alloc = A.calls
    ref = out.clone()
    assert A.live == held and n_alloc >= 2
    codes = []
    for k in range(1, n_alloc + 1):
        A.calls, A.fail_at = 0, k
        out.zero_()
        rc = upscale()
        torch.cuda.synchronize()
        A.fail_at = None
        codes.append(rc)
        assert rc in (0, 2), lib.zoom_last_error()
        if rc == 0:                            # only the optional blended-patch scratch may be refused
            assert torch.equal(out, ref)
        assert A.live == held, f"allocation {k} refused: memory left behind"
    assert codes.count(2) >= 1 and codes[-1] == 0
    ctx.sync_status()


def test_refused_patch_scratch_gives_the_same_bits(small):
    # zoom_upscale and zoom_reconstruct without room for the blended patches
    # (a request of n_q (s P)^2 floats refused): the one-pass overlap average
    import paper_1004_3980_gb300 as Z
    case = small[0]
    wl = case.wl
    A = CountingAllocator()
    ctx = Z.Context(0, allocator=A)
    _, d, ix = G.gpu_build(case, ctx)
    lr = torch.from_numpy(case.lr).cuda()
    nq = (wl.lr_h - wl.patch + 1) * (wl.lr_w - wl.patch + 1)
    q = Z.query(ix, lr, G.params(wl))
    ref_up = Z.upscale(ix, lr, G.params(wl))
    ref_rc = Z.reconstruct(ix, q["nbr"], q["wgt"], q["mu"], wl.lr_h, wl.lr_w)
    torch.cuda.synchronize()
    A.refuse_bytes = nq * (wl.scale * wl.patch) ** 2 * 4
    A.refused = 0
    up = Z.upscale(ix, lr, G.params(wl))
    rc = Z.reconstruct(ix, q["nbr"], q["wgt"], q["mu"], wl.lr_h, wl.lr_w)
    torch.cuda.synchronize()
    A.refuse_bytes = None
    assert A.refused == 2
    assert torch.equal(up, ref_up) and torch.equal(rc, ref_rc)
    assert np.isfinite(up.cpu().numpy()).all()
