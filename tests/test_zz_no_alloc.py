"""zoom_backproject_noalloc: the back-projection entry point for callers that
cannot allocate device memory (it works from a fixed static scratch array
inside the library).  Its output must match zoom_backproject, the
allocating entry point, on two calls in a row with different inputs, and
requests larger than its scratch must be refused.

This file is collected last, so that a run stopping at the first failure
has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import synth_inputs as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_backproject_matches_allocating_entry_point():
    from paper_1004_3980_gb300 import build
    build.build()
    import paper_1004_3980_gb300 as Z
    from paper_1004_3980_gb300 import capi
    lib = capi.lib()
    ctx = Z.Context(0)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (s, h, w, iters) in enumerate([(2, 40, 52, 3), (3, 33, 47, 4)]):
        y = S.make_image(300 + call, h, w)
        x0 = (np.kron(y, np.ones((s, s))) + 0.02 * S.make_image(400 + call, s * h, s * w)).astype(np.float32)
        p = Z.UpscaleParams(bp_iters=iters)
        y_t = torch.from_numpy(y).cuda()
        ref = torch.from_numpy(x0).cuda()
        Z.backproject(ctx, y_t, ref, s, p)
        out = torch.from_numpy(x0).cuda()
        degr = capi.Degradation(s, 1, 0.8)
        prm = p.c()
        rc = lib.zoom_backproject_noalloc(0, C.byref(degr), C.c_void_p(y_t.data_ptr()), h, w, C.byref(prm),
                                          C.c_void_p(out.data_ptr()), stream)
        assert rc == 0, lib.zoom_last_error()
        torch.cuda.synchronize()
        # same kernels in the same order: the tolerance of the back-projection
        # parity tests (1e-3 on the [0, 1] scale) is met with room to spare
        assert torch.max(torch.abs(out - ref)).item() <= 1e-6
        assert torch.max(torch.abs(out - torch.from_numpy(x0).cuda())).item() > 0


def test_noalloc_refuses_images_beyond_its_scratch():
    from paper_1004_3980_gb300 import capi
    import paper_1004_3980_gb300 as Z
    lib = capi.lib()
    h = w = 1024                               # 2x: 4 Mi HR floats > the 2 Mi maximum
    y = torch.zeros((h, w), device="cuda")
    out = torch.zeros((2 * h, 2 * w), device="cuda")
    degr = capi.Degradation(2, 1, 0.8)
    prm = Z.UpscaleParams(bp_iters=1).c()
    rc = lib.zoom_backproject_noalloc(0, C.byref(degr), C.c_void_p(y.data_ptr()), h, w, C.byref(prm),
                                      C.c_void_p(out.data_ptr()), None)
    assert rc == 1
    assert b"too large" in lib.zoom_last_error()


@pytest.mark.parametrize("h,w,accepted", [
    (1024, 1024, True),    # scale 1: 1 Mi HR floats + 1 Mi LR floats = the maximum exactly
    (1023, 1025, True),    # 1,048,575 HR floats round up to 1 Mi before the LR image: 2 Mi - 1
    (1024, 1025, False),   # one column more: 2 Mi + 2048
])
def test_noalloc_scratch_limit_is_exact(h, w, accepted):
    # the size check at its boundary: round_up(s^2 h w, 64) + h w floats
    # against ZOOM_NOALLOC_SCRATCH_FLOATS = 2 Mi; accepted sizes give the
    # allocating entry point's output
    from paper_1004_3980_gb300 import capi
    import paper_1004_3980_gb300 as Z
    lib = capi.lib()
    need = (h * w + 63) // 64 * 64 + h * w
    assert (need <= 2 * 1024 * 1024) == accepted
    y = torch.from_numpy(S.make_image(77, h, w)).cuda()
    x0 = torch.from_numpy(S.make_image(78, h, w)).cuda()
    p = Z.UpscaleParams(bp_iters=2)
    out = x0.clone()
    degr = capi.Degradation(1, 1, 0.8)
    prm = p.c()
    rc = lib.zoom_backproject_noalloc(0, C.byref(degr), C.c_void_p(y.data_ptr()), h, w, C.byref(prm),
                                      C.c_void_p(out.data_ptr()), None)
    if not accepted:
        assert rc == 1 and b"too large" in lib.zoom_last_error()
        return
    assert rc == 0, lib.zoom_last_error()
    ref = x0.clone()
    Z.backproject(Z.Context(0), y, ref, 1, p)
    torch.cuda.synchronize()
    assert torch.max(torch.abs(out - ref)).item() <= 1e-6
