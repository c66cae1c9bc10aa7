"""The allocation-free history slice against the context entry point.

kbe_history_slice_noalloc serves callers that cannot allocate device memory
(code inside another framework's memory pool or allocator hooks, graph
builders that may not allocate while recording, hosts that only hand over
fixed buffers).  It keeps its scratch in a static device array, so this
test checks that two calls in a row, the second reusing the array left by
the first, both match the context path (kbe_history_slice) through the
C ABI, and that sizes beyond the array are rejected on the host.

The file name sorts last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12  # the FP64 path's parity tolerance


@pytest.fixture(scope="module")
def kbe():
    import torch
    from paper_2405_08737_gb300 import build as B
    B.build()
    import paper_2405_08737_gb300 as K
    lib = K.lib()
    vp, i = ctypes.c_void_p, ctypes.c_int
    lib.kbe_history_slice_noalloc.argtypes = [i, i, vp, vp, i, vp, vp, vp, vp, vp, vp]
    torch.cuda.set_device(0)
    return K


def _ptr(x):
    return ctypes.c_void_p(x.data_ptr())


def _np(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _case(M, n_t, seed):
    import torch
    t, order = W.grid(n_t, 0.05, 0.4, seed)
    h = W.goe_h(M, seed)
    rho0 = W.half_filled_rho(h)
    L, R = W.free_triangles_torch(h, rho0, t, n_t, "cuda")
    U = np.linspace(0.5, 1.5, M)
    return t, order.astype(np.int32), h, U, L, R, torch


def _context_slice(kbe, ctx, n, L, R, Sl, Sg):
    import torch
    out = torch.zeros((2, n + 1, ctx.M, ctx.M), dtype=torch.complex128, device="cuda")
    ctx.history_slice(n, L, R, Sl[: n + 1].contiguous(), Sg[: n + 1].contiguous(), out)
    ctx.sync_status()
    return out


def _noalloc_slice(kbe, M, n, t, order, L, R, Sl, Sg):
    import torch
    out = torch.full((2, n + 1, M, M), float("nan"), dtype=torch.complex128, device="cuda")
    st = kbe.lib().kbe_history_slice_noalloc(M, n, _np(t), _np(order), len(t), _ptr(L), _ptr(R),
                                             _ptr(Sl), _ptr(Sg), _ptr(out),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == kbe.KBE_OK, kbe.lib().kbe_last_error(None)
    torch.cuda.synchronize()
    return out


def _rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("M,n_t,rows", [(8, 300, (299, 150)), (3, 50, (49, 0))])
def test_noalloc_matches_context_path_twice(kbe, M, n_t, rows):
    t, order, h, U, L, R, torch = _case(M, n_t, 11 + M)
    ctx = kbe.Context(M, n_t)
    ctx.set_grid(t, order)
    ctx.set_model(h, U, W.site_potential(M), None)
    Sl = torch.zeros((n_t, M, M), dtype=torch.complex128, device="cuda")
    Sg = torch.zeros_like(Sl)
    for n in rows:  # two calls in a row share the static scratch
        ctx.selfenergy_slice(n, L, R, Sl, Sg)
        ref = _context_slice(kbe, ctx, n, L, R, Sl, Sg)
        got = _noalloc_slice(kbe, M, n, t, order, L, R, Sl[: n + 1].contiguous(), Sg[: n + 1].contiguous())
        assert _rel(got, ref) < TOL, (M, n, _rel(got, ref))
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(kbe):
    import torch
    lib = kbe.lib()
    dummy = torch.zeros(16, dtype=torch.complex128, device="cuda")
    p = _ptr(dummy)
    t, order = W.grid(9000, 0.01, 0.3, 0)
    order = order.astype(np.int32)
    st = lib.kbe_history_slice_noalloc(4, 10, _np(t), _np(order), 9000, p, p, p, p, p, None)
    assert st == kbe.KBE_EINVAL
    assert b"8192" in lib.kbe_last_error(None)
    t2, o2 = t[:500].copy(), order[:500].copy()
    st = lib.kbe_history_slice_noalloc(64, 400, _np(t2), _np(o2), 500, p, p, p, p, p, None)
    assert st == kbe.KBE_EINVAL
    assert b"scratch" in lib.kbe_last_error(None)
