"""The allocation-free history slice against the context entry point.

kbe_history_slice_noalloc serves callers that cannot allocate device memory
(code inside another framework's memory pool or allocator hooks, where a
nested cudaMalloc would re-enter the allocator or escape its accounting,
and hosts that only hand over fixed buffers).  It keeps its scratch in a
static device array, so this test checks that calls in a row, each reusing
the array left by the one before (a larger row on another grid after a
smaller one included), match the context path (kbe_history_slice) through
the C ABI; that the device's free memory does not change across the calls
that follow the first; and that sizes beyond the array are rejected on the
host.

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


def _prepare(kbe, M, n_t, seed, n):
    """Inputs of row n on a seeded grid and the context path's slice."""
    t, order, h, U, L, R, torch = _case(M, n_t, seed)
    ctx = kbe.Context(M, n_t)
    ctx.set_grid(t, order)
    ctx.set_model(h, U, W.site_potential(M), None)
    Sl = torch.zeros((n_t, M, M), dtype=torch.complex128, device="cuda")
    Sg = torch.zeros_like(Sl)
    ctx.selfenergy_slice(n, L, R, Sl, Sg)
    Sl_n, Sg_n = Sl[: n + 1].contiguous(), Sg[: n + 1].contiguous()
    ref = torch.zeros((2, n + 1, M, M), dtype=torch.complex128, device="cuda")
    ctx.history_slice(n, L, R, Sl_n, Sg_n, ref)
    ctx.sync_status()
    ctx.close()
    out = torch.full((2, n + 1, M, M), float("nan"), dtype=torch.complex128, device="cuda")
    return dict(M=M, n=n, t=t, order=order, L=L, R=R, Sl=Sl_n, Sg=Sg_n, ref=ref, out=out)


def _noalloc(kbe, c):
    """One allocation-free call into the preallocated output (no torch work)."""
    import torch
    st = kbe.lib().kbe_history_slice_noalloc(c["M"], c["n"], _np(c["t"]), _np(c["order"]), len(c["t"]),
                                             _ptr(c["L"]), _ptr(c["R"]), _ptr(c["Sl"]), _ptr(c["Sg"]),
                                             _ptr(c["out"]),
                                             ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == kbe.KBE_OK, kbe.lib().kbe_last_error(None)
    torch.cuda.synchronize()


def _rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("M,n_t,rows", [(8, 300, (299, 150)), (3, 50, (49, 0))])
def test_noalloc_matches_context_path_twice(kbe, M, n_t, rows):
    cases = [_prepare(kbe, M, n_t, 11 + M, n) for n in rows]
    for c in cases:  # two calls in a row share the static scratch
        _noalloc(kbe, c)
        assert _rel(c["out"], c["ref"]) < TOL, (M, c["n"], _rel(c["out"], c["ref"]))


def test_noalloc_larger_row_on_another_grid_after_a_smaller_one(kbe):
    """A small row, then a larger row on a different seeded grid and orbital
    count, then the small one again: each result matches the context path,
    whatever the earlier call left in the shared array.  The device's free
    memory is the same after every call that follows the first."""
    import torch
    cases = [_prepare(kbe, 4, 120, 3, 40), _prepare(kbe, 6, 400, 7, 399), _prepare(kbe, 4, 120, 3, 40)]
    torch.cuda.synchronize()
    _noalloc(kbe, cases[0])  # the first call may look up the array's device address
    free0 = torch.cuda.mem_get_info()[0]
    for c in cases:
        c["out"].fill_(float("nan"))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for c in cases:
        _noalloc(kbe, c)
        assert torch.cuda.mem_get_info()[0] == free0, "the call changed the device's free memory"
        assert _rel(c["out"], c["ref"]) < TOL, (c["M"], c["n"], _rel(c["out"], c["ref"]))


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
