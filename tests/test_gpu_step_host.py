"""GPU tests of kbe_step_host: the KBE step with its history and stored
right-hand sides in host memory, uploaded in row chunks that overlap the
first history slice.

The step must give bitwise the rows of kbe_step on the same data (the same
kernels contract the same entries, only in column ranges), and so match the
oracle's step at the FP64 tolerance."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def kbe():
    import torch
    from paper_2405_08737_gb300 import build as B
    B.build()
    import paper_2405_08737_gb300 as K
    torch.cuda.set_device(0)
    return K


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _restart(kbe, name, n_t, seed):
    """A context and run at row n = n_t - 1 restarted from the
    non-interacting history with its exact right-hand sides."""
    cfg = W.CONFIGS[name]
    t, order = W.grid(cfg["n_t"], cfg["dt0"], cfg["sig"], seed)
    t, order = t[:n_t], order[:n_t]
    h, U, v, pulse = W.build_model(cfg, seed)
    if pulse is not None:
        pulse = dict(pulse, t0=t[n_t - 3], sigma=0.2)
    M, n = cfg["M"], n_t - 1
    L, R = W.free_triangles(h, W.half_filled_rho(h), t, n_rows=n)
    rows = oracle.f_rows_needed(order, n, n_t)
    Fr = W.free_rhs_rows(h, L, R, rows)
    ctx = kbe.Context(M, n_t)
    ctx.set_grid(t, order)
    ctx.set_model(h, U, v, pulse)
    return ctx, (t, order, h, U, v, pulse), (L, R, rows, Fr)


def _load(kbe, run, L, R, rows, Fr):
    import torch
    run.L.zero_()
    run.R.zero_()
    run.F.zero_()
    run.L[: len(L)].copy_(torch.as_tensor(L, device="cuda"))
    run.R[: len(R)].copy_(torch.as_tensor(R, device="cuda"))
    for j in rows:
        run.F[j % kbe.KBE_RING_ROWS, :, : j + 1].copy_(torch.as_tensor(Fr[j], device="cuda"))


@pytest.mark.parametrize("name,n_t,precision", [("chain_m8_n1024", 90, "fp64"), ("dimer_m2_n64", 64, "fp64"),
                                                ("chain_m8_n1024", 70, "split"), ("goe_m32_n1024", 24, "fp64")])
def test_step_host_equals_step(kbe, name, n_t, precision):
    import torch
    ctx, model, (L, R, rows, Fr) = _restart(kbe, name, n_t, 3)
    n, M = n_t - 1, ctx.M
    # device path
    run = kbe.Run(ctx)
    _load(kbe, run, L, R, rows, Fr)
    L_h = run.L.cpu().pin_memory()
    R_h = run.R.cpu().pin_memory()
    F_h = run.F.cpu().pin_memory()
    run.step(n, P=2, precision=precision)
    ctx.sync_status()
    p = W.tri_index(n, 0)
    ref_L, ref_R = run.L[p:p + n + 1].cpu().numpy(), run.R[p:p + n + 1].cpu().numpy()
    ref_I = run.I[:, : n + 1].cpu().numpy()
    # host path into zeroed device buffers of a second run on the same context
    run2 = kbe.Run(ctx)
    out_L = torch.empty((n + 1, M, M), dtype=torch.complex128).pin_memory()
    out_R = torch.empty_like(out_L).pin_memory()
    run2.step_host(n, L_h, R_h, F_h, out_L, out_R, P=2, precision=precision)
    ctx.sync_status()
    assert np.array_equal(out_L.numpy(), ref_L) and np.array_equal(out_R.numpy(), ref_R)
    assert np.array_equal(run2.I[:, : n + 1].cpu().numpy(), ref_I)
    # the uploaded history is the host's, and nothing above row n was written
    assert np.array_equal(run2.L[:p].cpu().numpy(), L_h[:p].numpy())
    assert np.array_equal(run2.R[:p].cpu().numpy(), R_h[:p].numpy())
    assert not run2.L[p + n + 1:].abs().any()
    if precision == "fp64":
        t, order, h, U, v, pulse = model
        Lf = np.zeros((W.tri_size(n_t), M, M), np.complex128)
        Rf = np.zeros_like(Lf)
        Lf[: len(L)], Rf[: len(R)] = L, R
        Lo, Ro, _ = oracle.run(t, order, h, U, v, pulse, 2, Lf, Rf, Fr, n, n_t,
                               nthreads=oracle.threads_available())
        assert _rel(out_L.numpy(), Lo[p:p + n + 1]) < TOL
        assert _rel(out_R.numpy(), Ro[p:p + n + 1]) < TOL
    ctx.close()


def test_step_host_repeated_and_after_device_steps(kbe):
    """Back-to-back host steps on one stream, between device steps on the
    same buffers: each upload waits for the work queued before it."""
    import torch
    ctx, _, (L, R, rows, Fr) = _restart(kbe, "chain_m8_n1024", 60, 5)
    n, M = 59, ctx.M
    run = kbe.Run(ctx)
    _load(kbe, run, L, R, rows, Fr)
    L_h, R_h, F_h = run.L.cpu().pin_memory(), run.R.cpu().pin_memory(), run.F.cpu().pin_memory()
    outs = [torch.empty((n + 1, M, M), dtype=torch.complex128).pin_memory() for _ in range(6)]
    for k in range(3):
        run.step(n, P=2)  # device step on the same buffers, then a host step that rewrites rows < n
        run.step_host(n, L_h, R_h, F_h, outs[2 * k], outs[2 * k + 1], P=2)
    ctx.sync_status()
    for k in range(1, 3):
        assert np.array_equal(outs[2 * k].numpy(), outs[0].numpy())
        assert np.array_equal(outs[2 * k + 1].numpy(), outs[1].numpy())
    ctx.close()


def test_step_host_null_host_pointer_is_einval(kbe):
    ctx, _, (L, R, rows, Fr) = _restart(kbe, "dimer_m2_n64", 12, 1)
    run = kbe.Run(ctx)
    vp = ctypes.c_void_p
    st = kbe.lib().kbe_step_host(ctx._h, 11, 2, 0, None, None, None, ctx._dev(run.L), ctx._dev(run.R),
                                 ctx._dev(run.Sl), ctx._dev(run.Sg), ctx._dev(run.I), ctx._dev(run.F), None, None,
                                 vp(0))
    assert st == kbe.KBE_EINVAL
    ctx.close()


@pytest.mark.parametrize("mode", ["df64", "dense"])
def test_step_host_other_paths_equal_step(kbe, mode):
    """A step that contracts with another kernel (KBE_DF64, which waits for
    the whole upload before the first sweep) or forms another self-energy
    (dense U, pipelined): kbe_step_host still gives kbe_step's rows."""
    import torch
    ctx, _, (L, R, rows, Fr) = _restart(kbe, "chain_m8_n1024", 50, 7)
    n, M = 49, ctx.M
    precision = "df64" if mode == "df64" else "fp64"
    if mode == "dense":
        ctx.set_interaction(W.coulomb_tensor(M, 7, U=1.0))
    run = kbe.Run(ctx)
    _load(kbe, run, L, R, rows, Fr)
    L_h, R_h, F_h = run.L.cpu().pin_memory(), run.R.cpu().pin_memory(), run.F.cpu().pin_memory()
    run.step(n, P=2, precision=precision)
    ctx.sync_status()
    p = W.tri_index(n, 0)
    ref_L, ref_R = run.L[p:p + n + 1].cpu().numpy(), run.R[p:p + n + 1].cpu().numpy()
    run2 = kbe.Run(ctx)
    out_L = torch.empty((n + 1, M, M), dtype=torch.complex128).pin_memory()
    out_R = torch.empty_like(out_L).pin_memory()
    run2.step_host(n, L_h, R_h, F_h, out_L, out_R, P=2, precision=precision)
    ctx.sync_status()
    assert np.array_equal(out_L.numpy(), ref_L) and np.array_equal(out_R.numpy(), ref_R)
    ctx.close()
