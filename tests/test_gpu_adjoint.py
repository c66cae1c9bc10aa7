"""GPU checks of the reverse-mode (adjoint) kernels through the C ABI.

The history slice is bilinear in the self-energy row and in the rows of
G, so its vector-Jacobian product is checked by the identity
  Re <dI, I(dS; G)> = Re <dS_bar, dS>   and
  Re <dI, I(S; G + dG) - I(S; G)> = Re <dL_bar, dL> + Re <dR_bar, dR>
with I evaluated by the oracle and random directions (a wrong adjoint
fails it with probability one).  The self-energy is a cubic polynomial in
(G, conj G) and quadratic in U, so two central differences of the oracle
with Richardson's combination give its exact directional derivative.
The window gradient is compared with the oracle's forward-mode (dual
number) derivative and with central finite differences (h = 1e-5)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kbe():
    import torch
    from paper_2405_08737_gb300 import build as B
    B.build()
    import paper_2405_08737_gb300 as K
    torch.cuda.set_device(0)
    return K


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def _inner(a, b):
    """Re sum conj(a) b"""
    return float(np.real(np.vdot(np.asarray(a).ravel(), np.asarray(b).ravel())))


def _rss(a, b):
    """Root-sum-square of the terms of Re <a, b>: the size of an inner product
    of random directions, against which its rounding is measured."""
    return float(np.linalg.norm(np.real(np.conj(np.asarray(a)) * np.asarray(b))))


def _oracle_vjp(t, order, n, L, R, Sl, Sg, dI, row_lo):
    """The exact vector-Jacobian product of the oracle's slice, written out
    as the transpose of its real-linear maps.  The slice is linear in the
    self-energy row at fixed G and linear in (L, R) at fixed Sigma (both
    terms of Eq. KBE2 are products of one Sigma factor and one G factor), so
    the image of each real basis direction e is the oracle's slice with e in
    place of that argument and the other one kept; the cotangent of the
    coordinate is Re <dI, slice(e)> (PyTorch convention: zbar = dF/dRe z +
    i dF/dIm z).  R(r,r) = -i 1 is fixed and gets none."""
    base = W.tri_size(row_lo)
    zL, zS = np.zeros_like(L), np.zeros_like(Sl)

    def pull(fn, shape, skip=()):
        out = np.zeros(shape, np.complex128)
        flat = out.reshape(-1)
        per = int(np.prod(shape[1:]))
        for j in range(flat.size):
            if j // per in skip:
                continue
            for unit, to in ((1.0, 1.0), (1j, 1j)):
                e = np.zeros(shape, np.complex128)
                e.reshape(-1)[j] = unit
                flat[j] += to * _inner(dI, fn(e))
        return out

    dSl = pull(lambda e: oracle.history_slice(t, order, n, L, R, e, zS), Sl.shape)
    dSg = pull(lambda e: oracle.history_slice(t, order, n, L, R, zS, e), Sg.shape)

    def rows(e_rows, which):
        e = np.zeros_like(L)
        e[base:] = e_rows
        return oracle.history_slice(t, order, n, e, zL, Sl, Sg) if which == "L" else \
            oracle.history_slice(t, order, n, zL, e, Sl, Sg)

    shape = (L.shape[0] - base,) + L.shape[1:]
    diag = {W.tri_index(r, r) - base for r in range(row_lo, n + 1)}
    dL = pull(lambda e: rows(e, "L"), shape)
    dR = pull(lambda e: rows(e, "R"), shape, skip=diag)
    return dSl, dSg, dL, dR


def _cplx(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _ctx(kbe, M, n_max, t, order, h, U):
    ctx = kbe.Context(M, n_max)
    ctx.set_grid(t, order)
    ctx.set_model(h, U, W.site_potential(M), None)
    return ctx


@pytest.mark.parametrize("M,n_t,n,row_lo", [(1, 6, 0, 0), (2, 20, 7, 0), (3, 30, 29, 12), (5, 41, 33, 33),
                                            (8, 64, 63, 40)])
def test_adjoint_slice_dot_products(kbe, M, n_t, n, row_lo):
    import torch
    rng = np.random.default_rng(100 * M + n)
    t, order = W.grid(n_t, 0.05, 0.4, M + n)
    L, R = W.random_triangles(M, n + 1, 7 * M + n)
    Sl, Sg = W.random_rows(M, n, 3 * M + n)
    dI = _cplx(rng, (2, n + 1, M, M))
    h = W.goe_h(M, 1)
    ctx = _ctx(kbe, M, n_t, t, order, h, np.ones(M))
    base = W.tri_size(row_lo)
    nblk = W.tri_size(n + 1) - base
    dSl = torch.zeros((n + 1, M, M), dtype=torch.complex128, device="cuda")
    dSg = torch.zeros_like(dSl)
    dL = torch.zeros((nblk, M, M), dtype=torch.complex128, device="cuda")
    dR = torch.zeros_like(dL)
    ctx.adjoint_slice(n, _dev(L), _dev(R), _dev(Sl), _dev(Sg), _dev(dI), dSl, dSg, dL, dR, row_lo)
    ctx.sync_status()
    dSl, dSg, dL, dR = (x.cpu().numpy() for x in (dSl, dSg, dL, dR))
    I0 = oracle.history_slice(t, order, n, L, R, Sl, Sg)
    for trial in range(3):
        # self-energy direction
        eSl, eSg = _cplx(rng, Sl.shape), _cplx(rng, Sg.shape)
        y = oracle.history_slice(t, order, n, L, R, eSl, eSg)
        lhs = _inner(dI, y)
        rhs = _inner(dSl, eSl) + _inner(dSg, eSg)
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + _rss(dI, y)), (trial, lhs, rhs)
        # G direction on rows row_lo..n (R(r,r) fixed)
        eL = np.zeros_like(L)
        eR = np.zeros_like(R)
        eL[base:] = _cplx(rng, eL[base:].shape)
        eR[base:] = _cplx(rng, eR[base:].shape)
        for r in range(row_lo, n + 1):
            eR[W.tri_index(r, r)] = 0
        # the slice is linear in (L, R) at fixed Sigma: evaluate the direction itself
        dIg = oracle.history_slice(t, order, n, eL, eR, Sl, Sg)
        lhs = _inner(dI, dIg)
        rhs = _inner(dL, eL[base:]) + _inner(dR, eR[base:])
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + _rss(dI, dIg)), (trial, lhs, rhs)
    # the diagonal blocks of R get no cotangent, rows below row_lo are not formed
    for r in range(row_lo, n + 1):
        assert not np.any(dR[W.tri_index(r, r) - base])
    ctx.close()


@pytest.mark.parametrize("M,n,row_lo", [(1, 4, 0), (2, 5, 0), (3, 6, 2), (2, 6, 6)])
def test_adjoint_slice_elementwise_against_oracle_transpose(kbe, M, n, row_lo):
    """Every entry of the Sigma-row and history cotangents of
    kbe_adjoint_slice equals the oracle's exact vector-Jacobian product
    (the transpose of its slice, built column by column from basis
    directions) to 1e-12 of the largest entry."""
    import torch
    n_t = n + 3
    rng = np.random.default_rng(1000 + 10 * M + n)
    t, order = W.grid(n_t, 0.05, 0.4, 50 + M + n)
    L, R = W.random_triangles(M, n + 1, 60 + M + n)
    Sl, Sg = W.random_rows(M, n, 70 + M + n)
    dI = _cplx(rng, (2, n + 1, M, M))
    ctx = _ctx(kbe, M, n_t, t, order, W.goe_h(M, 1), np.ones(M))
    base = W.tri_size(row_lo)
    nblk = W.tri_size(n + 1) - base
    dSl = torch.zeros((n + 1, M, M), dtype=torch.complex128, device="cuda")
    dSg = torch.zeros_like(dSl)
    dL = torch.zeros((nblk, M, M), dtype=torch.complex128, device="cuda")
    dR = torch.zeros_like(dL)
    ctx.adjoint_slice(n, _dev(L), _dev(R), _dev(Sl), _dev(Sg), _dev(dI), dSl, dSg, dL, dR, row_lo)
    ctx.sync_status()
    got = [x.cpu().numpy() for x in (dSl, dSg, dL, dR)]
    ref = _oracle_vjp(t, order, n, L, R, Sl, Sg, dI, row_lo)
    for name, a, b in zip(("dS<", "dS>", "dL", "dR"), got, ref):
        err = np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)
        assert err < 1e-12, (name, err)
    ctx.close()


def test_adjoint_slice_is_deterministic(kbe):
    import torch
    M, n_t, n = 8, 90, 89
    t, order = W.grid(n_t, 0.05, 0.4, 5)
    L, R = W.random_triangles(M, n + 1, 5)
    Sl, Sg = W.random_rows(M, n, 6)
    dI = _cplx(np.random.default_rng(7), (2, n + 1, M, M))
    ctx = _ctx(kbe, M, n_t, t, order, W.goe_h(M, 1), np.ones(M))
    outs = []
    for _ in range(2):
        bufs = [torch.zeros((n + 1, M, M), dtype=torch.complex128, device="cuda") for _ in range(2)]
        bufs += [torch.zeros((W.tri_size(n + 1), M, M), dtype=torch.complex128, device="cuda") for _ in range(2)]
        ctx.adjoint_slice(n, _dev(L), _dev(R), _dev(Sl), _dev(Sg), _dev(dI), *bufs, 0)
        outs.append([b.cpu().numpy() for b in bufs])
    ctx.sync_status()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    ctx.close()


def _sigma_dir(U, n, L, R, eL, eR, eU, h):
    """Directional derivative of the oracle's self-energy row (exact for a
    polynomial of degree <= 3 up to rounding: Richardson on two central
    differences)."""
    def D(s):
        p = oracle.sigma_row(oracle.local_U4(U + s * eU), n, L + s * eL, R + s * eR)
        m = oracle.sigma_row(oracle.local_U4(U - s * eU), n, L - s * eL, R - s * eR)
        return [(a - b) / (2 * s) for a, b in zip(p, m)]
    d1, d2 = D(h), D(2 * h)
    return [(4 * a - b) / 3 for a, b in zip(d1, d2)]


@pytest.mark.parametrize("M,n", [(1, 0), (2, 5), (4, 17), (8, 30)])
def test_adjoint_selfenergy_directional(kbe, M, n):
    import torch
    rng = np.random.default_rng(M + 50 * n)
    t, order = W.grid(n + 1, 0.05, 0.4, M)
    h = W.goe_h(M, M)
    L, R = W.free_triangles(h, W.half_filled_rho(h), t)
    U = np.linspace(0.7, 1.9, M)
    ctx = _ctx(kbe, M, n + 1, t, order, h, U)
    dSl, dSg = _cplx(rng, (n + 1, M, M)), _cplx(rng, (n + 1, M, M))
    gL = torch.zeros((n + 1, M, M), dtype=torch.complex128, device="cuda")
    gR = torch.zeros_like(gL)
    dU = torch.zeros(M, dtype=torch.float64, device="cuda")
    ctx.adjoint_selfenergy_slice(n, _dev(L), _dev(R), _dev(dSl), _dev(dSg), gL, gR, dU)
    ctx.sync_status()
    gL, gR, dU = gL.cpu().numpy(), gR.cpu().numpy(), dU.cpu().numpy()
    p = W.tri_index(n, 0)
    assert not np.any(gR[n])
    for trial in range(3):
        eL = np.zeros_like(L)
        eR = np.zeros_like(R)
        eL[p:p + n + 1] = _cplx(rng, (n + 1, M, M))
        eR[p:p + n] = _cplx(rng, (n, M, M))
        eU = rng.standard_normal(M) if trial else np.zeros(M)
        dsl, dsg = _sigma_dir(U, n, L, R, eL, eR, eU, 1e-3)
        lhs = _inner(dSl, dsl) + _inner(dSg, dsg)
        rhs = _inner(gL, eL[p:p + n + 1]) + _inner(gR, eR[p:p + n + 1]) + float(dU @ eU)
        assert abs(lhs - rhs) <= 1e-9 * (abs(lhs) + np.abs(dSl).max()), (trial, lhs, rhs)
    ctx.close()


def _window_case(M, n_t, n_start, seed, pulse_in_window):
    cfg = dict(W.CONFIGS["chain_m8_n1024"], M=M, n_t=n_t)
    t, order = W.grid(n_t, cfg["dt0"], cfg["sig"], seed)
    h, U, v, pulse = W.build_model(cfg, seed)
    if pulse_in_window:
        pulse = dict(pulse, t0=float(t[(n_start + n_t) // 2]), sigma=0.25)
    rho0 = W.half_filled_rho(h)
    L, R, F = W.restart_state(h, rho0, t, order, n_start, n_t)
    return t, order, h, U, v, pulse, L, R, F


@pytest.mark.parametrize("M,n_t,W_,P", [(2, 30, 12, 2), (4, 48, 16, 2), (3, 40, 20, 1), (4, 36, 8, 3)])
def test_window_gradient_matches_oracle_tangent(kbe, M, n_t, W_, P):
    """dF/dU_a and dF/dE0 of F = 2 Im L(N-1,N-1)_00 through a window of W_
    steps, against the oracle's forward-mode derivative, to 1e-9."""
    import torch
    n_start = n_t - W_
    t, order, h, U, v, pulse, L, R, F = _window_case(M, n_t, n_start, M + W_, True)
    ctx = kbe.Context(M, n_t)
    ctx.set_grid(t, order)
    win = kbe.Window(ctx, _dev(L), _dev(R), F, n_start, n_t, h, v, pulse, P=P)
    Ut = torch.tensor(U, dtype=torch.float64, requires_grad=True)
    E0 = torch.tensor(pulse["E0"], dtype=torch.float64, requires_grad=True)
    blk = kbe.window_final_block(Ut, E0, win)
    loss = 2.0 * blk[0, 0].imag
    loss.backward()
    ctx.sync_status()
    gU, gE = Ut.grad.numpy(), float(E0.grad)
    Lv = None
    for a in range(M):
        e = np.zeros(M)
        e[a] = 1.0
        Lv, Ld = oracle.run_tangent(t, order, h, U, e, v, pulse, 0.0, P, L, R, F, n_start, n_t, nthreads=4)
        ref = 2.0 * Ld[0, 0].imag
        assert abs(gU[a] - ref) <= 1e-9 * max(abs(ref), 1e-3), (a, gU[a], ref)
    _, Ld = oracle.run_tangent(t, order, h, U, np.zeros(M), v, pulse, 1.0, P, L, R, F, n_start, n_t, nthreads=4)
    ref = 2.0 * Ld[0, 0].imag
    assert abs(gE - ref) <= 1e-9 * max(abs(ref), 1e-3), (gE, ref)
    # the forward value is the oracle's
    assert np.abs(blk.detach().cpu().numpy() - Lv).max() < 1e-12 * np.abs(Lv).max()
    ctx.close()


def _window_full(kbe, pulse_in_window, seed=0):
    import torch
    cfg = W.CONFIGS["chain_m16_n512_w32"]
    M, n_t, Wn = cfg["M"], cfg["n_t"], cfg["window"]
    n_start = n_t - Wn
    t, order = W.grid(n_t, cfg["dt0"], cfg["sig"], seed)
    h, U, v, pulse = W.build_model(cfg, seed)
    if pulse_in_window:
        pulse = dict(pulse, t0=float(t[-1] - 0.35))
    rho0 = W.half_filled_rho(h)
    L, R, F = W.restart_state(h, rho0, t, order, n_start, n_t, device="cuda")
    ctx = kbe.Context(M, n_t)
    ctx.set_grid(t, order)
    win = kbe.Window(ctx, L, R, F, n_start, n_t, h, v, pulse, P=2)
    return ctx, win, U, pulse


def _density(win, U, E0):
    return 2.0 * float(win.forward(U, E0)[0, 0].imag.cpu())


@pytest.mark.parametrize("pulse_in_window", [False, True])
def test_window_gradient_full_size_vs_finite_differences(kbe, pulse_in_window):
    """Differentiation workload (16-orbital chain, 512 points, last 32
    steps): the adjoint gradient against central differences of the same
    forward, h = 1e-5; 1e-6 relative for the uniform U and a random
    per-site direction, and for E0 when the pulse acts inside the window
    (centred 0.35 before the final time).  With the pulse centred at t = 5
    the field in the window is ~1e-7 of its peak; there the E0 derivative
    is compared in absolute terms."""
    import torch
    ctx, win, U, pulse = _window_full(kbe, pulse_in_window)
    E0 = pulse["E0"]
    Ut = torch.tensor(U, dtype=torch.float64, requires_grad=True)
    Et = torch.tensor(E0, dtype=torch.float64, requires_grad=True)
    loss = 2.0 * kbe.window_final_block(Ut, Et, win)[0, 0].imag
    loss.backward()
    ctx.sync_status()
    gU, gE = Ut.grad.numpy(), float(Et.grad)
    h = 1e-5
    rng = np.random.default_rng(3)
    for name, d in (("uniform", np.ones_like(U)), ("random", rng.standard_normal(U.shape))):
        fd = (_density(win, U + h * d, E0) - _density(win, U - h * d, E0)) / (2 * h)
        ad = float(gU @ d)
        print(name, "U: adjoint", ad, "fd", fd)
        assert abs(ad - fd) <= 1e-6 * abs(fd), (name, ad, fd)
    fd = (_density(win, U, E0 + h) - _density(win, U, E0 - h)) / (2 * h)
    print("E0: adjoint", gE, "fd", fd)
    if pulse_in_window:
        assert abs(gE - fd) <= 1e-6 * abs(fd), (gE, fd)
    else:
        assert abs(gE - fd) <= 1e-9, (gE, fd)
    ctx.close()


def test_window_gradient_double_float(kbe):
    """A window run with the double-float contraction (KBE_DF64 forward and
    recompute, FP64 adjoint kernels): its gradient against the oracle's
    forward-mode derivative (1e-8: the forward differs from the FP64 one by
    the contraction's ~2^-47 of the terms), and kbe_step_adjoint rejects the
    split precision."""
    import torch
    M, n_t, W_, P = 3, 24, 6, 2
    n_start = n_t - W_
    t, order, h, U, v, pulse, L, R, F = _window_case(M, n_t, n_start, 11, True)
    ctx = kbe.Context(M, n_t)
    ctx.set_grid(t, order)
    win = kbe.Window(ctx, _dev(L), _dev(R), F, n_start, n_t, h, v, pulse, P=P, precision="df64")
    Ut = torch.tensor(U, dtype=torch.float64, requires_grad=True)
    E0 = torch.tensor(pulse["E0"], dtype=torch.float64, requires_grad=True)
    blk = kbe.window_final_block(Ut, E0, win)
    (2.0 * blk[0, 0].imag).backward()
    ctx.sync_status()
    gU, gE = Ut.grad.numpy(), float(E0.grad)
    for a in range(M):
        e = np.zeros(M)
        e[a] = 1.0
        _, Ld = oracle.run_tangent(t, order, h, U, e, v, pulse, 0.0, P, L, R, F, n_start, n_t, nthreads=4)
        ref = 2.0 * Ld[0, 0].imag
        assert abs(gU[a] - ref) <= 1e-8 * max(abs(ref), 1e-3), (a, gU[a], ref)
    _, Ld = oracle.run_tangent(t, order, h, U, np.zeros(M), v, pulse, 1.0, P, L, R, F, n_start, n_t, nthreads=4)
    ref = 2.0 * Ld[0, 0].imag
    assert abs(gE - ref) <= 1e-8 * max(abs(ref), 1e-3), (gE, ref)
    with pytest.raises(ValueError):
        kbe.Window(ctx, _dev(L), _dev(R), F, n_start, n_t, h, v, pulse, P=P, precision="split")
    dL = torch.zeros((W.tri_size(n_t), M, M), dtype=torch.complex128, device="cuda")
    dU = torch.zeros(M, dtype=torch.float64, device="cuda")
    dE = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(kbe.KBEError) as err:
        ctx.step_adjoint(n_t - 1, P, win.L, win.R, win.F, win.j0, dL, dL.clone(), 0, torch.zeros_like(win.F), dU, dE,
                         precision="split")
    assert err.value.status == kbe.KBE_EINVAL
    ctx.close()
