"""Pins for the oracle's adaptive history-order selection (Sec. 3.2): the test
integral of every order against an independent polynomial interpolation, the
test integrand against Eq. (KBE1), and conservation along an adaptive run."""
import numpy as np
import pytest

import oracle
import workloads as W

tri = W.tri_index


def _interp_integrals(t, n, kmax, u):
    """I^(k), k = 1..kmax, by fitting the degree-k polynomial through
    (t_{n-k..n}, u) with numpy and integrating it over [t_{n-1}, t_n]."""
    M = u.shape[-1]
    h = t[n] - t[n - 1]
    out = {}
    for k in range(1, kmax + 1):
        x = (t[n - k:n + 1] - t[n]) / h           # nodes, scaled, x_n = 0
        vals = u[kmax - k:].reshape(k + 1, -1)
        I = np.zeros(M * M, np.complex128)
        for e in range(M * M):
            cr = np.polynomial.polynomial.polyfit(x, vals[:, e].real, k)
            ci = np.polynomial.polynomial.polyfit(x, vals[:, e].imag, k)
            pr, pi = np.polynomial.polynomial.polyint(cr), np.polynomial.polynomial.polyint(ci)
            lo = (t[n - 1] - t[n]) / h
            I[e] = h * ((np.polynomial.polynomial.polyval(0.0, pr) - np.polynomial.polynomial.polyval(lo, pr))
                        + 1j * (np.polynomial.polynomial.polyval(0.0, pi)
                                - np.polynomial.polynomial.polyval(lo, pi)))
        out[k] = I
    return out


@pytest.mark.parametrize("kind,seed", [("smooth", 0), ("smooth", 1), ("rough", 2), ("rough", 3)])
def test_choose_order_matches_polynomial_interpolation(kind, seed):
    rng = np.random.default_rng(seed)
    t, _ = W.grid(40, 0.08, 0.4, seed)
    n, K, M = 30, 7, 2
    kmax = min(K, n)
    om = rng.uniform(-3, 3, (M, M))
    amp = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    pts = t[n - kmax:n + 1]
    u = amp[None] * np.exp(1j * om[None] * pts[:, None, None])
    if kind == "rough":  # data no polynomial fits: the differences stop falling
        u = u + 1e-3 * (rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape))
    k_opt, diffs = oracle.choose_order(t, n, K, u)
    ref = _interp_integrals(t, n, kmax, u)
    d_ref = {k: np.abs(ref[k] - ref[k - 1]).max() for k in range(2, kmax + 1)}
    mag = max(np.abs(ref[k]).max() for k in ref)
    for k in range(2, kmax + 1):
        assert abs(diffs[k] - d_ref[k]) <= 1e-9 * mag, (k, diffs[k], d_ref[k])
    dmin = min(d_ref.values())
    # the chosen order reaches the minimum difference (within the rounding tolerance)
    assert d_ref[k_opt] <= dmin + 1e-9 * mag
    assert all(d_ref[k] > dmin + 1e-9 * mag for k in range(2, k_opt)), (k_opt, d_ref)
    if kind == "smooth":
        assert k_opt == kmax  # differences fall with the order for smooth data
    else:
        assert 2 <= k_opt < kmax  # noise makes high orders worse


def test_choose_order_degenerate_cases():
    t, _ = W.grid(10, 0.1, 0.3, 0)
    u = np.ones((2, 1, 1), np.complex128)
    assert oracle.choose_order(t, 1, 5, u)[0] == 1  # one interval: only k = 1
    u = np.ones((5, 2, 2), np.complex128)
    assert oracle.choose_order(t, 4, 4, u)[0] == 2  # constants: all orders agree, the lowest is taken


def test_test_integrand_is_the_kbe1_integrand():
    """u(t_bar) integrates, with the composite weights of row n, to the lesser
    Eq. (KBE1) integral at (t_n, t_n)."""
    M = 2
    h = W.goe_h(M, 3)
    t, order = W.grid(26, 0.06, 0.4, 3)
    n = 25
    L, R = W.free_triangles(h, W.half_filled_rho(h), t)
    U = np.array([1.0, 1.6])
    Sl, Sg = oracle.sigma_row(oracle.local_U4(U), n, L, R)
    w = oracle.composite_row(t, order, n)
    total = sum(w[l] * oracle.order_test_integrand(n, l, L, R, Sl, Sg) for l in range(n + 1))
    J = oracle.kbe1_slice(t, order, n, L, R, Sl, Sg)[n]
    assert np.abs(total - J).max() < 1e-13 * np.abs(J).max()
    k, u = oracle.select_order(t, n, 6, L, R, Sl, Sg)
    for i in range(7):
        assert np.array_equal(u[i], oracle.order_test_integrand(n, n - 6 + i, L, R, Sl, Sg))
    assert k == oracle.choose_order(t, n, 6, u)[0]


def _adaptive_run(M, h, U, v, pulse, t, order, K_sel, P=2):
    rho0 = W.half_filled_rho(h)
    N = len(t)
    L0, R0, F0 = oracle.initial_rhs(t, order, h, U, v, pulse, rho0)
    L = np.zeros((W.tri_size(N), M, M), np.complex128)
    R = np.zeros_like(L)
    L[0], R[0] = L0[0], R0[0]
    return oracle.run_adaptive(t, order, [0], K_sel, h, U, v, pulse, P, L, R, {0: F0}, 1, N, nthreads=4)


def test_adaptive_run_conserves_number_and_varies_orders():
    M = 3
    h = W.goe_h(M, 2)
    U = np.array([1.0, 1.5, 0.7])
    v = W.site_potential(M)
    t, order = W.grid(60, 0.05, 0.3, 1)
    L, R, _, hord = _adaptive_run(M, h, U, v, None, t, order, 6)
    na0 = np.real(np.diag(-1j * L[0]))
    for n in (10, 30, 59):
        D = L[tri(n, n)]
        assert abs(np.sum(np.real(np.diag(-1j * D))) - np.sum(na0)) < 1e-12
        assert np.abs(D + D.conj().T).max() < 1e-14
    ks = hord[1:60]
    assert all(1 <= k <= min(6, l) for l, k in enumerate(ks, start=1))
    assert len(set(ks[6:])) > 1  # the choice follows the data


def test_adaptive_run_uses_the_orders_it_chooses():
    """Replaying an adaptive run with its chosen history orders fixed gives
    the same rows bitwise (one sweep per step, since the order is chosen again
    in every sweep), and an adaptive run and a fixed-order run approach the
    same solution under refinement."""
    M = 2
    h = W.chain_h(M)
    v = W.site_potential(M)
    U = np.full(M, 1.0)
    pulse = {"E0": 0.5, "t0": 1.5, "sigma": 0.5, "omega": 2.0}
    t, order = W.grid(50, 0.05, 0.3, 4)
    L1, R1, _, hord = _adaptive_run(M, h, U, v, pulse, t, order, 6, P=1)
    rho0 = W.half_filled_rho(h)
    L0, R0, F0 = oracle.initial_rhs(t, order, h, U, v, pulse, rho0)
    L = np.zeros_like(L1)
    R = np.zeros_like(R1)
    L[0], R[0] = L0[0], R0[0]
    L2, R2, _, h2 = oracle.run_adaptive(t, order, hord, 0, h, U, v, pulse, 1, L, R, {0: F0}, 1, len(t), nthreads=4)
    assert np.array_equal(L1, L2) and np.array_equal(R1, R2) and np.array_equal(hord, h2)
    assert len(set(hord[6:])) > 1
    ref = None
    for N, adaptive in ((161, False), (81, True)):
        tt, oo = W.uniform_grid(N, 4.0 / (N - 1), 3)
        if adaptive:
            Lr, _, _, _ = _adaptive_run(M, h, U, v, None, tt, oo, 6)
        else:
            Lr, _, _ = oracle.run(tt, oo, h, U, v, None, 2, *_start(M, h, U, v, tt, oo), 1, N, nthreads=4)
        val = Lr[tri(N - 1, N - 1)]
        ref = val if ref is None else ref
    assert np.abs(val - ref).max() < 1e-4


def _start(M, h, U, v, t, order):
    rho0 = W.half_filled_rho(h)
    L0, R0, F0 = oracle.initial_rhs(t, order, h, U, v, None, rho0)
    N = len(t)
    L = np.zeros((W.tri_size(N), M, M), np.complex128)
    R = np.zeros_like(L)
    L[0], R[0] = L0[0], R0[0]
    return L, R, {0: F0}
