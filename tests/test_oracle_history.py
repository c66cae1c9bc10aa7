"""Pins for the oracle's history slice (Eq. KBE2) and its Eq. (KBE1) form."""
import numpy as np
import pytest

import oracle
import workloads as W
from closed_forms import history_closed_form


def _free_case(M, n_t, seed, U=None, grid=None):
    h = W.goe_h(M, seed)
    rho0 = W.half_filled_rho(h)
    t, order = grid if grid is not None else W.grid(n_t, 0.1, 0.4, seed)
    L, R = W.free_triangles(h, rho0, t)
    U = np.linspace(0.6, 1.4, M) if U is None else U
    return h, rho0, U, t, order, L, R


def _slice(t, order, n, L, R, U, nthreads=4):
    Sl, Sg = oracle.sigma_row(oracle.local_U4(U), n, L, R)
    return oracle.history_slice(t, order, n, L, R, Sl, Sg, nthreads=nthreads), Sl, Sg


def test_zero_length_history_vanishes():
    _, _, U, t, order, L, R = _free_case(2, 6, 1)
    I, _, _ = _slice(t, order, 0, L, R, U)
    assert np.array_equal(I, np.zeros_like(I))


def test_single_orbital_constant_integrand_is_exact():
    """For one orbital the non-interacting integrands of Eq. (KBE2) do not
    depend on the integration variable, so every composite rule is exact:
    I^s(n,c) = t_n * [Sigma^R G^s](n,c) + t_c * [Sigma^s G^A](n,c)."""
    h = np.array([[0.37]], np.complex128)
    rho0 = np.array([[0.5]], np.complex128)
    for seed in (0, 1, 2):
        t, order = W.grid(40, 0.07, 0.5, seed)
        L, R = W.free_triangles(h, rho0, t)
        U = np.array([1.3])
        n = 39
        I, Sl, Sg = _slice(t, order, n, L, R, U)
        for c in range(n + 1):
            exc = history_closed_form(h, rho0, U, t[n], t[c])
            assert np.allclose(I[:, c], exc, rtol=1e-13, atol=1e-14), c


@pytest.mark.parametrize("k,expect", [(1, 2.0), (2, 3.0), (3, 3.0)])
def test_convergence_against_closed_form(k, expect):
    """Uniform grids with all requested orders k: the error against the exact
    integral falls as h^(k+1) for k = 1, 2.  For k >= 3 the first intervals
    are capped at order min(k, l) (backward stencils only), which limits the
    composite rule to third order -- the expected rate."""
    M = 3
    h = W.goe_h(M, 5)
    rho0 = W.half_filled_rho(h)
    U = np.array([1.0, 0.7, 1.3])
    T = 2.0
    errs = []
    for N in (21, 41, 81):
        t, order = W.uniform_grid(N, T / (N - 1), k)
        L, R = W.free_triangles(h, rho0, t)
        n, c = N - 1, (N - 1) // 2
        I, _, _ = _slice(t, order, n, L, R, U)
        ex = history_closed_form(h, rho0, U, t[n], t[c])
        errs.append(np.abs(I[:, c] - ex).max() / np.abs(ex).max())
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - expect) < 0.25 for r in rates), (errs, rates)


def test_nonuniform_grid_close_to_closed_form():
    M = 3
    h = W.goe_h(M, 9)
    rho0 = W.half_filled_rho(h)
    U = np.array([0.9, 1.4, 0.5])
    t, order = W.grid(80, 0.03, 0.4, 4)
    L, R = W.free_triangles(h, rho0, t)
    n = 79
    I, _, _ = _slice(t, order, n, L, R, U)
    for c in (0, 17, 40, 78, 79):
        ex = history_closed_form(h, rho0, U, t[n], t[c])
        assert np.abs(I[:, c] - ex).max() < 2e-4 * np.abs(ex).max(), c


# ------------------------------------------------------------ brute force --
def _vandermonde_weights(t, order, n):
    """Composite row by the paper's route (V^T w = T per interval), in numpy."""
    row = np.zeros(n + 1)
    for l in range(1, n + 1):
        k = min(order[l], l)
        x = t[l - k:l + 1] - t[l - k]
        V = np.vander(x, k + 1, increasing=True)
        a, b = t[l - 1] - t[l - k], t[l] - t[l - k]
        T = np.array([(b ** (i + 1) - a ** (i + 1)) / (i + 1) for i in range(k + 1)])
        row[l - k:l + 1] += np.linalg.solve(V.T, T)
    return row


def _brute_force(t, order, n, L, R, Sl, Sg):
    """Full (N M) x (N M) planes and the weight matrix, then the Langreth
    products of Eq. (KBE2) as matrix algebra."""
    M = L.shape[-1]
    N = n + 1
    Pl = np.zeros((N, N, M, M), np.complex128)
    Pg = np.zeros_like(Pl)
    PA = np.zeros_like(Pl)
    for r in range(N):
        for c in range(r + 1):
            p = W.tri_index(r, c)
            Pl[r, c] = L[p]
            Pg[r, c] = R[p] + L[p]
            PA[c, r] = R[p].conj().T
            if r != c:
                Pl[c, r] = -L[p].conj().T
                Pg[c, r] = -(R[p] + L[p]).conj().T
    Wm = np.zeros((N, N))
    for c in range(N):
        Wm[c, : c + 1] = _vandermonde_weights(t, order, c)
    SR = Sg - Sl
    out = np.zeros((2, N, M, M), np.complex128)
    for s, (P, S) in enumerate([(Pl, Sl), (Pg, Sg)]):
        for c in range(N):
            t1 = np.einsum("m,mab,mbd->ad", Wm[n], SR, P[:, c])
            t2 = np.einsum("m,mab,mbd->ad", Wm[c], S, PA[:, c])  # Wm[c, m] = 0 for m > c
            out[s, c] = t1 + t2
    return out


@pytest.mark.parametrize("M,n_t,seed", [(1, 6, 0), (2, 8, 1), (3, 7, 2), (2, 5, 3)])
def test_brute_force_on_tiny_grids(M, n_t, seed):
    t, order = W.grid(n_t, 0.2, 0.5, seed)
    # random histories exercise every symmetry-derived block
    L, R = W.random_triangles(M, n_t, seed)
    for n in range(n_t):
        Sl, Sg = W.random_rows(M, n, 100 + seed)
        I = oracle.history_slice(t, order, n, L, R, Sl, Sg)
        ref = _brute_force(t, order, n, L, R, Sl, Sg)
        scale = np.abs(ref).max() + 1e-300
        assert np.abs(I - ref).max() < 1e-12 * scale, n


def test_kbe1_form_is_minus_adjoint_of_kbe2_form():
    """Eq. (KBE1) lesser integrals at (t_c, t_n) equal -I^<(n,c)^+: taking ^+
    of the Eq. (KBE2) integrand and using the symmetry maps one form onto
    the other term by term, with the same weights."""
    for M, seed in ((2, 0), (3, 1)):
        _, _, U, t, order, L, R = _free_case(M, 30, seed)
        for n in (0, 1, 7, 29):
            I, Sl, Sg = _slice(t, order, n, L, R, U)
            J = oracle.kbe1_slice(t, order, n, L, R, Sl, Sg)
            ref = -np.conj(np.swapaxes(I[0], 1, 2))
            assert np.abs(J - ref).max() < 1e-14 * (np.abs(ref).max() + 1e-300) * 10, (M, n)


def test_bilinearity():
    M = 2
    t, order = W.grid(12, 0.1, 0.4, 5)
    L, R = W.random_triangles(M, 12, 5)
    n = 11
    Sl, Sg = W.random_rows(M, n, 6)
    I = oracle.history_slice(t, order, n, L, R, Sl, Sg)
    I2 = oracle.history_slice(t, order, n, L, R, 2.5 * Sl, 2.5 * Sg)
    assert np.allclose(I2, 2.5 * I, rtol=1e-14, atol=1e-13)
    # linear in (Sl, Sg) jointly: I(S1 + S2) = I(S1) + I(S2)
    Sl2, Sg2 = W.random_rows(M, n, 7)
    Ia = oracle.history_slice(t, order, n, L, R, Sl2, Sg2)
    Ib = oracle.history_slice(t, order, n, L, R, Sl + Sl2, Sg + Sg2)
    assert np.allclose(Ib, I + Ia, rtol=1e-13, atol=1e-12)


def test_columns_subset_matches_full_slice():
    M = 3
    t, order = W.grid(20, 0.1, 0.4, 8)
    L, R = W.random_triangles(M, 20, 8)
    n = 17
    Sl, Sg = W.random_rows(M, n, 9)
    I = oracle.history_slice(t, order, n, L, R, Sl, Sg, nthreads=3)
    cols = [0, 5, 16, 17]
    Ic = oracle.history_columns(t, order, n, L, R, Sl, Sg, cols, nthreads=2)
    assert np.array_equal(Ic, I[:, cols])
