"""Pins for the oracle's KBE stepper and its forward-mode derivatives."""
import numpy as np
import pytest

import oracle
import workloads as W
from closed_forms import free_lesser, free_retarded

tri = W.tri_index


def run_full(h, U, v, pulse, rho0, t, order, P=2, nthreads=4):
    """A run from the uncorrelated state at t = 0 (interaction switched on at t = 0)."""
    M = h.shape[0]
    N = len(t)
    L0, R0, F0 = oracle.initial_rhs(t, order, h, U, v, pulse, rho0)
    L = np.zeros((W.tri_size(N), M, M), np.complex128)
    R = np.zeros_like(L)
    L[0], R[0] = L0[0], R0[0]
    return oracle.run(t, order, h, U, v, pulse, P, L, R, {0: F0}, 1, N, nthreads=nthreads)


def energy_and_number(h, U, L, R, t, order, n):
    """Spin-summed E(t_n) = 2 Tr[h rho] + sum_a U_a n_a^2 + E_c with the
    Galitskii-Migdal correlation term E_c = -i Tr I^<(t_n, t_n), and
    N(t_n) = 2 sum_a n_a, rho = -i G^<(t_n, t_n)."""
    rho = -1j * L[tri(n, n)]
    Sl, Sg = oracle.sigma_row(oracle.local_U4(U), n, L, R)
    I = oracle.history_slice(t, order, n, L, R, Sl, Sg, nthreads=4)
    na = np.real(np.diag(rho))
    Ec = -1j * np.trace(I[0, n])
    E = 2 * np.real(np.trace(h @ rho)) + np.sum(U * na ** 2) + Ec
    return E, 2 * np.sum(na)


@pytest.mark.parametrize("k,expect", [(1, 2.0), (2, 3.0)])
def test_noninteracting_run_converges_to_free_propagators(k, expect):
    """U = 0: the run reproduces G^R(t,t') = -i e^{-ih(t-t')} and
    G^<(t,t') = i e^{-iht} rho0 e^{iht'} at the order of the rule."""
    M = 2
    h = W.chain_h(M)
    rho0 = W.half_filled_rho(h)
    v = W.site_potential(M)
    errs = []
    for N in (21, 41, 81):
        t, order = W.uniform_grid(N, 2.0 / (N - 1), k)
        L, R, _ = run_full(h, np.zeros(M), v, None, rho0, t, order)
        n, c = N - 1, (N - 1) // 2
        errs.append(max(np.abs(L[tri(n, c)] - free_lesser(h, rho0, t[n], t[c])).max(),
                        np.abs(R[tri(n, c)] - free_retarded(h, t[n], t[c])).max(),
                        np.abs(L[tri(n, n)] - free_lesser(h, rho0, t[n], t[n])).max()))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - expect) < 0.35 for r in rates), (errs, rates)


def test_second_born_conserves_energy_and_number():
    """GF2 is Phi-derivable (Sec. 5.3): after the quench at t = 0 the total
    energy is constant, so the drift of E(T) - E(0) must fall with the step
    (third order for k = 2), and the particle number stays fixed."""
    M = 2
    h = W.chain_h(M)
    rho0 = W.half_filled_rho(h)
    v = W.site_potential(M)
    U = np.full(M, 1.0)
    drift = []
    for N in (41, 81, 161):
        t, order = W.uniform_grid(N, 4.0 / (N - 1), 2)
        L, R, _ = run_full(h, U, v, None, rho0, t, order)
        E0, N0 = energy_and_number(h, U, L, R, t, order, 0)
        E1, N1 = energy_and_number(h, U, L, R, t, order, N - 1)
        assert abs(E1.imag) < 1e-12
        assert abs(N1 - N0) < 1e-12
        drift.append(abs(E1 - E0))
    assert drift[1] < drift[0] / 6 and drift[2] < drift[1] / 6, drift
    assert drift[2] < 1e-4


def test_number_conserved_goe_nonuniform():
    M = 3
    h = W.goe_h(M, 2)
    rho0 = W.half_filled_rho(h)
    v = W.site_potential(M)
    U = np.array([1.0, 1.5, 0.7])
    t, order = W.grid(60, 0.05, 0.3, 1)
    L, R, _ = run_full(h, U, v, None, rho0, t, order)
    _, N0 = energy_and_number(h, U, L, R, t, order, 0)
    for n in (10, 30, 59):
        _, Nn = energy_and_number(h, U, L, R, t, order, n)
        assert abs(Nn - N0) < 1e-12
        D = L[tri(n, n)]
        assert np.abs(D + D.conj().T).max() < 1e-14  # G^<(t,t) stays anti-Hermitian


def test_energy_changes_under_pulse_and_number_does_not():
    M = 2
    h = W.chain_h(M)
    rho0 = W.half_filled_rho(h)
    v = W.site_potential(M)
    U = np.full(M, 1.0)
    t, order = W.grid(64, 0.05, 0.3, 0)
    pulse = {"E0": 0.5, "t0": 1.5, "sigma": 0.5, "omega": 2.0}
    L, R, _ = run_full(h, U, v, pulse, rho0, t, order)
    _, N0 = energy_and_number(h, U, L, R, t, order, 0)
    _, N1 = energy_and_number(h, U, L, R, t, order, 63)
    assert abs(N1 - N0) < 1e-12
    # the field pushes charge between the two sites
    n_site = -1j * np.diag(L[tri(63, 63)])
    assert abs(n_site[0].real - n_site[1].real) > 1e-3


def _window_case():
    M = 2
    h = W.chain_h(M)
    rho0 = W.half_filled_rho(h)
    v = W.site_potential(M)
    t, order = W.grid(24, 0.1, 0.3, 3)
    N, ns = 24, 18
    L, R = W.free_triangles(h, rho0, t, n_rows=ns)
    Lf = np.zeros((W.tri_size(N), M, M), np.complex128)
    Rf = np.zeros_like(Lf)
    Lf[: len(L)], Rf[: len(R)] = L, R
    Fr = W.free_rhs_rows(h, L, R, oracle.f_rows_needed(order, ns, N))
    pulse = {"E0": 0.5, "t0": t[N - 1] - 0.3, "sigma": 0.5, "omega": 2.0}
    return M, h, v, t, order, N, ns, L, R, Lf, Rf, Fr, pulse


def test_tangent_matches_central_differences():
    """Forward-mode duals through a window of steps vs central differences
    (h = 1e-5) of the same map; the tangent is exact for the discrete map."""
    M, h, v, t, order, N, ns, L, R, Lf, Rf, Fr, pulse = _window_case()

    def n0(Uv, E0):
        p = dict(pulse, E0=E0)
        L2, _, _ = oracle.run(t, order, h, np.full(M, Uv), v, p, 2, Lf, Rf, Fr, ns, N)
        return L2[tri(N - 1, N - 1)][0, 0].imag

    eps = 1e-5
    _, dU = oracle.run_tangent(t, order, h, np.full(M, 1.0), np.ones(M), v, pulse, 0.0, 2, L, R, Fr, ns, N)
    fdU = (n0(1 + eps, 0.5) - n0(1 - eps, 0.5)) / (2 * eps)
    _, dE = oracle.run_tangent(t, order, h, np.full(M, 1.0), np.zeros(M), v, pulse, 1.0, 2, L, R, Fr, ns, N)
    fdE = (n0(1.0, 0.5 + eps) - n0(1.0, 0.5 - eps)) / (2 * eps)
    assert abs(dU[0, 0].imag - fdU) < 1e-7 * abs(fdU)
    assert abs(dE[0, 0].imag - fdE) < 1e-7 * abs(fdE)
    # the value part of the tangent run equals the plain run
    Lv, _ = oracle.run_tangent(t, order, h, np.full(M, 1.0), np.ones(M), v, pulse, 0.0, 2, L, R, Fr, ns, N)
    L2, _, _ = oracle.run(t, order, h, np.full(M, 1.0), v, pulse, 2, Lf, Rf, Fr, ns, N)
    assert np.array_equal(Lv, L2[tri(N - 1, N - 1)])
