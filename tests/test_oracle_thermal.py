"""Pins for the oracle's thermal branch (Sec. 2, Eq. KBE3 and the tau terms
of Eq. KBE2) on a uniform tau grid: the split Matsubara convolution against
closed forms, the mixed self-energy against the local-interaction reduction,
the non-interacting run against the exact mixed function, and convergence in
the tau grid with interaction."""
import numpy as np
import pytest

import oracle
import workloads as W


def _gm_scalar(eps, beta, tau):
    """Free Matsubara function of one level at chemical potential 0."""
    return -np.exp(-eps * tau) / (1.0 + np.exp(-beta * eps))


def _conv_error(a, eps, N, beta=4.0, ktau=5):
    tau = beta * np.arange(N) / (N - 1)
    S = np.exp(a * tau).reshape(N, 1, 1).astype(np.complex128)
    GM = _gm_scalar(eps, beta, tau).reshape(N, 1, 1).astype(np.complex128)
    out = oracle.matsubara_conv(beta, ktau, S, GM)[:, 0, 0]
    c = 1.0 / (1.0 + np.exp(-beta * eps))          # 1 - f
    k = a - eps
    prim = lambda x: np.exp(k * x) / k
    left = c * np.exp(-eps * (beta - tau)) * (prim(tau) - prim(0.0))      # s in [0, tau]
    right = -c * np.exp(eps * tau) * (prim(beta) - prim(tau))             # s in [tau, beta]
    ref = left + right
    err = np.abs(out - ref) / np.abs(ref).max()
    return err


@pytest.mark.parametrize("a,eps", [(0.7, 1.3), (-1.1, -0.6), (0.3, 2.0)])
def test_matsubara_convolution_closed_form(a, eps):
    """int_0^beta e^{a s} G^M(s - tau) ds with the antiperiodic G^M(s - tau)
    = -G^M(beta + s - tau) for s < tau, in closed form.  Away from the ends
    the rule has its full order; a piece of fewer than ktau intervals on one
    side of the split (tau within ktau points of 0 or beta) is integrated at
    the order its own nodes allow, so the error there falls at least like
    h^3."""
    e1, e2 = _conv_error(a, eps, 81), _conv_error(a, eps, 161)
    inner1, inner2 = e1[3:-3:2].max(), e2[6:-6:4].max()  # the same tau points on both grids
    assert inner2 < 1e-10 and inner1 > 30 * inner2        # interior: order ktau + 1 = 6
    assert e2.max() < 2e-5
    assert e1.max() > 6 * e2.max()                        # ends: at least third order


def test_sigma_mixed_local_reduction():
    """With U_abcd = U_a delta_abcd, Eq. (SE) for the mixed component reduces
    to Sigma^|_ab(t,tau) = U_a U_b G^|_ab(t,tau)^2 G^|-_ba(tau,t), with
    G^|-(tau,t) = G^|(t, beta - tau)^+."""
    M, N, n = 3, 9, 2
    rng = np.random.default_rng(4)
    Gm = rng.standard_normal((n + 1, N, M, M)) + 1j * rng.standard_normal((n + 1, N, M, M))
    U = np.array([0.5, 1.2, 2.0])
    S = oracle.sigma_mixed(oracle.local_U4(U), n, Gm)
    for k in range(N):
        adj_ba = np.conj(Gm[n, N - 1 - k])  # G^|-(tau_k, t_n)_ba = conj(G^|(t_n, beta - tau_k)_ab)
        ref = np.outer(U, U) * Gm[n, k] ** 2 * adj_ba
        assert np.abs(S[k] - ref).max() < 1e-13 * np.abs(ref).max()


def _free_run(dt, n_t=21, M=2, beta=5.0, N=41):
    h = W.goe_h(M, 1)
    t, order = W.uniform_grid(n_t, dt, 5)
    GM, rho, mix = W.thermal_free(h, beta, N, t)
    L, R, Gm = oracle.run_thermal(t, order, h, np.zeros(M), W.site_potential(M), None, 2, beta, N, 5, GM,
                                  1j * rho, -1j * np.eye(M))
    Lf, Rf = W.free_triangles(h, rho, t)
    return np.abs(Gm - mix).max(), np.abs(L - Lf).max(), Gm, rho


def test_free_thermal_run_is_the_exact_mixed_function():
    """U = 0: G^|(t,tau) = i e^{-iht} f(h) e^{h tau} and G^< from the Fermi
    state; the stepper's error falls with the step."""
    e1, l1, Gm, rho = _free_run(0.1, n_t=11)
    e2, l2, _, _ = _free_run(0.05, n_t=21)
    assert e2 < 2e-5 and l2 < 2e-5
    assert e1 > 8 * e2  # same end time, half the step
    # the initial mixed row is -i G^M(beta - tau), whose tau = 0 end is G^<(0,0) = i rho
    assert np.abs(Gm[0, 0] - 1j * rho).max() < 1e-14


def _interacting(N, n_t=16, ktau=4):
    M = 2
    h = W.chain_h(M)
    beta = 4.0
    t, order = W.uniform_grid(n_t, 0.05, 4)
    GM, rho, _ = W.thermal_free(h, beta, N)
    U = np.array([1.0, 1.5])
    return oracle.run_thermal(t, order, h, U, W.site_potential(M), None, 2, beta, N, ktau, GM, 1j * rho,
                              -1j * np.eye(M), nthreads=4)


def test_interacting_run_converges_in_the_tau_grid():
    """With interaction the tau integrals enter the dynamics: the rows
    converge at the order of the tau rule as the grid is refined, and the
    diagonal stays anti-Hermitian."""
    runs = {N: _interacting(N) for N in (41, 81, 161)}
    d1 = np.abs(runs[41][0] - runs[81][0]).max()
    d2 = np.abs(runs[81][0] - runs[161][0]).max()
    assert d1 > 8 * d2 and d2 < 1e-6  # at least third order (the end pieces), measured ~22x per halving
    L = runs[161][0]
    n = 15
    D = L[W.tri_index(n, n)]
    assert np.abs(D + D.conj().T).max() < 1e-14
    # the thermal terms matter: without them (same initial density) the rows differ
    M = 2
    h = W.chain_h(M)
    t, order = W.uniform_grid(16, 0.05, 4)
    _, rho, _ = W.thermal_free(h, 4.0, 21)
    L0, R0, F0 = oracle.initial_rhs(t, order, h, np.array([1.0, 1.5]), W.site_potential(M), None, rho)
    Lz = np.zeros_like(L)
    Rz = np.zeros_like(L)
    Lz[0], Rz[0] = L0[0], R0[0]
    Lz, _, _ = oracle.run(t, order, h, np.array([1.0, 1.5]), W.site_potential(M), None, 2, Lz, Rz, {0: F0}, 1, 16)
    assert np.abs(Lz - L).max() > 1e-3


def test_number_conservation_needs_mirror_symmetric_tau_weights():
    """For the second-Born self-energy, Tr[Sigma^|(t,tau) G^|-(tau,t)] at tau
    and at beta - tau are complex conjugates (Eq. SE with G^|-(tau,t) =
    G^|(t,beta-tau)^+), so the KBE2 mixed term keeps dN/dt = 0 exactly when
    the tau weights are mirror-symmetric (odd ktau, centred windows), and not
    otherwise."""
    h = W.chain_h(2)
    _, rho, _ = W.thermal_free(h, 4.0, 41)
    n0 = np.trace(rho).real
    for ktau, ok in ((5, True), (3, True), (4, False)):
        L, _, _ = _interacting(41, ktau=ktau)
        dev = max(abs(np.trace(-1j * L[W.tri_index(n, n)]).real - n0) for n in range(16))
        assert (dev < 1e-13) == ok, (ktau, dev)


def test_free_mixed_adjoint_relation():
    """The relation the oracle uses for G^|-(tau, t) = G^|(t, beta - tau)^+
    reproduces the free G^|-(tau,t) = -i e^{-h tau} (1 - f(h)) e^{iht}."""
    M, N, beta = 3, 21, 3.0
    h = W.goe_h(M, 2)
    t = np.linspace(0.0, 1.0, 5)
    _, _, mix = W.thermal_free(h, beta, N, t)
    e, V = np.linalg.eigh(h)
    tau = beta * np.arange(N) / (N - 1)
    one_m_f = 0.5 * (1.0 + np.tanh(0.5 * beta * e))
    for r in range(len(t)):
        for k in range(N):
            direct = -1j * (V * (np.exp(-e * tau[k]) * one_m_f * np.exp(1j * e * t[r]))) @ V.conj().T
            assert np.abs(mix[r, N - 1 - k].conj().T - direct).max() < 1e-13
