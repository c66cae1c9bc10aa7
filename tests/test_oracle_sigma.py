"""Pins for the oracle's self-energy row (Sec. 2, Eq. SE)."""
import numpy as np
import pytest

import oracle
import workloads as W


def _free(M, seed, n_t=12):
    h = W.goe_h(M, seed)
    rho0 = W.half_filled_rho(h)
    t, order = W.grid(n_t, 0.1, 0.3, seed)
    L, R = W.free_triangles(h, rho0, t)
    return h, rho0, t, order, L, R


def _plane_less(L, r, c):
    if r >= c:
        return L[W.tri_index(r, c)]
    return -L[W.tri_index(c, r)].conj().T


def _plane_great(L, R, r, c):
    if r >= c:
        return R[W.tri_index(r, c)] + L[W.tri_index(r, c)]
    return -(R[W.tri_index(c, r)] + L[W.tri_index(c, r)]).conj().T


@pytest.mark.parametrize("M", [1, 2, 3])
def test_local_tensor_reduces_to_hubbard_form(M):
    """With U_abcd = U_a delta_abcd, UEx = U and Eq. (SE) reduces to
    Sigma^<>_ij(t,t') = U_i U_j G^<>_ij(t,t')^2 G^><_ji(t',t)."""
    _, _, t, order, L, R = _free(M, 11 + M)
    U = np.linspace(0.5, 1.7, M)
    n = 9
    Sl, Sg = oracle.sigma_row(oracle.local_U4(U), n, L, R)
    for c in range(n + 1):
        gl, gg = _plane_less(L, n, c), _plane_great(L, R, n, c)
        gl_t, gg_t = _plane_less(L, c, n), _plane_great(L, R, c, n)
        UU = np.outer(U, U)
        assert np.allclose(Sl[c], UU * gl ** 2 * gg_t.T, atol=1e-15, rtol=0)
        assert np.allclose(Sg[c], UU * gg ** 2 * gl_t.T, atol=1e-15, rtol=0)


def test_equal_time_sign():
    """At equal times a greater function has i*X^> positive semidefinite and a
    lesser one has -i*X^< positive semidefinite (true of G: i G^> = 1 - rho,
    -i G^< = rho).  The self-energy of Eq. (SE) inherits both."""
    _, _, t, order, L, R = _free(3, 4)
    U = np.array([1.0, 2.0, 0.5])
    for n in (0, 5, 11):
        Sl, Sg = oracle.sigma_row(oracle.local_U4(U), n, L, R)
        Xg = 1j * Sg[n]
        Xl = -1j * Sl[n]
        assert np.allclose(Xg, Xg.conj().T, atol=1e-14)
        assert np.allclose(Xl, Xl.conj().T, atol=1e-14)
        assert np.linalg.eigvalsh(Xg).min() > -1e-13
        assert np.linalg.eigvalsh(Xl).min() > -1e-13
        assert np.linalg.eigvalsh(Xg).max() > 1e-3


def test_antihermitian_symmetry_of_sigma():
    """Sigma^<>(t,t') = -Sigma^<>(t',t)^+ (same symmetry as G, Sec. 2), so
    every equal-time block is anti-Hermitian."""
    _, _, t, order, L, R = _free(3, 8)
    U = np.array([1.1, 0.3, 0.8])
    U4 = oracle.local_U4(U)
    n = 10
    for c in (0, 3, 10):
        Sl_c, Sg_c = oracle.sigma_row(U4, c, L, R)
        # Sigma(t_c, t_c) is anti-Hermitian
        assert np.allclose(Sl_c[c], -Sl_c[c].conj().T, atol=1e-14)
        assert np.allclose(Sg_c[c], -Sg_c[c].conj().T, atol=1e-14)
    # A general real tensor with the 8-fold symmetry of Coulomb integrals in
    # chemists' order (ij|kl) = (ji|kl) = (ij|lk) = (kl|ij) keeps the
    # equal-time block anti-Hermitian as well.
    rng = np.random.default_rng(3)
    A = rng.normal(size=(3, 3, 3, 3))
    perms = [(0, 1, 2, 3), (1, 0, 2, 3), (0, 1, 3, 2), (1, 0, 3, 2),
             (2, 3, 0, 1), (3, 2, 0, 1), (2, 3, 1, 0), (3, 2, 1, 0)]
    U4g = sum(A.transpose(p) for p in perms)
    Sl_g, Sg_g = oracle.sigma_row(U4g, n, L, R)
    scale = max(np.abs(Sl_g[n]).max(), np.abs(Sg_g[n]).max())
    assert np.abs(Sl_g[n] + Sl_g[n].conj().T).max() < 1e-13 * scale
    assert np.abs(Sg_g[n] + Sg_g[n].conj().T).max() < 1e-13 * scale


def test_sigma_scales_quadratically_in_U():
    _, _, t, order, L, R = _free(2, 2)
    U = np.array([0.7, 1.3])
    a = oracle.sigma_row(oracle.local_U4(U), 6, L, R)
    b = oracle.sigma_row(oracle.local_U4(3.0 * U), 6, L, R)
    assert np.allclose(b[0], 9.0 * a[0], atol=1e-14, rtol=1e-14)
    assert np.allclose(b[1], 9.0 * a[1], atol=1e-14, rtol=1e-14)
