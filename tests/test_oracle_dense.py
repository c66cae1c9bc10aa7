"""Pins for the oracle with a general four-index interaction: the self-energy
of Eq. (SE) and the Fock matrix of Eq. (eps) for a dense real tensor, and
whole runs built on them.

Closed forms used here (derived by hand from Eq. SE / Eq. eps):
  * product tensor U_pqrs = a_p b_q c_r d_s in the first factor and
    a'_p b'_q c'_r d'_s in UEx:  every index sum separates into bilinear forms,
      Sigma_ij = a_i a'_j (d'^T G' c) [2 (b^T G b')(d^T G c') - (b^T G c')(d^T G b')],
    with G = G^<>(t_n,t_c), G' = G^><(t_c,t_n); a sum of product tensors gives
    the sum over all ordered pairs.  Each of the eight index slots carries
    its own vector, so a wrong index anywhere changes the result.
  * density-density tensor U_pqrs = delta_pq delta_rs V_pr (extended Hubbard):
      Sigma_ij = 2 G_ij [V (G o G'^T) V]_ij - sum_bd V_id V_jb G_ib G'_bd G_dj,
    the second-order bubble (spin factor 2) minus the second-order exchange;
      eps_ij = h_ij + i V_ij G^<_ji - 2 i delta_ij sum_b V_ib G^<_bb,
    Hartree (spin factor 2) and exchange.
"""
import numpy as np
import pytest

import oracle
import workloads as W

tri = W.tri_index


def _free(M, seed, n_t=12):
    h = W.goe_h(M, seed)
    rho0 = W.half_filled_rho(h)
    t, order = W.grid(n_t, 0.1, 0.3, seed)
    L, R = W.free_triangles(h, rho0, t)
    return h, rho0, t, order, L, R


def _less(L, r, c):
    return L[tri(r, c)] if r >= c else -L[tri(c, r)].conj().T


def _great(L, R, r, c):
    return R[tri(r, c)] + L[tri(r, c)] if r >= c else -(R[tri(c, r)] + L[tri(c, r)]).conj().T


def _blocks(L, R, n, c, s):
    """(G, G') = (G^s(t_n,t_c), G^s'(t_c,t_n)), s' the other component."""
    if s == 0:
        return _less(L, n, c), _great(L, R, c, n)
    return _great(L, R, n, c), _less(L, c, n)


@pytest.mark.parametrize("M,rank,seed", [(2, 1, 0), (3, 2, 1), (4, 3, 2)])
def test_sigma_product_tensor_closed_form(M, rank, seed):
    rng = np.random.default_rng(seed)
    vecs = rng.standard_normal((rank, 4, M))  # [r][a,b,c,d][index]
    U4 = sum(np.einsum("p,q,r,s->pqrs", *vecs[r]) for r in range(rank))
    _, _, t, order, L, R = _free(M, 20 + seed)
    n = 9
    Sl, Sg = oracle.sigma_row(U4, n, L, R)
    for c in range(n + 1):
        for s, S in ((0, Sl), (1, Sg)):
            G, Gp = _blocks(L, R, n, c, s)
            ref = np.zeros((M, M), np.complex128)
            for r in range(rank):
                a, b, cc, d = vecs[r]
                for q in range(rank):
                    a2, b2, c2, d2 = vecs[q]
                    f = (d2 @ Gp @ cc) * (2 * (b @ G @ b2) * (d @ G @ c2) - (b @ G @ c2) * (d @ G @ b2))
                    ref += f * np.outer(a, a2)
            scale = max(np.abs(ref).max(), 1e-300)
            assert np.abs(S[c] - ref).max() < 1e-13 * scale, (c, s)


@pytest.mark.parametrize("M,seed", [(2, 3), (3, 4), (5, 5)])
def test_sigma_density_density_second_born(M, seed):
    rng = np.random.default_rng(seed)
    A = rng.uniform(0.2, 1.5, (M, M))
    V = (A + A.T) / 2
    U4 = np.einsum("pq,rs,pr->pqrs", np.eye(M), np.eye(M), V)
    _, _, t, order, L, R = _free(M, 30 + seed)
    n = 10
    Sl, Sg = oracle.sigma_row(U4, n, L, R)
    for c in (0, 4, n):
        for s, S in ((0, Sl), (1, Sg)):
            G, Gp = _blocks(L, R, n, c, s)
            direct = 2 * G * (V @ (G * Gp.T) @ V)
            exch = np.einsum("id,jb,ib,bd,dj->ij", V, V, G, Gp, G)
            ref = direct - exch
            assert np.abs(S[c] - ref).max() < 1e-13 * np.abs(ref).max(), (c, s)


def _rand_lnn(M, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    return 1j * (X @ X.conj().T) / M  # i * (positive Hermitian), like G^<(t,t)


@pytest.mark.parametrize("M,seed", [(2, 0), (3, 1), (6, 2)])
def test_fock_product_tensor_closed_form(M, seed):
    rng = np.random.default_rng(40 + seed)
    a, b, c, d = rng.standard_normal((4, M))
    U4 = np.einsum("p,q,r,s->pqrs", a, b, c, d)
    h = W.goe_h(M, seed)
    G = _rand_lnn(M, seed)
    eps = oracle.fock(0.3, h, None, W.site_potential(M), None, G, U4=U4)
    ref = h + 1j * ((c @ G @ b) * np.outer(a, d) - 2 * (c @ G @ d) * np.outer(a, b))
    assert np.abs(eps - ref).max() < 1e-14 * np.abs(ref).max()


def test_fock_density_density_hartree_fock_and_local_reduction():
    M = 4
    rng = np.random.default_rng(7)
    A = rng.uniform(0.2, 1.5, (M, M))
    V = (A + A.T) / 2
    U4 = np.einsum("pq,rs,pr->pqrs", np.eye(M), np.eye(M), V)
    h = W.chain_h(M)
    v = W.site_potential(M)
    pulse = {"E0": 0.7, "t0": 1.0, "sigma": 0.5, "omega": 2.0}
    G = _rand_lnn(M, 3)
    tt = 1.2
    eps = oracle.fock(tt, h, None, v, pulse, G, U4=U4)
    field = pulse["E0"] * np.exp(-(tt - 1.0) ** 2 / (2 * 0.25)) * np.cos(2.0 * tt)
    ref = h + field * np.diag(v) + 1j * V * G.T - 2j * np.diag(V @ np.diag(G))
    assert np.abs(eps - ref).max() < 1e-14 * np.abs(ref).max()
    # local tensor: the general formula gives the local model's eps = h + diag(U_a n_a)
    U = np.array([0.5, 1.0, 1.5, 2.0])
    G = 1j * np.real(-1j * G)  # anti-Hermitian, as an equal-time G^< is
    e_loc = oracle.fock(tt, h, U, v, pulse, G)
    e_gen = oracle.fock(tt, h, None, v, pulse, G, U4=oracle.local_U4(U))
    assert np.abs(e_loc - e_gen).max() < 1e-15
    n_a = np.real(np.diag(-1j * G))
    assert np.abs(e_loc - (h + field * np.diag(v) + np.diag(U * n_a))).max() < 1e-15


def _start(t, order, h, U, v, pulse, rho0, U4=None):
    M = h.shape[0]
    L0, R0, F0 = oracle.initial_rhs(t, order, h, U, v, pulse, rho0, U4=U4)
    N = len(t)
    L = np.zeros((W.tri_size(N), M, M), np.complex128)
    R = np.zeros_like(L)
    L[0], R[0] = L0[0], R0[0]
    return L, R, {0: F0}


def test_dense_run_with_local_tensor_is_the_local_run():
    M = 3
    h = W.chain_h(M)
    U = np.array([1.0, 2.0, 1.5])
    v = W.site_potential(M)
    pulse = {"E0": 0.5, "t0": 1.0, "sigma": 0.5, "omega": 2.0}
    t, order = W.grid(30, 0.05, 0.3, 2)
    rho0 = W.half_filled_rho(h)
    N = len(t)
    La, Ra, _ = oracle.run(t, order, h, U, v, pulse, 2, *_start(t, order, h, U, v, pulse, rho0), 1, N, nthreads=4)
    U4 = oracle.local_U4(U)
    Lb, Rb, _ = oracle.run(t, order, h, None, v, pulse, 2, *_start(t, order, h, None, v, pulse, rho0, U4), 1, N,
                           nthreads=4, U4=U4)
    assert np.abs(La - Lb).max() < 1e-14 * np.abs(La).max()
    assert np.abs(Ra - Rb).max() < 1e-14 * np.abs(Ra).max()


def test_dense_run_is_covariant_under_orbital_rotation():
    """G'(t,t') = O^T G(t,t') O for h' = O^T h O, U'_pqrs = U_abcd O_ap O_bq
    O_cr O_ds and rho0' = O^T rho0 O (no field): Eq. (SE) and Eq. (eps) are
    tensor contractions, and the quadrature acts on the time arguments only."""
    M = 3
    h = W.goe_h(M, 5)
    U4 = W.coulomb_tensor(M, 6, U=1.2)
    v = np.zeros(M)
    rng = np.random.default_rng(8)
    O, _ = np.linalg.qr(rng.standard_normal((M, M)))
    h2 = O.T @ h @ O
    U42 = np.einsum("abcd,ap,bq,cr,ds->pqrs", U4, O, O, O, O)
    t, order = W.grid(24, 0.08, 0.3, 9)
    rho0 = W.half_filled_rho(h)
    N = len(t)
    La, Ra, _ = oracle.run(t, order, h, None, v, None, 2, *_start(t, order, h, None, v, None, rho0, U4), 1, N,
                           nthreads=4, U4=U4)
    Lb, Rb, _ = oracle.run(t, order, h2, None, v, None, 2,
                           *_start(t, order, h2, None, v, None, O.T @ rho0 @ O, U42), 1, N, nthreads=4, U4=U42)
    La2 = np.einsum("ap,kab,bq->kpq", O, La, O)
    Ra2 = np.einsum("ap,kab,bq->kpq", O, Ra, O)
    assert np.abs(Lb - La2).max() < 1e-12 * np.abs(La).max()
    assert np.abs(Rb - Ra2).max() < 1e-12 * np.abs(Ra).max()
    # the correlated run differs from the free one
    Lf, _ = W.free_triangles(h, rho0, t)
    assert np.abs(La[tri(N - 1, N - 1)] - Lf[tri(N - 1, N - 1)]).max() > 1e-3


def test_dense_run_conserves_number_and_symmetry():
    M = 3
    h = W.chain_h(M)
    U4 = W.coulomb_tensor(M, 11, U=1.0)
    v = W.site_potential(M)
    pulse = {"E0": 0.8, "t0": 0.8, "sigma": 0.3, "omega": 2.0}
    t, order = W.grid(40, 0.05, 0.3, 12)
    rho0 = W.half_filled_rho(h)
    L, R, _ = oracle.run(t, order, h, None, v, pulse, 2, *_start(t, order, h, None, v, pulse, rho0, U4), 1, len(t),
                         nthreads=4, U4=U4)
    n0 = np.trace(rho0).real
    for n in (10, 25, 39):
        D = L[tri(n, n)]
        assert abs(np.trace(-1j * D).real - n0) < 1e-12
        assert np.abs(D + D.conj().T).max() < 1e-14
