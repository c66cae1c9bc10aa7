"""Closed forms of the non-interacting problem used to pin the oracle.

For a time-independent one-body matrix h = V diag(e) V^+ and a stationary
initial density rho0 = V diag(f) V^+, the non-interacting Green's functions
are finite sums of exponentials in t - t':
    G^<_ab(t,t') = i sum_k V_ak f_k V*_bk e^{-i e_k (t-t')},
    G^>_ab(t,t') = -i sum_k V_ak (1-f_k) V*_bk e^{-i e_k (t-t')},
    G^R_ab(t,t') = -i sum_k V_ak V*_bk e^{-i e_k (t-t')}      (t >= t').
The local second-Born self-energy built from them (Sec. 2, Eq. SE with
U_abcd = U_a delta_abcd) is again a sum of exponentials, so each history
integral of Eq. (KBE2) is a sum of integral_0^T e^{i w s} ds terms, which
are evaluated exactly here, independently of any quadrature weights.
"""
import numpy as np


def expint(om, T):
    """integral_0^T exp(i om s) ds, with the series near om = 0."""
    om = np.asarray(om, dtype=np.complex128)
    x = om * T
    small = np.abs(x) < 1e-5
    safe = np.where(small, 1.0, om)
    return np.where(small, T * (1 + 1j * x / 2 - x * x / 6 - 1j * x ** 3 / 24),
                    (np.exp(1j * x) - 1) / (1j * safe))


def spectral(h, rho0):
    e, V = np.linalg.eigh(h)
    f = np.real(np.einsum("ka,ab,bk->k", V.conj().T, rho0, V))
    return e, V, f


def history_closed_form(h, rho0, U, tn, tc):
    """Exact I^s(t_n, t_c), s in {<, >}, for the local second-Born self-energy
    of the non-interacting propagators; returns [2, M, M]."""
    e, V, f = spectral(h, rho0)
    M = len(e)
    gl = 1j * np.einsum("ak,k,bk->abk", V, f, V.conj())
    gg = -1j * np.einsum("ak,k,bk->abk", V, 1 - f, V.conj())
    # G^A_xb(tau, tc) = conj(G^R_bx(tc, tau)) = sum_k i V_xk V*_bk e^{-i e_k (tau - tc)}
    ga = 1j * np.einsum("xk,bk->xbk", V, V.conj())
    UU = np.outer(U, U)[:, :, None]
    # Sigma^>_ab = -U_a U_b (G^>_ab)^2 conj(G^<_ab), Sigma^< with < and > swapped
    Sg = -UU * np.einsum("abk,abl,abm->abklm", gg, gg, gl.conj()).reshape(M, M, -1)
    Sl = -UU * np.einsum("abk,abl,abm->abklm", gl, gl, gg.conj()).reshape(M, M, -1)
    Om = (e[:, None, None] + e[None, :, None] - e[None, None, :]).reshape(-1)
    SR = Sg - Sl
    out = np.zeros((2, M, M), np.complex128)
    # e^{-i Om (tn - tau)} e^{-i e_k (tau - tc)} = e^{-i Om tn + i e_k tc} e^{i (Om - e_k) tau}
    pre = np.exp(-1j * Om[:, None] * tn + 1j * e[None, :] * tc)
    ph1 = pre * expint(Om[:, None] - e[None, :], tn)
    ph2 = pre * expint(Om[:, None] - e[None, :], tc)
    for s, (gs, Ss) in enumerate([(gl, Sl), (gg, Sg)]):
        out[s] = (np.einsum("axK,xbk,Kk->ab", SR, gs, ph1)
                  + np.einsum("axK,xbk,Kk->ab", Ss, ga, ph2))
    return out


def free_lesser(h, rho0, t, tp):
    """G^<(t, t') = i e^{-iht} rho0 e^{iht'}."""
    e, V = np.linalg.eigh(h)
    A = V @ np.diag(np.exp(-1j * e * t)) @ V.conj().T
    B = V @ np.diag(np.exp(-1j * e * tp)) @ V.conj().T
    return 1j * A @ rho0 @ B.conj().T


def free_retarded(h, t, tp):
    e, V = np.linalg.eigh(h)
    return -1j * V @ np.diag(np.exp(-1j * e * (t - tp))) @ V.conj().T
