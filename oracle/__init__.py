"""TEST INFRASTRUCTURE ONLY: the FP64 CPU oracle for the KBE hot path.

A ctypes wrapper around ``kbe_oracle.cpp``, a plain, slow, obviously correct
C++ restatement of the paper's definitions (arXiv 2405.08737): the
interpolatory quadrature weights (Sec. 3.2, Eq. weights), the second-Born
self-energy (Sec. 2, Eq. SE), the history integrals of Eq. (KBE2) and
Eq. (KBE1), and an integral-form Adams stepper built on them.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this module.  The
product package never imports it and shares no code with it.

Array conventions (input format only): two-time arrays are complex128
``[tri(N), M, M]`` holding the lower triangle ``r >= c`` at block
``r*(r+1)/2 + c``; ``L = G^<``, ``R = G^R`` with ``R(r,r) = -i*1``.
Self-energy rows are ``[n+1, M, M]``; history slices ``[2, n+1, M, M]``
with ``s = 0`` for ``<`` and ``s = 1`` for ``>``.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kbe_oracle.cpp")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile the oracle with g++ (portable flags, OpenMP)."""
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-fopenmp", "-fPIC",
                           "-shared", "-o", tmp, _SRC])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle %s rejected its arguments (rc=%d)" % (what, rc))


def threads_available():
    return int(lib().orc_threads_available())


def gauss_legendre(q):
    x = np.zeros(q)
    w = np.zeros(q)
    _check(lib().orc_gauss_legendre(ctypes.c_int(q), _p(x), _p(w)), "gauss_legendre")
    return x, w


def lagrange_weights(tau, lo, hi):
    """Weights of the interpolatory rule on nodes ``tau`` over [lo, hi]."""
    tau = _f64(tau)
    w = np.zeros(len(tau))
    _check(lib().orc_lagrange_weights(_p(tau), ctypes.c_int(len(tau) - 1),
                                      ctypes.c_double(lo), ctypes.c_double(hi), _p(w)),
           "lagrange_weights")
    return w


def composite_row(t, order, n):
    """w_{n,m}, m = 0..n (Sec. 3.2), as a direct sum over intervals."""
    t, order = _f64(t), _i32(order)
    row = np.zeros(n + 1)
    _check(lib().orc_composite_row(_p(t), _p(order), ctypes.c_int(n), _p(row)), "composite_row")
    return row


def local_U4(U):
    """Four-index tensor U_abcd = U_a delta_abcd of a local interaction."""
    U = np.asarray(U, dtype=np.float64)
    M = len(U)
    U4 = np.zeros((M, M, M, M))
    for a in range(M):
        U4[a, a, a, a] = U[a]
    return U4


def sigma_row(U4, n, L, R):
    """Row n of Eq. (SE) for a general real four-index tensor."""
    U4 = _f64(U4)
    M = U4.shape[0]
    L, R = _c128(L), _c128(R)
    Sl = np.zeros((n + 1, M, M), np.complex128)
    Sg = np.zeros((n + 1, M, M), np.complex128)
    _check(lib().orc_sigma_row(ctypes.c_int(M), ctypes.c_int(n), _p(U4), _p(L), _p(R),
                               _p(Sl), _p(Sg)), "sigma_row")
    return Sl, Sg


def history_slice(t, order, n, L, R, Sl, Sg, nthreads=1):
    """I^s(n,c) of Eq. (KBE2) for s in {<,>}, c = 0..n; [2, n+1, M, M]."""
    t, order = _f64(t), _i32(order)
    L, R, Sl, Sg = _c128(L), _c128(R), _c128(Sl), _c128(Sg)
    M = L.shape[-1]
    out = np.zeros((2, n + 1, M, M), np.complex128)
    _check(lib().orc_history_slice(ctypes.c_int(M), ctypes.c_int(n), _p(t), _p(order), _p(L), _p(R),
                                   _p(Sl), _p(Sg), _p(out), ctypes.c_int(nthreads)), "history_slice")
    return out


def history_columns(t, order, n, L, R, Sl, Sg, cols, nthreads=1):
    """The history slice at the listed output columns only; [2, len(cols), M, M]."""
    t, order = _f64(t), _i32(order)
    L, R, Sl, Sg = _c128(L), _c128(R), _c128(Sl), _c128(Sg)
    cols = _i32(cols)
    M = L.shape[-1]
    out = np.zeros((2, len(cols), M, M), np.complex128)
    _check(lib().orc_history_columns(ctypes.c_int(M), ctypes.c_int(n), _p(t), _p(order), _p(L), _p(R),
                                     _p(Sl), _p(Sg), _p(cols), ctypes.c_int(len(cols)), _p(out),
                                     ctypes.c_int(nthreads)), "history_columns")
    return out


def kbe1_slice(t, order, n, L, R, Sl, Sg, nthreads=1):
    """Lesser Eq. (KBE1) history integrals at (t_c, t_n), c = 0..n; [n+1, M, M]."""
    t, order = _f64(t), _i32(order)
    L, R, Sl, Sg = _c128(L), _c128(R), _c128(Sl), _c128(Sg)
    M = L.shape[-1]
    out = np.zeros((n + 1, M, M), np.complex128)
    _check(lib().orc_kbe1_slice(ctypes.c_int(M), ctypes.c_int(n), _p(t), _p(order), _p(L), _p(R),
                                _p(Sl), _p(Sg), _p(out), ctypes.c_int(nthreads)), "kbe1_slice")
    return out


def _pulse4(pulse):
    if pulse is None:  # no field: E0 = 0 (sigma = 1 keeps the envelope finite)
        return _f64([0.0, 0.0, 1.0, 0.0])
    return _f64([pulse["E0"], pulse["t0"], pulse["sigma"], pulse["omega"]])


def fock(t, h0, U, v, pulse, Lnn, U4=None):
    """Fock matrix of Eq. (eps) at time t from G^<(t,t) = Lnn: [M, M].  With
    ``U4`` (real [M, M, M, M], ``U4[i, a, b, j] = U_iabj``) the general
    tensor, else the local interaction ``U``."""
    h0, Lnn, v = _c128(h0), _c128(Lnn), _f64(v)
    M = h0.shape[0]
    Uv = _f64(U if U is not None else np.zeros(M))
    U4p = _p(_f64(U4)) if U4 is not None else None
    eps = np.zeros((M, M), np.complex128)
    _check(lib().orc_fock(ctypes.c_int(M), ctypes.c_double(t), _p(h0), _p(Uv), U4p, _p(v),
                          _p(_pulse4(pulse)), _p(Lnn), _p(eps)), "fock")
    return eps


def rhs_row(j, t, order, h0, U, v, pulse, L, R, nthreads=1, U4=None):
    """F^s(j,c) = -i(eps(t_j) G^s(j,c) + I^s(j,c)), c = 0..j; [2, j+1, M, M].
    ``U4`` selects the general tensor in Eq. (SE) and Eq. (eps)."""
    t, order = _f64(t), _i32(order)
    h0, L, R = _c128(h0), _c128(L), _c128(R)
    v = _f64(v)
    M = h0.shape[0]
    F = np.zeros((2, j + 1, M, M), np.complex128)
    if U4 is not None:
        _check(lib().orc_rhs_row_u4(ctypes.c_int(M), ctypes.c_int(j), _p(t), _p(order), _p(h0), _p(_f64(U4)),
                                    _p(v), _p(_pulse4(pulse)), _p(L), _p(R), _p(F), ctypes.c_int(nthreads)),
               "rhs_row_u4")
        return F
    U = _f64(U)
    _check(lib().orc_rhs_row(ctypes.c_int(M), ctypes.c_int(j), _p(t), _p(order), _p(h0), _p(U), _p(v),
                             _p(_pulse4(pulse)), _p(L), _p(R), _p(F), ctypes.c_int(nthreads)), "rhs_row")
    return F


def max_order(order, n_end):
    return max(1, int(np.max(order[1:n_end]))) if n_end > 1 else 1


def f_rows_needed(order, n_start, n_end):
    """Right-hand-side rows that the stepper needs on entry at n_start."""
    K = max_order(order, n_end)
    return list(range(max(0, n_start - K), n_start))


def _run_u4(t, order, hord, K_sel, h0, U4, v, pulse, P, L, R, F_rows, n_start, n_end, nthreads):
    t, order = _f64(t), _i32(order)
    h0, v = _c128(h0), _f64(v)
    M = h0.shape[0]
    L = np.array(L, dtype=np.complex128, copy=True)
    R = np.array(R, dtype=np.complex128, copy=True)
    need = f_rows_needed(order, n_start, n_end)
    Fin = np.concatenate([_c128(F_rows[j]).ravel() for j in need]) if need else np.zeros(1, np.complex128)
    I_last = np.zeros((2, n_end, M, M), np.complex128)
    hp = _p(hord) if hord is not None else None
    _check(lib().orc_run_u4(ctypes.c_int(M), ctypes.c_int(n_start), ctypes.c_int(n_end), _p(t), _p(order), hp,
                            ctypes.c_int(K_sel), _p(h0), _p(_f64(U4)), _p(v), _p(_pulse4(pulse)), ctypes.c_int(P),
                            _p(L), _p(R), _p(Fin), _p(I_last), ctypes.c_int(nthreads)), "run_u4")
    return L, R, I_last


def run(t, order, h0, U, v, pulse, P, L, R, F_rows, n_start, n_end, nthreads=1, U4=None):
    """KBE steps n_start..n_end-1.  ``L``/``R`` are triangles of n_end rows,
    filled for rows < n_start; ``F_rows`` maps each row j of
    ``f_rows_needed`` to its [2, j+1, M, M] right-hand side.  Returns
    (L, R, I_last) with the history slice of the last row.  ``U4`` selects
    the general tensor in Eq. (SE) and Eq. (eps) (``U`` is then unused)."""
    if U4 is not None:
        return _run_u4(t, order, None, 0, h0, U4, v, pulse, P, L, R, F_rows, n_start, n_end, nthreads)
    t, order = _f64(t), _i32(order)
    h0 = _c128(h0)
    U, v = _f64(U), _f64(v)
    M = h0.shape[0]
    L = np.array(L, dtype=np.complex128, copy=True)
    R = np.array(R, dtype=np.complex128, copy=True)
    need = f_rows_needed(order, n_start, n_end)
    Fin = np.concatenate([_c128(F_rows[j]).ravel() for j in need]) if need else np.zeros(1, np.complex128)
    I_last = np.zeros((2, n_end, M, M), np.complex128)
    _check(lib().orc_run(ctypes.c_int(M), ctypes.c_int(n_start), ctypes.c_int(n_end), _p(t), _p(order),
                         _p(h0), _p(U), _p(v), _p(_pulse4(pulse)), ctypes.c_int(P), _p(L), _p(R),
                         _p(Fin), _p(I_last), ctypes.c_int(nthreads)), "run")
    return L, R, I_last


def run_adaptive(t, order, hord, K_sel, h0, U, v, pulse, P, L, R, F_rows, n_start, n_end, nthreads=1, U4=None):
    """``run`` with the history quadrature orders chosen per step (Sec. 3.2)
    up to K_sel; ``hord`` gives the orders of intervals 1..n_start-1.  Returns
    (L, R, I_last, hord) with the chosen orders filled in up to n_end-1."""
    if U4 is not None:
        ho = np.zeros(len(t), np.int32)
        ho[: len(hord)] = np.asarray(hord, np.int32)[: len(t)]
        out = _run_u4(t, order, ho, K_sel, h0, U4, v, pulse, P, L, R, F_rows, n_start, n_end, nthreads)
        return out + (ho,)
    t, order = _f64(t), _i32(order)
    h0 = _c128(h0)
    U, v = _f64(U), _f64(v)
    M = h0.shape[0]
    L = np.array(L, dtype=np.complex128, copy=True)
    R = np.array(R, dtype=np.complex128, copy=True)
    ho = np.zeros(len(t), np.int32)
    ho[: len(hord)] = np.asarray(hord, np.int32)[: len(t)]
    need = f_rows_needed(order, n_start, n_end)
    Fin = np.concatenate([_c128(F_rows[j]).ravel() for j in need]) if need else np.zeros(1, np.complex128)
    I_last = np.zeros((2, n_end, M, M), np.complex128)
    _check(lib().orc_run_adaptive(ctypes.c_int(M), ctypes.c_int(n_start), ctypes.c_int(n_end), _p(t), _p(order),
                                  _p(ho), ctypes.c_int(K_sel), _p(h0), _p(U), _p(v), _p(_pulse4(pulse)),
                                  ctypes.c_int(P), _p(L), _p(R), _p(Fin), _p(I_last), ctypes.c_int(nthreads)),
           "run_adaptive")
    return L, R, I_last, ho


def choose_order(t, n, K, u):
    """Order chosen from test-integrand values u [kmax+1, M, M] at
    t_{n-kmax}..t_n, and the differences |I^(k) - I^(k-1)| (index k)."""
    t = _f64(t)
    u = _c128(u)
    M = u.shape[-1]
    diffs = np.zeros(13)
    k = ctypes.c_int()
    _check(lib().orc_choose_order(ctypes.c_int(M), ctypes.c_int(n), _p(t), ctypes.c_int(K), _p(u), _p(diffs),
                                  ctypes.byref(k)), "choose_order")
    return k.value, diffs


def select_order(t, n, K, L, R, Sl, Sg):
    """(chosen order, test-integrand values [kmax+1, M, M]) of row n."""
    t = _f64(t)
    L, R, Sl, Sg = _c128(L), _c128(R), _c128(Sl), _c128(Sg)
    M = L.shape[-1]
    kmax = min(K, n)
    u = np.zeros((kmax + 1, M, M), np.complex128)
    k = ctypes.c_int()
    _check(lib().orc_select_order(ctypes.c_int(M), ctypes.c_int(n), _p(t), ctypes.c_int(K), _p(L), _p(R), _p(Sl),
                                  _p(Sg), _p(u), ctypes.byref(k)), "select_order")
    return k.value, u


def order_test_integrand(n, l, L, R, Sl, Sg):
    """u(t_l) of row n (Sec. 3.2 order selection), [M, M]."""
    L, R, Sl, Sg = _c128(L), _c128(R), _c128(Sl), _c128(Sg)
    M = L.shape[-1]
    u = np.zeros((M, M), np.complex128)
    _check(lib().orc_test_integrand(ctypes.c_int(M), ctypes.c_int(n), ctypes.c_int(l), _p(L), _p(R), _p(Sl),
                                    _p(Sg), _p(u)), "test_integrand")
    return u


def run_tangent(t, order, h0, U, dU, v, pulse, dE0, P, L, R, F_rows, n_start, n_end, nthreads=1):
    """Forward-mode derivative of ``run`` along (dU, dE0).  Returns the value
    and derivative of the final diagonal block L(n_end-1, n_end-1)."""
    t, order = _f64(t), _i32(order)
    h0 = _c128(h0)
    U, dU, v = _f64(U), _f64(dU), _f64(v)
    M = h0.shape[0]
    L, R = _c128(L), _c128(R)
    need = f_rows_needed(order, n_start, n_end)
    Fin = np.concatenate([_c128(F_rows[j]).ravel() for j in need]) if need else np.zeros(1, np.complex128)
    Lv = np.zeros((M, M), np.complex128)
    Ld = np.zeros((M, M), np.complex128)
    _check(lib().orc_run_tangent(ctypes.c_int(M), ctypes.c_int(n_start), ctypes.c_int(n_end), _p(t),
                                 _p(order), _p(h0), _p(U), _p(dU), _p(v), _p(_pulse4(pulse)),
                                 ctypes.c_double(dE0), ctypes.c_int(P), _p(L), _p(R), _p(Fin), _p(Lv),
                                 _p(Ld), ctypes.c_int(nthreads)), "run_tangent")
    return Lv, Ld


def initial_rhs(t, order, h0, U, v, pulse, rho0, U4=None):
    """Row 0 of a run from an uncorrelated state: L(0,0) = i rho0,
    R(0,0) = -i, and its right-hand side (the history integral over a
    zero-length interval vanishes)."""
    h0 = _c128(h0)
    M = h0.shape[0]
    L0 = (1j * _c128(rho0)).reshape(1, M, M)
    R0 = (-1j * np.eye(M)).reshape(1, M, M).astype(np.complex128)
    F0 = rhs_row(0, t, order, h0, U, v, pulse, L0, R0, U4=U4)
    return L0, R0, F0

def run_controlled(h0, U, v, pulse, rho0, rtol, atol, dt0, t_end, n_max, q_max=12, k_hist=5, K_sel=0,
                   h_max=0.0, U4=None, replay=None):
    """Adaptive time stepping of Sec. 3.1 from the uncorrelated state rho0
    (L(0,0) = i rho0, R(0,0) = -i): variable-step, variable-order Adams
    (orders 1..q_max) with fixed-point iteration, WRMS error control
    (rtol, atol), step dt0 to start, history orders k_hist per interval (or
    chosen up to K_sel, Sec. 3.2).  Returns a dict with the accepted grid
    ``t``, step orders ``q``, history orders ``korder``, triangles ``L``,
    ``R`` of the accepted rows, ``stats`` = (steps, error-test failures,
    convergence failures, right-hand-side evaluations, reconstructed blocks)
    and the run ``status`` (0 reached t_end, 1 storage full, 2 failure).
    ``replay = (t, q)`` takes exactly those accepted points and step orders
    instead of choosing them."""
    h0 = _c128(h0)
    M = h0.shape[0]
    v = _f64(v)
    Uv = _f64(U if U is not None else np.zeros(M))
    U4p = _p(_f64(U4)) if U4 is not None else None
    L = np.zeros((_tri_size(n_max), M, M), np.complex128)
    R = np.zeros_like(L)
    L[0] = 1j * _c128(rho0)
    R[0] = -1j * np.eye(M)
    t = np.zeros(n_max)
    q = np.zeros(n_max, np.int32)
    ko = np.zeros(n_max, np.int32)
    n_rows = ctypes.c_int()
    stats = np.zeros(5, np.int32)
    opts = _f64([rtol, atol, dt0, h_max, t_end])
    iopts = _i32([q_max, k_hist, K_sel, n_max])
    tf = qf = None
    nf = 0
    if replay is not None:
        tf, qf = _f64(replay[0]), _i32(replay[1])
        nf = len(tf)
    rc = lib().orc_run_controlled(ctypes.c_int(M), _p(opts), _p(iopts), _p(h0), _p(Uv), U4p, _p(v),
                                  _p(_pulse4(pulse)), _p(L), _p(R), _p(t), _p(q), _p(ko), ctypes.byref(n_rows),
                                  _p(stats), _p(tf) if tf is not None else None,
                                  _p(qf) if qf is not None else None, ctypes.c_int(nf))
    if rc < 0:
        raise RuntimeError("oracle run_controlled: invalid arguments")
    n = n_rows.value
    return {"t": t[:n], "q": q[:n], "korder": ko[:n], "L": L[:_tri_size(n)], "R": R[:_tri_size(n)],
            "stats": tuple(int(x) for x in stats), "status": int(rc), "n": n}


def adams_error_integrals(t, n, q):
    """(E_p, E_c, C) of the order-q Adams pair at step n (without 1/q!)."""
    out = np.zeros(3)
    _check(lib().orc_adams_error_integrals(_p(_f64(t)), ctypes.c_int(n), ctypes.c_int(q), _p(out)),
           "adams_error_integrals")
    return tuple(out)


def _tri_size(n):
    return n * (n + 1) // 2



def run_thermal(t, order, h0, U, v, pulse, P, beta, N, ktau, GM, L0, R0, U4=None, nthreads=1):
    """Stepper runs with the thermal branch (Sec. 2, Eq. KBE3): rows 1..n_t-1
    from row 0 (L0, R0 blocks) and G^M on the uniform tau grid of N points
    (GM [N, M, M], tau_0 = 0+, tau_{N-1} = beta-).  Returns (L, R, Gm) with
    the mixed rows Gm [n_t, N, M, M]."""
    t, order = _f64(t), _i32(order)
    h0, v = _c128(h0), _f64(v)
    M = h0.shape[0]
    n_t = len(t)
    L = np.zeros((_tri_size(n_t), M, M), np.complex128)
    R = np.zeros_like(L)
    L[0], R[0] = _c128(L0), _c128(R0)
    Gm = np.zeros((n_t, N, M, M), np.complex128)
    Uv = _f64(U if U is not None else np.zeros(M))
    U4p = _p(_f64(U4)) if U4 is not None else None
    _check(lib().orc_run_thermal(ctypes.c_int(M), ctypes.c_int(n_t), _p(t), _p(order), _p(h0), _p(Uv), U4p, _p(v),
                                 _p(_pulse4(pulse)), ctypes.c_int(P), ctypes.c_double(beta), ctypes.c_int(N),
                                 ctypes.c_int(ktau), _p(_c128(GM)), _p(L), _p(R), _p(Gm), ctypes.c_int(nthreads)),
           "run_thermal")
    return L, R, Gm


def matsubara_conv(beta, ktau, S, GM):
    """int_0^beta S(s) G^M(s - tau_j) ds on the uniform tau grid (split at s = tau_j)."""
    S, GM = _c128(S), _c128(GM)
    N, M = S.shape[0], S.shape[-1]
    out = np.zeros_like(S)
    _check(lib().orc_matsubara_conv(ctypes.c_int(M), ctypes.c_int(N), ctypes.c_double(beta), ctypes.c_int(ktau),
                                    _p(S), _p(GM), _p(out)), "matsubara_conv")
    return out


def sigma_mixed(U4, n, Gm):
    """Sigma^|(t_n, tau_k) of Eq. (SE) from mixed rows Gm [rows, N, M, M]."""
    U4, Gm = _f64(U4), _c128(Gm)
    N, M = Gm.shape[1], Gm.shape[-1]
    out = np.zeros((N, M, M), np.complex128)
    _check(lib().orc_sigma_mixed(ctypes.c_int(M), ctypes.c_int(N), ctypes.c_int(n), _p(U4), _p(Gm), _p(out)),
           "sigma_mixed")
    return out
