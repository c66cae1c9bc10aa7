"""Pins for the oracle's adaptive time stepping (Sec. 3.1): error integrals
of the variable-step Adams pair against textbook constants, tolerance
proportionality against the exact non-interacting solution, recovery from
rejected steps, agreement with the independent fixed-grid stepper, and
conservation laws."""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "adams_error_constants.txt")
tri = W.tri_index


def _golden():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                q, a, b, c, d = (int(x) for x in line.split())
                rows[q] = (a / b, c / d)
    return rows


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 6])
def test_error_integrals_match_textbook_constants(q):
    """On a uniform grid, E_p / q! and E_c / q! are the Adams-Bashforth and
    implicit Adams error constants times h^{q+1}; the Milne constant is
    C_AM / (C_AB - C_AM)."""
    hh = 0.37
    t = hh * np.arange(12)
    n = 9
    Ep, Ec, C = oracle.adams_error_integrals(t, n, q)
    cab, cam = _golden()[q]
    scale = math.factorial(q) * hh ** (q + 1)
    assert abs(Ep / scale - cab) < 1e-13 and abs(Ec / scale - cam) < 1e-13
    assert abs(C - cam / (cab - cam)) < 1e-13


def test_error_integrals_on_nonuniform_nodes():
    """q = 1 pairs explicit and implicit Euler on any step: C = -1/2.  For
    q = 2 the integrals are the closed forms of int (t - t_{n-1})(t - t_{n-2})
    and int (t - t_n)(t - t_{n-1}) over [t_{n-1}, t_n]."""
    t, _ = W.grid(12, 0.1, 0.5, 3)
    for n in (3, 7, 11):
        assert abs(oracle.adams_error_integrals(t, n, 1)[2] + 0.5) < 1e-14
        h, h1 = t[n] - t[n - 1], t[n - 1] - t[n - 2]
        Ep, Ec, _ = oracle.adams_error_integrals(t, n, 2)
        assert abs(Ep - (h ** 3 / 3 + h1 * h ** 2 / 2)) < 1e-14
        assert abs(Ec - (-h ** 3 / 6)) < 1e-14


def _free_case(M=2, seed=1):
    h = W.goe_h(M, seed)
    return h, W.half_filled_rho(h)


def test_free_run_error_follows_the_tolerance():
    """U = 0: the exact solution is the free propagator.  The global error
    falls with the tolerance (about in proportion), the step count grows and
    the order rises above 1."""
    h, rho = _free_case()
    errs, steps = [], []
    for rtol in (1e-5, 1e-7, 1e-9):
        r = oracle.run_controlled(h, np.zeros(2), W.site_potential(2), None, rho, rtol, rtol * 1e-2, 0.01, 3.0, 2000)
        assert r["status"] == 0 and abs(r["t"][-1] - 3.0) < 1e-12
        L, R = W.free_triangles(h, rho, r["t"])
        err = max(np.abs(r["L"] - L).max(), np.abs(r["R"] - R).max())
        assert err < 30 * rtol
        errs.append(err)
        steps.append(r["n"])
        assert r["q"].max() >= 5
        assert np.all(r["korder"][1:] == 5)  # fixed history orders
    assert errs[0] > 10 * errs[1] > 100 * errs[2]
    assert steps[0] < steps[1] < steps[2]


def test_rejected_steps_recover():
    """A far too large first step fails the error test, is retried smaller,
    and the run still meets the tolerance."""
    h, rho = _free_case(M=3, seed=4)
    r = oracle.run_controlled(h, np.zeros(3), W.site_potential(3), None, rho, 1e-7, 1e-9, 1.0, 2.0, 2000)
    assert r["status"] == 0
    assert r["stats"][1] >= 1  # error-test failures
    L, _ = W.free_triangles(h, rho, r["t"])
    assert np.abs(r["L"] - L).max() < 3e-6
    dt = np.diff(r["t"])
    assert dt[0] < 0.05 and dt.max() > 10 * dt[0]  # the steps grow again


def test_interacting_run_matches_fixed_grid_stepper():
    """Second Born with a pulse: the controlled run (rtol 1e-9) and the
    fixed-grid integral-form stepper on 121 uniform points agree at the final
    time within the latter's discretisation error; particle number and the
    anti-Hermitian diagonal are kept along the run."""
    h = W.chain_h(2)
    rho = W.half_filled_rho(h)
    U = np.ones(2)
    v = W.site_potential(2)
    pulse = {"E0": 0.5, "t0": 1.0, "sigma": 0.3, "omega": 2.0}
    r = oracle.run_controlled(h, U, v, pulse, rho, 1e-9, 1e-11, 0.01, 2.0, 2000)
    n = r["n"]
    last = r["L"][tri(n - 1, n - 1)]
    N = 121
    tt, oo = W.uniform_grid(N, 2.0 / (N - 1), 5)
    L0, R0, F0 = oracle.initial_rhs(tt, oo, h, U, v, pulse, rho)
    Lf = np.zeros((W.tri_size(N), 2, 2), np.complex128)
    Rf = np.zeros_like(Lf)
    Lf[0], Rf[0] = L0[0], R0[0]
    Lf, _, _ = oracle.run(tt, oo, h, U, v, pulse, 2, Lf, Rf, {0: F0}, 1, N, nthreads=4)
    assert np.abs(Lf[tri(N - 1, N - 1)] - last).max() < 5e-7
    n0 = np.trace(rho).real
    for k in range(1, n):
        D = r["L"][tri(k, k)]
        assert abs(np.trace(-1j * D).real - n0) < 1e-12
        assert np.abs(D + D.conj().T).max() < 1e-14


def test_dense_interaction_and_adaptive_history_orders():
    """The controller with a dense Coulomb tensor and history orders chosen
    per interval (Sec. 3.2) converges in the tolerance: rtol 1e-6 and 1e-8
    agree to the looser one's accuracy."""
    M = 2
    h = W.goe_h(M, 2)
    rho = W.half_filled_rho(h)
    U4 = W.coulomb_tensor(M, 3, U=1.0)
    v = W.site_potential(M)
    out = []
    for rtol in (1e-6, 1e-8):
        r = oracle.run_controlled(h, None, v, None, rho, rtol, rtol * 1e-2, 0.01, 1.5, 2000, K_sel=6, U4=U4)
        assert r["status"] == 0
        assert len(set(r["korder"][7:])) > 1
        out.append(r["L"][tri(r["n"] - 1, r["n"] - 1)])
    assert np.abs(out[0] - out[1]).max() < 1e-5


def test_replay_reproduces_the_run():
    """Replaying a run's accepted points and step orders gives the same rows
    bitwise (rejected attempts leave nothing behind)."""
    h = W.chain_h(2)
    rho = W.half_filled_rho(h)
    a = oracle.run_controlled(h, np.ones(2), W.site_potential(2), None, rho, 1e-7, 1e-9, 0.01, 1.0, 300)
    assert a["stats"][1] > 0  # the run had rejected attempts
    b = oracle.run_controlled(h, np.ones(2), W.site_potential(2), None, rho, 1e-7, 1e-9, 0.01, 1.0, 300,
                              replay=(a["t"], a["q"]))
    assert b["status"] == 0 and b["n"] == a["n"] and b["stats"][1] == 0
    assert np.array_equal(a["t"], b["t"]) and np.array_equal(a["L"], b["L"]) and np.array_equal(a["R"], b["R"])
