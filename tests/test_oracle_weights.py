"""Pins for the oracle's quadrature weights (Sec. 3.2, Eq. weights and the
composite-row recursion), checked against mathematics the paper fixes rather
than against the oracle itself."""
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "adams_coefficients.txt")


def _golden():
    rows = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        kind, k, den, *num = line.split()
        rows[(kind, int(k))] = np.array([float(x) for x in num]) / float(den)
    return rows


def test_gauss_legendre_matches_numpy():
    # a library routine computes the same rule
    for q in (1, 2, 5, 12):
        x, w = oracle.gauss_legendre(q)
        xn, wn = np.polynomial.legendre.leggauss(q)
        idx = np.argsort(x)
        assert np.allclose(x[idx], xn, atol=1e-15, rtol=0)
        assert np.allclose(w[idx], wn, atol=1e-14, rtol=0)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_uniform_grid_gives_adams_moulton(k):
    """On a uniform grid the interpolatory rule through t_{n-k..n} over
    [t_{n-1},t_n] is the textbook k-step Adams-Moulton rule."""
    g = _golden()
    h = 0.37
    t = h * np.arange(12)
    n = 9
    w = oracle.lagrange_weights(t[n - k:n + 1], t[n - 1], t[n])
    assert np.allclose(w / h, g[("AM", k)], atol=1e-14, rtol=0)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_uniform_grid_extrapolation_gives_adams_bashforth(q):
    """The predictor's rule through t_{n-q..n-1} over [t_{n-1},t_n] is the
    textbook q-step Adams-Bashforth rule."""
    g = _golden()
    h = 0.21
    t = h * np.arange(12)
    n = 9
    w = oracle.lagrange_weights(t[n - q:n], t[n - 1], t[n])
    assert np.allclose(w / h, g[("AB", q)], atol=1e-13, rtol=0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_local_weights_exact_on_polynomials(seed):
    """Degree-k weights integrate (s - t_{l-1})^i exactly for i <= k on a
    seeded nonuniform grid, and miss degree k+1 (so the order is exactly k)."""
    t, order = W.grid(40, 0.05, 0.4, seed)
    for l in range(6, 40, 5):
        for k in range(1, 6):
            tau = t[l - k:l + 1]
            w = oracle.lagrange_weights(tau, t[l - 1], t[l])
            h = t[l] - t[l - 1]
            for i in range(k + 2):
                f = ((tau - t[l - 1]) / h) ** i
                exact = h / (i + 1)
                err = abs(w @ f - exact) / exact
                if i <= k:
                    assert err < 5e-13, (l, k, i, err)
                else:
                    assert err > 1e-9, (l, k, i, err)


def test_local_weights_match_vandermonde_solve():
    """The paper's route: solve V^T w = T with T_i = int (s - t_{l-k})^i."""
    t, order = W.grid(30, 0.05, 0.4, 7)
    for l in range(5, 30):
        for k in range(1, 6):
            tau = t[l - k:l + 1]
            x = tau - tau[0]
            V = np.vander(x, k + 1, increasing=True)  # V[j, i] = x_j^i
            a, b = t[l - 1] - tau[0], t[l] - tau[0]
            T = np.array([(b ** (i + 1) - a ** (i + 1)) / (i + 1) for i in range(k + 1)])
            w_lu = np.linalg.solve(V.T, T)
            w = oracle.lagrange_weights(tau, t[l - 1], t[l])
            assert np.allclose(w, w_lu, rtol=0, atol=1e-13 * (t[l] - t[l - 1]) * 10)


@pytest.mark.parametrize("seed", [0, 1])
def test_composite_row_properties(seed):
    t, order = W.grid(64, 0.05, 0.3, seed)
    K = int(order[1:].max())
    prev = None
    for n in range(64):
        row = oracle.composite_row(t, order, n)
        assert row.shape == (n + 1,)
        # integrates 1 exactly: sum_m w_{n,m} = t_n
        assert abs(row.sum() - t[n]) < 1e-14 * max(1.0, t[n]) * 10
        # integrates s exactly (every interval has order >= 1)
        assert abs(row @ t[: n + 1] - t[n] ** 2 / 2) < 1e-13 * max(1.0, t[n] ** 2)
        if prev is not None:
            # the paper's recursion: the new row differs from the previous one
            # only in the last k_opt+1 entries, by the local weights
            kap = min(order[n], n)
            loc = oracle.lagrange_weights(t[n - kap:n + 1], t[n - 1], t[n])
            rec = np.concatenate([prev, [0.0]])
            rec[n - kap:] += loc
            assert np.allclose(row, rec, rtol=0, atol=1e-15 * 10)
            # settled part: w_{n,i} = w_{n-1,i} for i < n - K
            if n - K > 0:
                assert np.array_equal(row[: n - K], prev[: n - K]) or np.allclose(
                    row[: n - K], prev[: n - K], rtol=0, atol=1e-16)
        prev = row


def test_composite_row_zero_and_first():
    t, order = W.grid(8, 0.1, 0.3, 3)
    assert np.array_equal(oracle.composite_row(t, order, 0), [0.0])
    h = t[1] - t[0]
    # first interval is always the trapezoid (kappa_1 = min(k_1, 1) = 1)
    assert np.allclose(oracle.composite_row(t, order, 1), [h / 2, h / 2], rtol=1e-15, atol=0)


def test_composite_rows_integrate_smooth_function():
    """Composite rows on a fine uniform grid with k = 2 integrate cos(s)
    over [0, t_n] with the expected third-order convergence."""
    errs = []
    for N in (41, 81, 161):
        t, order = W.uniform_grid(N, 2.0 / (N - 1), 2)
        row = oracle.composite_row(t, order, N - 1)
        errs.append(abs(row @ np.cos(t) - np.sin(2.0)))
    r1, r2 = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    assert 2.7 < r1 < 3.4 and 2.7 < r2 < 3.4, errs
