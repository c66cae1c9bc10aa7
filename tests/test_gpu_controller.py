"""GPU checks of the adaptive time stepping (Sec. 3.1, kbe_run_controlled)
against the oracle's controlled runs.

Decisions: the same number of steps, failures, step orders and history
orders.  Step sizes follow from the error estimate ||y - y(0)||, a
difference of two values that agree to about rtol, so its relative
precision is about eps / rtol; each step factor inherits that, and the
deviations add up along the run.  Two correct evaluations therefore place
the points apart by up to about n eps / rtol of t after n steps; the test
allows 10 n eps / rtol (``_t_tol``).  The rows may then differ by what the
solution changes over the measured shift of their two time arguments:
the run's largest |dG/dt| (divided differences of the oracle's rows along
both arguments) times the measured drift of the points, with a factor 4
for the curvature between grid points, plus 1e-12 of the rows for the
arithmetic (``_row_bound``).  Arithmetic: the oracle replaying the device's
accepted points and orders gives the device's rows within 1e-12."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12
tri = W.tri_index


@pytest.fixture(scope="module")
def kbe():
    import torch
    from paper_2405_08737_gb300 import build as B
    B.build()
    import paper_2405_08737_gb300 as K
    torch.cuda.set_device(0)
    return K


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _t_tol(n, rtol):
    """Relative bound on the drift of the accepted points after n steps."""
    return 10.0 * n * np.finfo(float).eps / rtol


def _row_bound(L, t, t_other):
    """Absolute bound on |L_gpu - L_oracle| implied by the shift of the
    accepted points between the two runs (t: the oracle's, t_other: the
    device's): 4 x max |dG/dt| over both time arguments x the largest shift
    of a point, twice (both arguments of a block move), plus 1e-12 of the
    rows."""
    n = len(t)
    drift = float(np.abs(np.asarray(t_other) - np.asarray(t)).max())
    dmax = 0.0
    for j in range(1, n):
        p, q = W.tri_size(j), W.tri_size(j - 1)
        dt = t[j] - t[j - 1]
        # along the first argument: (j, c) against (j-1, c), c < j
        dmax = max(dmax, float(np.abs(L[p:p + j] - L[q:q + j]).max()) / dt)
        # along the second argument: (j, c) against (j, c-1), c = 1..j
        dc = np.diff(t[: j + 1])
        dmax = max(dmax, float((np.abs(L[p + 1:p + j + 1] - L[p:p + j]).max(axis=(1, 2)) / dc).max()))
    return 4.0 * 2.0 * dmax * drift + 1e-12 * float(np.abs(L).max()), drift, dmax


CASES = {  # name: (M, kind, U, dense, pulse, rtol, t_end, K_sel)
    "dimer_pulse": (2, "chain", 1.0, False, True, 1e-7, 1.5, 0),
    "goe3": (3, "goe", 1.5, False, False, 1e-6, 1.2, 0),
    "dense4_adaptive_orders": (4, "goe", 1.0, True, False, 1e-6, 1.0, 6),
}


def _model(M, kind, U, dense, pulse_on, seed=3):
    h = W.chain_h(M) if kind == "chain" else W.goe_h(M, seed)
    v = W.site_potential(M)
    pulse = {"E0": 0.5, "t0": 0.6, "sigma": 0.25, "omega": 2.0} if pulse_on else None
    Uv = np.full(M, U)
    U4 = W.coulomb_tensor(M, seed, U=U) if dense else None
    return h, Uv, U4, v, pulse


def _both(kbe, name, precision="fp64", n_max=400):
    M, kind, U, dense, pulse_on, rtol, t_end, K_sel = CASES[name]
    h, Uv, U4, v, pulse = _model(M, kind, U, dense, pulse_on)
    rho = W.half_filled_rho(h)
    o = oracle.run_controlled(h, None if dense else Uv, v, pulse, rho, rtol, rtol * 1e-2, 0.01, t_end, n_max,
                              K_sel=K_sel, U4=U4)
    ctx = kbe.Context(M, n_max)
    ctx.set_model(h, Uv, v, pulse)
    if dense:
        ctx.set_interaction(U4)
    g = ctx.run_controlled(rho, rtol, rtol * 1e-2, 0.01, t_end, K_sel=K_sel, precision=precision)
    ctx.sync_status()
    return o, g, ctx


@pytest.mark.parametrize("name", sorted(CASES))
def test_controlled_run_matches_oracle(kbe, name):
    o, g, ctx = _both(kbe, name)
    assert o["status"] == 0 and g["status"] == kbe.KBE_OK
    assert g["n"] == o["n"] and g["stats"] == o["stats"], (g["stats"], o["stats"])
    assert np.array_equal(g["q"], o["q"]) and np.array_equal(g["korder"], o["korder"])
    M, kind, U, dense, pulse_on, rtol, t_end, K_sel = CASES[name]
    tt = _t_tol(o["n"], rtol)
    assert np.abs(g["t"] - o["t"]).max() <= tt * o["t"][-1]
    assert g["q"].max() >= 3 and g["stats"][4] > 0
    p = W.tri_size(o["n"])
    Lg, Rg = g["L"][:p].cpu().numpy(), g["R"][:p].cpu().numpy()
    for name, a, b in (("L", Lg, o["L"]), ("R", Rg, o["R"])):
        bound, drift, dmax = _row_bound(b, o["t"], g["t"])
        err = float(np.abs(a - b).max())
        assert err <= bound, (name, err, bound, drift, dmax)
    # the oracle on the device's accepted points and orders: the same rows
    h, Uv, U4, v, pulse = _model(M, kind, U, dense, pulse_on)
    r = oracle.run_controlled(h, None if dense else Uv, v, pulse, W.half_filled_rho(h), rtol, rtol * 1e-2, 0.01,
                              t_end, 400, K_sel=K_sel, U4=U4, replay=(g["t"], g["q"]))
    assert r["status"] == 0 and r["n"] == g["n"] and np.array_equal(r["korder"], g["korder"])
    assert _rel(Lg, r["L"]) < TOL and _rel(Rg, r["R"]) < TOL
    ctx.close()


def test_context_grid_is_the_accepted_grid(kbe):
    """After the run the context holds the accepted grid: a history slice of
    the last row matches the oracle's slice on that grid."""
    import torch
    o, g, ctx = _both(kbe, "goe3")
    n = g["n"] - 1
    Sl = torch.zeros((n + 1, ctx.M, ctx.M), dtype=torch.complex128, device="cuda")
    Sg = torch.zeros_like(Sl)
    ctx.selfenergy_slice(n, g["L"], g["R"], Sl, Sg)
    out = torch.zeros((2, n + 1, ctx.M, ctx.M), dtype=torch.complex128, device="cuda")
    ctx.history_slice(n, g["L"], g["R"], Sl, Sg, out)
    ctx.sync_status()
    L, R = g["L"][:W.tri_size(n + 1)].cpu().numpy(), g["R"][:W.tri_size(n + 1)].cpu().numpy()
    ol, og = oracle.sigma_row(oracle.local_U4(np.full(3, 1.5)), n, L, R)
    ref = oracle.history_slice(g["t"], g["korder"], n, L, R, ol, og)
    assert _rel(out.cpu().numpy(), ref) < TOL
    ctx.close()


def test_free_run_against_the_exact_propagator(kbe):
    M = 4
    h = W.goe_h(M, 7)
    rho = W.half_filled_rho(h)
    ctx = kbe.Context(M, 600)
    ctx.set_model(h, np.zeros(M), W.site_potential(M), None)
    for rtol in (1e-6, 1e-9):
        g = ctx.run_controlled(rho, rtol, rtol * 1e-2, 0.01, 3.0)
        L, R = W.free_triangles(h, rho, g["t"])
        p = W.tri_size(g["n"])
        err = max(np.abs(g["L"][:p].cpu().numpy() - L).max(), np.abs(g["R"][:p].cpu().numpy() - R).max())
        assert err < 30 * rtol, (rtol, err)
    ctx.close()


def test_split_precision_controlled_run(kbe):
    """With the split contraction the run takes nearly the same steps and
    stays within the tolerance's accuracy of the FP64 run."""
    o, g, ctx = _both(kbe, "dimer_pulse", precision="split")
    assert g["status"] == kbe.KBE_OK and abs(g["n"] - o["n"]) <= 2
    a = g["L"][tri(g["n"] - 1, g["n"] - 1)].cpu().numpy()
    b = o["L"][tri(o["n"] - 1, o["n"] - 1)]
    assert np.abs(a - b).max() < 1e-5
    ctx.close()


def test_double_float_controlled_run(kbe):
    """With the double-float contraction (its rounding about 2^6 times
    FP64's) the controller takes the oracle's decisions: the same step count,
    statistics and orders, the accepted points within 64 times the FP64
    drift bound, and the oracle replaying the device's points and orders
    gives the same rows to 1e-11."""
    o, g, ctx = _both(kbe, "goe3", precision="df64")
    M, kind, U, dense, pulse_on, rtol, t_end, K_sel = CASES["goe3"]
    assert g["status"] == kbe.KBE_OK and g["n"] == o["n"] and g["stats"] == o["stats"]
    assert np.array_equal(g["q"], o["q"])
    assert np.abs(g["t"] - o["t"]).max() <= 64 * _t_tol(o["n"], rtol) * o["t"][-1]
    h, Uv, U4, v, pulse = _model(M, kind, U, dense, pulse_on)
    r = oracle.run_controlled(h, Uv, v, pulse, W.half_filled_rho(h), rtol, rtol * 1e-2, 0.01, t_end, 400,
                              K_sel=K_sel, replay=(g["t"], g["q"]))
    p = W.tri_size(g["n"])
    assert _rel(g["L"][:p].cpu().numpy(), r["L"]) < 1e-11 and _rel(g["R"][:p].cpu().numpy(), r["R"]) < 1e-11
    ctx.close()


def test_controlled_run_errors_and_full_storage(kbe):
    M = 2
    h = W.chain_h(M)
    rho = W.half_filled_rho(h)
    ctx = kbe.Context(M, 12)
    with pytest.raises(kbe.KBEError) as e:
        ctx.run_controlled(rho, 1e-6, 1e-8, 0.01, 1.0)
    assert e.value.status == kbe.KBE_ESTATE  # no model
    ctx.set_model(h, np.ones(M), W.site_potential(M), None)
    with pytest.raises(kbe.KBEError) as e:
        ctx.run_controlled(rho, 1e-6, 0.0, 0.01, 1.0)
    assert e.value.status == kbe.KBE_EINVAL
    with pytest.raises(kbe.KBEError) as e:
        ctx.run_controlled(rho, 1e-6, 1e-8, 0.01, 1.0, q_max=13)
    assert e.value.status == kbe.KBE_EINVAL
    g = ctx.run_controlled(rho, 1e-8, 1e-10, 0.01, 5.0)  # 12 rows cannot reach t = 5
    assert g["status"] == kbe.KBE_ERANGE and g["n"] == 12 and g["t"][-1] < 5.0
    o = oracle.run_controlled(h, np.ones(M), W.site_potential(M), None, rho, 1e-8, 1e-10, 0.01, 5.0, 12)
    assert o["status"] == 1 and np.abs(g["t"] - o["t"]).max() <= _t_tol(12, 1e-8) * o["t"][-1]
    ctx.sync_status()
    ctx.close()
