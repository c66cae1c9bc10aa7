"""GPU parity of the split-precision history slice (KBE_SPLIT_BF16).

Stated bound: 1e-8 relative in the max norm per slice (the error bound set
for the precision form) on physical histories; the scheme's own error is
about 1e-9.  A fixed-point scheme's error is relative to the magnitude of
the terms, not of their sum, so for random stress data (which cancel
heavily) the test bounds the error by 1e-8 times the slice of magnitudes
(the same contraction of |S|, |G| and |w|)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
TOL_SPLIT = 1e-8


@pytest.fixture(scope="module")
def kbe():
    import torch
    from paper_2405_08737_gb300 import build as B
    B.build()
    import paper_2405_08737_gb300 as K
    torch.cuda.set_device(0)
    return K


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _case(M, n_t, seed, kind):
    t, order = W.grid(n_t, 0.05, 0.4, seed)
    h = W.goe_h(M, seed)
    rho0 = W.half_filled_rho(h)
    if kind == "free":
        L, R = W.free_triangles(h, rho0, t)
    else:
        L, R = W.random_triangles(M, n_t, seed)
    return t, order, h, L, R


def _magnitude_slice(t, order, n, L, R, Sl, Sg):
    """max over the slice of sum_m |w| |Sigma| |G| (both terms): the scale of
    the terms a fixed-point contraction rounds against."""
    M = L.shape[-1]
    t_u = t.copy()
    wn = np.abs(oracle.composite_row(t, order, n))
    best = 0.0
    P = lambda r, c: np.abs(L[W.tri_index(r, c)]) if r >= c else np.abs(L[W.tri_index(c, r)]).T
    Q = lambda r, c: np.abs(R[W.tri_index(r, c)]) if r >= c else np.abs(R[W.tri_index(c, r)]).T
    aS = np.abs(Sg) + np.abs(Sl)
    for c in range(n + 1):
        wc = np.abs(oracle.composite_row(t, order, c))
        acc = np.zeros((M, M))
        for m in range(n + 1):
            acc += wn[m] * aS[m] @ (P(m, c) + Q(m, c))
        for m in range(c + 1):
            acc += wc[m] * aS[m] @ Q(c, m).T
        best = max(best, acc.max())
    del t_u
    return best


def _split_slice(kbe, M, n_t, t, order, h, n, Ld, Rd, Sl, Sg, path="planes"):
    import torch
    ctx = kbe.Context(M, n_t)
    ctx.set_grid(t, order)
    ctx.set_model(h, np.ones(M), W.site_potential(M), None)
    ctx.set_split_planes(path == "planes")
    out = torch.full((2, n + 1, M, M), float("nan"), dtype=torch.complex128, device="cuda")
    ctx.history_slice(n, Ld, Rd, _dev(Sl), _dev(Sg), out, precision="split")
    ctx.sync_status()
    res = out.cpu().numpy()
    ctx.close()
    return res


@pytest.mark.parametrize("path", ["planes", "fused"])
@pytest.mark.parametrize("M", [1, 2, 3, 4, 5, 8, 12, 16, 24, 32])
@pytest.mark.parametrize("kind", ["free", "random"])
def test_split_slice_matches_oracle(kbe, M, kind, path):
    n_t = 37 if M <= 16 else 21
    t, order, h, L, R = _case(M, n_t, 3 * M + (kind == "free"), kind)
    Ld, Rd = _dev(L), _dev(R)
    U = np.linspace(0.5, 1.5, M)
    for n in (0, 1, 2, 9, n_t - 1):
        if kind == "free":
            Sl, Sg = oracle.sigma_row(oracle.local_U4(U), n, L, R)
        else:
            Sl, Sg = W.random_rows(M, n, 5 * n + M)
        I = _split_slice(kbe, M, n_t, t, order, h, n, Ld, Rd, Sl, Sg, path)
        ref = oracle.history_slice(t, order, n, L, R, Sl, Sg, nthreads=8)
        if kind == "free":
            err = _rel(I, ref)
            assert err < TOL_SPLIT, (M, kind, n, err)
        else:
            mag = _magnitude_slice(t, order, n, L, R, Sl, Sg)
            err = np.abs(I - ref).max() / max(mag, 1e-300)
            assert err < TOL_SPLIT, (M, kind, n, err, _rel(I, ref))


def _just_below_powers_of_two(x):
    """Each real and imaginary part moved to just below the next power of two
    of its magnitude (same sign): 2^k (1 - 2^-40), whose significand's top 32
    bits are all ones, so the entry that sets a column's exponent rounds up
    to the fixed-point maximum."""
    def f(a):
        k = np.ceil(np.log2(np.maximum(np.abs(a), 1e-300)))
        return np.where(a == 0, 0.0, np.sign(a) * np.exp2(k) * (1.0 - 2.0 ** -40))
    return f(x.real) + 1j * f(x.imag)


@pytest.mark.parametrize("path", ["planes", "fused"])
@pytest.mark.parametrize("M", [2, 8])
def test_split_entries_just_below_a_power_of_two(kbe, M, path):
    """Entries within 2^-40 of a power of two (as a half-filled occupation
    1 - 1e-12 is) take the largest fixed-point value, never 0: the slice
    stays within the bound of the oracle's."""
    n_t = 37
    t, order, h, L, R = _case(M, n_t, 70 + M, "random")
    L, R = _just_below_powers_of_two(L), _just_below_powers_of_two(R)
    Ld, Rd = _dev(L), _dev(R)
    for n in (1, 9, n_t - 1):
        Sl, Sg = W.random_rows(M, n, 3 * n + M)
        Sl, Sg = _just_below_powers_of_two(Sl), _just_below_powers_of_two(Sg)
        I = _split_slice(kbe, M, n_t, t, order, h, n, Ld, Rd, Sl, Sg, path)
        ref = oracle.history_slice(t, order, n, L, R, Sl, Sg, nthreads=8)
        mag = _magnitude_slice(t, order, n, L, R, Sl, Sg)
        err = np.abs(I - ref).max() / max(mag, 1e-300)
        assert err < TOL_SPLIT, (M, n, path, err)


@pytest.mark.parametrize("path", ["planes", "fused"])
def test_split_is_deterministic(kbe, path):
    M, n_t = 8, 60
    t, order, h, L, R = _case(M, n_t, 1, "random")
    Ld, Rd = _dev(L), _dev(R)
    n = n_t - 1
    Sl, Sg = W.random_rows(M, n, 2)
    a = _split_slice(kbe, M, n_t, t, order, h, n, Ld, Rd, Sl, Sg, path)
    b = _split_slice(kbe, M, n_t, t, order, h, n, Ld, Rd, Sl, Sg, path)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("M,n_t", [(3, 150), (8, 300), (16, 130), (24, 90), (32, 70)])
def test_split_paths_agree(kbe, M, n_t):
    """The fused contraction (digits formed inside the kernel, column
    exponents per 8 history entries) and the planes path (encoder, exponents
    per 16 entries) round the same values to different fixed-point grids,
    each within the split path's bound of the exact slice (tested against
    the oracle above), so they agree within that bound."""
    t, order, h, L, R = _case(M, n_t, 40 + M, "free")
    Ld, Rd = _dev(L), _dev(R)
    n = n_t - 1
    Sl, Sg = oracle.sigma_row(oracle.local_U4(np.linspace(0.5, 1.5, M)), n, L, R)
    a = _split_slice(kbe, M, n_t, t, order, h, n, Ld, Rd, Sl, Sg, "planes")
    b = _split_slice(kbe, M, n_t, t, order, h, n, Ld, Rd, Sl, Sg, "fused")
    assert _rel(b, a) < TOL_SPLIT, (M, _rel(b, a))


@pytest.mark.parametrize("path", ["planes", "fused"])
@pytest.mark.parametrize("name", ["chain_m8_n1024", "goe_m32_n1024"])
def test_split_full_size_sampled(kbe, name, path):
    """Full-size slice n = N_t - 1 of the chain and GOE workloads; the oracle
    evaluates sampled output columns."""
    import torch
    cfg = W.CONFIGS[name]
    M, n_t = cfg["M"], cfg["n_t"]
    t, order = W.grid(n_t, cfg["dt0"], cfg["sig"], 0)
    h, U, v, pulse = W.build_model(cfg, 0)
    rho0 = W.half_filled_rho(h)
    Ld, Rd = W.free_triangles_torch(h, rho0, t, n_t, "cuda")
    ctx = kbe.Context(M, n_t)
    ctx.set_grid(t, order)
    ctx.set_model(h, U, v, pulse)
    ctx.set_split_planes(path == "planes")
    n = n_t - 1
    Sl = torch.zeros((n + 1, M, M), dtype=torch.complex128, device="cuda")
    Sg = torch.zeros_like(Sl)
    ctx.selfenergy_slice(n, Ld, Rd, Sl, Sg)
    out = torch.zeros((2, n + 1, M, M), dtype=torch.complex128, device="cuda")
    ctx.history_slice(n, Ld, Rd, Sl, Sg, out, precision="split")
    ctx.sync_status()
    I = out.cpu().numpy()
    L, R = Ld.cpu().numpy(), Rd.cpu().numpy()
    cols = [0, 1, 100, 511, 700, n - 1, n]
    ref = oracle.history_columns(t, order, n, L, R, Sl.cpu().numpy(), Sg.cpu().numpy(), cols,
                                 nthreads=oracle.threads_available())
    err = _rel(I[:, cols], ref)
    print(name, "split max rel err on sampled columns", err)
    assert err < TOL_SPLIT
    ctx.close()


def test_split_stepper_tracks_oracle(kbe):
    """KBE steps with the split-precision contraction (everything else FP64)
    stay within the accumulated effect of the 1e-9 slice error of the FP64
    oracle run: 63 steps of the dimer and 31 of the 8-orbital chain."""
    for name, n_t in (("dimer_m2_n64", 64), ("chain_m8_n1024", 32)):
        cfg = W.CONFIGS[name]
        t, order = W.grid(cfg["n_t"], cfg["dt0"], cfg["sig"], 4)
        t, order = t[:n_t], order[:n_t]
        h, U, v, pulse = W.build_model(cfg, 4)
        if pulse is not None:
            pulse = dict(pulse, t0=t[n_t // 2], sigma=0.2)
        rho0 = W.half_filled_rho(h)
        M = cfg["M"]
        ctx = kbe.Context(M, n_t)
        ctx.set_grid(t, order)
        ctx.set_model(h, U, v, pulse)
        run = kbe.Run(ctx)
        run.init_uncorrelated(rho0)
        for n in range(1, n_t):
            run.step(n, P=2, precision="split")
        ctx.sync_status()
        L0, R0, F0 = oracle.initial_rhs(t, order, h, U, v, pulse, rho0)
        Lo = np.zeros((W.tri_size(n_t), M, M), np.complex128)
        Ro = np.zeros_like(Lo)
        Lo[0], Ro[0] = L0[0], R0[0]
        Lo, Ro, _ = oracle.run(t, order, h, U, v, pulse, 2, Lo, Ro, {0: F0}, 1, n_t,
                               nthreads=oracle.threads_available())
        Lg = run.L[: W.tri_size(n_t)].cpu().numpy()
        err = _rel(Lg, Lo)
        print(name, "split stepper max rel err over the run", err)
        assert err < 1e-8, (name, err)
        ctx.close()


@pytest.mark.parametrize("name,n_t", [("chain_m8_n1024", 40), ("goe_m32_n1024", 24)])
def test_split_plane_cache_is_exact(kbe, name, n_t):
    """KBE steps that reuse the digit planes of earlier rows give bitwise the
    rows of steps that encode every row again (kbe_reset_cache before each
    step), including a repeated step of the same row.  A step re-encodes
    only the entries of the rows it changed; with 16 (M = 8) and 4 (M = 32)
    columns per tile the changed rows fall at every position of a tile."""
    import torch
    cfg = W.CONFIGS[name]
    t, order = W.grid(cfg["n_t"], cfg["dt0"], cfg["sig"], 6)
    t, order = t[:n_t], order[:n_t]
    h, U, v, pulse = W.build_model(cfg, 6)
    rho0 = W.half_filled_rho(h)
    runs = []
    for fresh in (False, True):
        ctx = kbe.Context(cfg["M"], n_t)
        ctx.set_grid(t, order)
        ctx.set_model(h, U, v, pulse)
        run = kbe.Run(ctx)
        run.init_uncorrelated(rho0)
        for n in list(range(1, n_t)) + [n_t - 1]:
            if fresh:
                ctx.reset_cache()
            run.step(n, P=2, precision="split")
        ctx.sync_status()
        runs.append(run)
    assert torch.equal(runs[0].L, runs[1].L) and torch.equal(runs[0].R, runs[1].R)
    for r in runs:
        r.ctx.close()


@pytest.mark.parametrize("M,n_t,kind", [(3, 50, "goe"), (5, 40, "chain"), (12, 28, "goe"), (24, 16, "chain")])
def test_split_steps_other_orbital_counts(kbe, M, n_t, kind):
    """Split KBE steps at orbital counts whose tiles hold 42, 25, 10 and 5
    columns (the new row's columns are encoded by the encoder's narrow form,
    a block padded to whole warps): cached planes give bitwise the rows of
    steps that encode everything again, and the run stays within the
    compounded split bound (5e-8) of the oracle's FP64 run."""
    import torch
    t, order = W.grid(n_t, 0.05, 0.4, 60 + M)
    h = W.chain_h(M, 1.0) if kind == "chain" else W.goe_h(M, 60 + M)
    U = np.linspace(0.5, 2.0, M)
    v = W.site_potential(M)
    rho0 = W.half_filled_rho(h)
    runs = []
    for fresh in (False, True):
        ctx = kbe.Context(M, n_t)
        ctx.set_grid(t, order)
        ctx.set_model(h, U, v, None)
        run = kbe.Run(ctx)
        run.init_uncorrelated(rho0)
        for n in range(1, n_t):
            if fresh:
                ctx.reset_cache()
            run.step(n, P=2, precision="split")
        ctx.sync_status()
        runs.append(run)
    assert torch.equal(runs[0].L, runs[1].L) and torch.equal(runs[0].R, runs[1].R)
    L0, R0, F0 = oracle.initial_rhs(t, order, h, U, v, None, rho0)
    Lo = np.zeros((W.tri_size(n_t), M, M), np.complex128)
    Ro = np.zeros_like(Lo)
    Lo[0], Ro[0] = L0[0], R0[0]
    Lo, Ro, _ = oracle.run(t, order, h, U, v, None, 2, Lo, Ro, {0: F0}, 1, n_t,
                           nthreads=oracle.threads_available())
    err = _rel(runs[0].L[: W.tri_size(n_t)].cpu().numpy(), Lo)
    assert err < 5e-8, (M, err)
    for r in runs:
        r.ctx.close()


@pytest.mark.parametrize("path", ["planes", "fused"])
def test_split_wait_timeout_is_reported_and_the_context_recovers(kbe, path):
    """The device-side failure path of the contraction's pipeline, with no
    fault: one work unit's copies are withheld (kbe_debug_withhold_split)
    and the waits give up after 4096 polls.  The launch returns, the
    status reads KBE_ETIMEOUT, and the next slice on the same context is
    correct again."""
    import torch
    M, n_t = 8, 200
    n = n_t - 1
    t, order, h, L, R = _case(M, n_t, 31, "free")
    Sl, Sg = oracle.sigma_row(oracle.local_U4(np.ones(M)), n, L, R)
    ref = oracle.history_slice(t, order, n, L, R, Sl, Sg, nthreads=oracle.threads_available())
    ctx = kbe.Context(M, n_t)
    ctx.set_grid(t, order)
    ctx.set_model(h, np.ones(M), W.site_potential(M), None)
    ctx.set_split_planes(path == "planes")
    Ld, Rd, Sld, Sgd = _dev(L), _dev(R), _dev(Sl), _dev(Sg)
    out = torch.zeros((2, n + 1, M, M), dtype=torch.complex128, device="cuda")
    ctx.history_slice(n, Ld, Rd, Sld, Sgd, out, precision="split")  # planes allocated, kernels loaded
    ctx.sync_status()
    ctx.debug_withhold_split(3, 4096)
    ctx.history_slice(n, Ld, Rd, Sld, Sgd, out, precision="split")
    with pytest.raises(kbe.KBEError) as e:
        ctx.sync_status()
    assert e.value.status == kbe.KBE_ETIMEOUT
    out.fill_(float("nan"))
    ctx.history_slice(n, Ld, Rd, Sld, Sgd, out, precision="split")
    ctx.sync_status()
    assert _rel(out.cpu().numpy(), ref) < TOL_SPLIT
    ctx.close()
