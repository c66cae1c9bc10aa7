"""GPU parity of the general four-index interaction (Eq. SE, Eq. eps): the
dense self-energy kernel and whole runs against the oracle.

Tolerance: 1e-12 relative in the max norm per row (FP64 sums in another
order than the oracle's).  Where the oracle's M^8 sum per block is too slow
(norb 12..32), the reference is the closed form of Eq. (SE) for sums of
product tensors, which the oracle's own tests pin at small norb."""
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


def _dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _general_tensor(M, seed):
    """A real tensor with no index symmetry at all."""
    return np.random.default_rng(seed).standard_normal((M, M, M, M)) / M


def _ctx(kbe, M, n_max, t=None, order=None, h=None):
    ctx = kbe.Context(M, n_max)
    if t is None:
        t, order = W.grid(n_max, 0.05, 0.3, M)
    ctx.set_grid(t, order)
    ctx.set_model(W.goe_h(M, 1) if h is None else h, np.ones(M), W.site_potential(M), None)
    return ctx


def _gpu_row(kbe, ctx, n, L, R):
    import torch
    M = ctx.M
    Sl = torch.zeros((n + 1, M, M), dtype=torch.complex128, device="cuda")
    Sg = torch.zeros_like(Sl)
    ctx.selfenergy_slice(n, _dev(L), _dev(R), Sl, Sg)
    ctx.sync_status()
    return Sl.cpu().numpy(), Sg.cpu().numpy()


# pair tiles of the kernel: one tile (M <= 4), several with a ragged last
# tile (M = 5, 6, 7), sixteen full tiles (M = 8)
@pytest.mark.parametrize("M,n,kind", [(1, 5, "random"), (2, 9, "free"), (3, 7, "random"), (4, 6, "free"),
                                      (5, 6, "random"), (6, 4, "free"), (7, 3, "random"), (8, 2, "random")])
def test_dense_sigma_row_matches_oracle(kbe, M, n, kind):
    U4 = _general_tensor(M, 10 + M)
    if kind == "free":
        h = W.goe_h(M, M)
        t, _ = W.grid(n + 1, 0.1, 0.3, M)
        L, R = W.free_triangles(h, W.half_filled_rho(h), t)
    else:
        L, R = W.random_triangles(M, n + 1, M)
    ctx = _ctx(kbe, M, n + 1)
    ctx.set_interaction(U4)
    Sl, Sg = _gpu_row(kbe, ctx, n, L, R)
    ol, og = oracle.sigma_row(U4, n, L, R)
    assert _rel(Sl, ol) < TOL and _rel(Sg, og) < TOL, (_rel(Sl, ol), _rel(Sg, og))
    assert ctx.last_launch_count == 0
    ctx.close()


def test_dense_selfenergy_all_matches_oracle(kbe):
    """Whole-triangle launch: the kernel finds the diagonal blocks itself."""
    import torch
    M, n_t = 3, 14
    U4 = W.coulomb_tensor(M, 2, U=1.3)
    L, R = W.random_triangles(M, n_t, 5)
    ctx = _ctx(kbe, M, n_t)
    ctx.set_interaction(U4)
    Sl = torch.zeros((W.tri_size(n_t), M, M), dtype=torch.complex128, device="cuda")
    Sg = torch.zeros_like(Sl)
    ctx.selfenergy_all(n_t, _dev(L), _dev(R), Sl, Sg)
    ctx.sync_status()
    Sl, Sg = Sl.cpu().numpy(), Sg.cpu().numpy()
    for n in range(n_t):
        ol, og = oracle.sigma_row(U4, n, L, R)
        p = tri(n, 0)
        assert _rel(Sl[p:p + n + 1], ol) < TOL and _rel(Sg[p:p + n + 1], og) < TOL, n
    ctx.close()


def _product_sigma(vecs, G, Gp):
    """Eq. (SE) for U = sum_r a^r (x) b^r (x) c^r (x) d^r, blocks stacked on
    the first axis: Sigma = sum_{r,q} (d^q G' c^r) [2 (b^r G b^q)(d^r G c^q)
    - (b^r G c^q)(d^r G b^q)] a^r a^q^T."""
    bil = lambda x, A, y: np.einsum("i,kij,j->k", x, A, y)
    out = np.zeros(G.shape, np.complex128)
    for r in range(len(vecs)):
        a, b, c, d = vecs[r]
        for q in range(len(vecs)):
            a2, b2, c2, d2 = vecs[q]
            f = bil(d2, Gp, c) * (2 * bil(b, G, b2) * bil(d, G, c2) - bil(b, G, c2) * bil(d, G, b2))
            out += f[:, None, None] * np.outer(a, a2)[None]
    return out


@pytest.mark.parametrize("M", [12, 16, 24, 32])
def test_dense_sigma_product_tensor_large_norb(kbe, M):
    rng = np.random.default_rng(M)
    vecs = rng.standard_normal((2, 4, M)) / np.sqrt(M)
    U4 = sum(np.einsum("p,q,r,s->pqrs", *vecs[r]) for r in range(2))
    n = 5
    L, R = W.random_triangles(M, n + 1, M + 1)
    ctx = _ctx(kbe, M, n + 1)
    ctx.set_interaction(U4)
    Sl, Sg = _gpu_row(kbe, ctx, n, L, R)
    Lr, Rr = L[tri(n, 0):tri(n, 0) + n + 1], R[tri(n, 0):tri(n, 0) + n + 1]
    Gl, Gg = Lr, Rr + Lr
    # G^s'(t_c, t_n) = -G^s'(t_n, t_c)^+ off the diagonal, the stored block on it
    Gl_t = -np.conj(np.transpose(Gl, (0, 2, 1)))
    Gg_t = -np.conj(np.transpose(Gg, (0, 2, 1)))
    Gl_t[n], Gg_t[n] = Gl[n], Gg[n]
    ref_l = _product_sigma(vecs, Gl, Gg_t)
    ref_g = _product_sigma(vecs, Gg, Gl_t)
    assert _rel(Sl, ref_l) < TOL and _rel(Sg, ref_g) < TOL, (_rel(Sl, ref_l), _rel(Sg, ref_g))
    ctx.close()


def test_dense_sigma_full_size_sampled_blocks(kbe):
    """Row n = 1023 of a 1024-point grid at norb 8 (the size the benchmark
    times): sampled blocks against the oracle.  A block of Eq. (SE) needs
    only G(t_n,t_c), so each sample is the oracle's row 1 of a two-row
    triangle holding (t_n,t_c) and (t_n,t_n)."""
    import torch
    M, n = 8, 1023
    U4 = W.coulomb_tensor(M, 3, U=1.0)
    Lr, Rr = W.random_rows(M, n, 9)  # row n of L and R
    Rr[n] = -1j * np.eye(M)
    ctx = kbe.Context(M, n + 1)
    ctx.set_grid(*W.grid(n + 1, 0.02, 0.4, 1))
    ctx.set_model(W.chain_h(M), np.ones(M), W.site_potential(M), None)
    ctx.set_interaction(U4)
    L = torch.zeros((W.tri_size(n + 1), M, M), dtype=torch.complex128, device="cuda")
    R = torch.zeros_like(L)
    L[tri(n, 0):tri(n, 0) + n + 1] = _dev(Lr)
    R[tri(n, 0):tri(n, 0) + n + 1] = _dev(Rr)
    Sl = torch.zeros((n + 1, M, M), dtype=torch.complex128, device="cuda")
    Sg = torch.zeros_like(Sl)
    ctx.selfenergy_slice(n, L, R, Sl, Sg)
    ctx.sync_status()
    Sl, Sg = Sl.cpu().numpy(), Sg.cpu().numpy()
    del L, R
    for c in (0, 1, 511, 1022):
        L2 = np.stack([Lr[n], Lr[c], Lr[n]])
        R2 = np.stack([Rr[n], Rr[c], Rr[n]])
        ol, og = oracle.sigma_row(U4, 1, L2, R2)
        assert _rel(Sl[c], ol[0]) < TOL and _rel(Sg[c], og[0]) < TOL, c
        assert _rel(Sl[n], ol[1]) < TOL and _rel(Sg[n], og[1]) < TOL
    ctx.close()


def _setup(M, n_t, kind, seed, with_pulse):
    t, order = W.grid(n_t, 0.05, 0.3, seed)
    h = W.chain_h(M, 1.0) if kind == "chain" else W.goe_h(M, seed)
    U4 = W.coulomb_tensor(M, seed, U=1.2)
    v = W.site_potential(M)
    pulse = dict(W.PULSE_CHAIN, t0=float(t[n_t // 2]), sigma=0.4) if with_pulse else None
    return t, order, h, U4, v, pulse


def _oracle_run(t, order, h, U4, v, pulse, P=2, K_sel=None):
    M = h.shape[0]
    n_t = len(t)
    rho0 = W.half_filled_rho(h)
    L0, R0, F0 = oracle.initial_rhs(t, order, h, None, v, pulse, rho0, U4=U4)
    L = np.zeros((W.tri_size(n_t), M, M), np.complex128)
    R = np.zeros_like(L)
    L[0], R[0] = L0[0], R0[0]
    if K_sel is None:
        Lo, Ro, _ = oracle.run(t, order, h, None, v, pulse, P, L, R, {0: F0}, 1, n_t, nthreads=4, U4=U4)
        return Lo, Ro, None
    return oracle.run_adaptive(t, order, [0], K_sel, h, None, v, pulse, P, L, R, {0: F0}, 1, n_t, nthreads=4,
                               U4=U4)[0::3]


def _gpu_run(kbe, t, order, h, U4, v, pulse, precision="fp64", P=2, K_sel=0):
    M = h.shape[0]
    n_t = len(t)
    ctx = kbe.Context(M, n_t)
    ctx.set_grid(t, order)
    ctx.set_model(h, np.zeros(M), v, pulse)
    ctx.set_interaction(U4)
    if K_sel:
        ctx.set_adaptive_orders(K_sel)
    run = kbe.Run(ctx)
    run.init_uncorrelated(W.half_filled_rho(h))
    for n in range(1, n_t):
        run.step(n, P=P, precision=precision)
    ctx.sync_status()
    return ctx, run


@pytest.mark.parametrize("M,n_t,kind,seed,pulse", [(2, 48, "chain", 0, True), (4, 32, "goe", 1, False),
                                                   (6, 20, "chain", 2, True)])
def test_dense_run_matches_oracle(kbe, M, n_t, kind, seed, pulse):
    t, order, h, U4, v, pl = _setup(M, n_t, kind, seed, pulse)
    Lo, Ro, _ = _oracle_run(t, order, h, U4, v, pl)
    ctx, run = _gpu_run(kbe, t, order, h, U4, v, pl)
    p = W.tri_size(n_t)
    assert _rel(run.L[:p].cpu().numpy(), Lo) < TOL
    assert _rel(run.R[:p].cpu().numpy(), Ro) < TOL
    ctx.close()


def test_dense_run_split_precision_and_adaptive_orders(kbe):
    M, n_t = 4, 32
    t, order, h, U4, v, pl = _setup(M, n_t, "chain", 3, True)
    Lo, _, _ = _oracle_run(t, order, h, U4, v, pl)
    ctx, run = _gpu_run(kbe, t, order, h, U4, v, pl, precision="split")
    assert _rel(run.L[:W.tri_size(n_t)].cpu().numpy(), Lo) < 5e-8  # compounded over the run
    ctx.close()
    La, hord = _oracle_run(t, order, h, U4, v, pl, K_sel=6)
    ctx, run = _gpu_run(kbe, t, order, h, U4, v, pl, K_sel=6)
    assert np.array_equal(ctx.history_orders(n_t)[1:], hord[1:n_t])
    assert _rel(run.L[:W.tri_size(n_t)].cpu().numpy(), La) < TOL
    ctx.close()


def test_dense_with_local_tensor_is_the_local_path(kbe):
    import torch
    M, n_t = 5, 24
    t, order = W.grid(n_t, 0.05, 0.3, 4)
    h = W.chain_h(M)
    U = np.linspace(0.8, 2.0, M)
    v = W.site_potential(M)
    runs = []
    for dense in (False, True):
        ctx = kbe.Context(M, n_t)
        ctx.set_grid(t, order)
        ctx.set_model(h, U, v, W.PULSE_CHAIN)
        if dense:
            ctx.set_interaction(oracle.local_U4(U))
        run = kbe.Run(ctx)
        run.init_uncorrelated(W.half_filled_rho(h))
        for n in range(1, n_t):
            run.step(n)
        ctx.sync_status()
        runs.append((ctx, run))
    p = W.tri_size(n_t)
    # the local kernel forms its products in double-float, the dense one in FP64
    assert _rel(runs[1][1].L[:p].cpu().numpy(), runs[0][1].L[:p].cpu().numpy()) < 1e-13
    ctx = runs[1][0]
    ctx.set_interaction(None)  # back to the local interaction: same kernel, same numbers
    L, R = runs[0][1].L, runs[0][1].R
    Sa = [torch.zeros((n_t, M, M), dtype=torch.complex128, device="cuda") for _ in range(4)]
    runs[0][0].selfenergy_slice(n_t - 1, L, R, Sa[0], Sa[1])
    ctx.selfenergy_slice(n_t - 1, L, R, Sa[2], Sa[3])
    torch.cuda.synchronize()
    assert torch.equal(Sa[0], Sa[2]) and torch.equal(Sa[1], Sa[3])
    for c, _ in runs:
        c.close()


def test_dense_interaction_errors(kbe):
    import torch
    M = 3
    ctx = _ctx(kbe, M, 8)
    bad = W.coulomb_tensor(M, 1)
    bad[0, 1, 2, 0] = np.nan
    with pytest.raises(kbe.KBEError) as e:
        ctx.set_interaction(bad)
    assert e.value.status == kbe.KBE_EINVAL
    ctx.set_interaction(W.coulomb_tensor(M, 1))
    run = kbe.Run(ctx)
    run.init_uncorrelated(W.half_filled_rho(W.goe_h(M, 1)))
    run.step(1)
    with pytest.raises(kbe.KBEError) as e:
        kbe.Batch([run])
    assert e.value.status == kbe.KBE_EINVAL
    z = torch.zeros((2, M, M), dtype=torch.complex128, device="cuda")
    dU = torch.zeros(M, dtype=torch.float64, device="cuda")
    with pytest.raises(kbe.KBEError) as e:
        ctx.adjoint_selfenergy_slice(1, run.L, run.R, z, z.clone(), z.clone(), z.clone(), dU)
    assert e.value.status == kbe.KBE_ESTATE
    ctx.sync_status()
    ctx.close()
    big = kbe.Context(33, 4)
    with pytest.raises(kbe.KBEError) as e:
        big.set_interaction(np.zeros((33,) * 4))
    assert e.value.status == kbe.KBE_ERANGE
    big.close()
