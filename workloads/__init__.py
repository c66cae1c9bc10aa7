"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module only generates inputs: time grids with per-interval orders,
one-body Hamiltonians, interaction strengths, pulse parameters, initial
density matrices and two-time histories of the non-interacting (U = 0)
problem or seeded random stress data.  It holds none of the method's
arithmetic: no quadrature weights, self-energies, history integrals or time
stepping.  Both the oracle and the CUDA path read what it produces.

Two-time arrays use the triangle-packed layout ``[tri(N), M, M]`` with block
``r*(r+1)/2 + c`` for ``r >= c``; ``L = G^<`` and ``R = G^R``.

Workload recipes (the shapes of the paper's model systems, Sec. 5-6; the
paper's own inputs are not available):
  * time grid: ``dt_l = dt0 * exp(sig * z_l)``, ``z ~ N(0,1)`` from numpy's
    PCG64 with the given seed, then per-interval orders ``k_l`` uniform in
    ``{kmin..kmax}`` from the same generator (z first, then k);
  * Hubbard chain: ``h_{i,i+1} = h_{i+1,i} = -J`` (open chain);
  * GOE one-body matrix: ``A_ij ~ N(0, 1/M)``, ``h = (A + A^T)/2``;
  * half filling: the lowest ``M//2`` eigenvectors of h occupied, per spin;
  * pulse: ``E(t) = E0 exp(-(t-t0)^2/(2 sigma^2)) cos(omega t)`` entering as
    the site potential ``E(t) * (i - (M-1)/2)``;
  * dense Coulomb tensor (chemists' order, ``U[p,q,r,s] = (pq|rs)``, the
    shape of quantum-chemistry integrals, which the paper takes from pyscf):
    ``(pq|rs) = sum_k B^k_pq B^k_rs`` with symmetric ``B^k``, entries
    ``N(0,1)`` symmetrised, scaled so that the mean of ``(pp|pp)`` is ``U``.
    This has the 8-fold symmetry of real-orbital integrals and is positive
    semidefinite as a matrix over orbital pairs.
"""
import numpy as np

try:  # torch is only needed for the large, device-side histories
    import torch
except Exception:  # pragma: no cover
    torch = None


def tri_size(n):
    return n * (n + 1) // 2


def tri_index(r, c):
    return r * (r + 1) // 2 + c


def grid(n_t, dt0, sig, seed, kmin=1, kmax=5):
    """Nonuniform grid t[0..n_t-1] (t[0] = 0) and orders order[1..n_t-1]
    (order[0] = 0 is unused)."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(n_t - 1)
    k = rng.integers(kmin, kmax + 1, size=n_t - 1)
    t = np.zeros(n_t)
    t[1:] = np.cumsum(dt0 * np.exp(sig * z))
    order = np.zeros(n_t, dtype=np.int32)
    order[1:] = k
    return t, order


def uniform_grid(n_t, h, k):
    t = h * np.arange(n_t, dtype=np.float64)
    order = np.full(n_t, k, dtype=np.int32)
    order[0] = 0
    return t, order


def chain_h(M, J=1.0):
    h = np.zeros((M, M), np.complex128)
    for i in range(M - 1):
        h[i, i + 1] = -J
        h[i + 1, i] = -J
    return h


def goe_h(M, seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(0.0, 1.0 / np.sqrt(M), size=(M, M))
    return ((A + A.T) / 2).astype(np.complex128)


def site_potential(M):
    return np.arange(M, dtype=np.float64) - (M - 1) / 2.0


def coulomb_tensor(M, seed, U=1.0, rank=None):
    """Real [M, M, M, M] tensor with the symmetries of Coulomb integrals."""
    rng = np.random.default_rng(seed)
    K = M * (M + 1) // 2 if rank is None else rank
    B = rng.standard_normal((K, M, M))
    B = (B + B.transpose(0, 2, 1)) / 2
    T = np.einsum("kpq,krs->pqrs", B, B)
    d = np.mean([T[p, p, p, p] for p in range(M)])
    return T * (U / d)


def thermal_free(h, beta, N, t=None):
    """Non-interacting equilibrium at inverse temperature beta (chemical
    potential 0) on the uniform tau grid tau_k = k beta / (N - 1):
    G^M(tau_k) = -V diag(e^{-e tau} (1 - f(e))) V^+ (tau_0 = 0+, tau_{N-1} =
    beta-), the density f(h), and, for times t, the mixed function
    G^|(t, tau) = i V diag(e^{-i e t} f(e) e^{e tau}) V^+ [len(t), N, M, M]."""
    e, V = np.linalg.eigh(h)
    tau = beta * np.arange(N) / (N - 1)
    f = 0.5 * (1.0 - np.tanh(0.5 * beta * e))
    # e^{-e tau}(1 - f) and f e^{e tau}, written to stay finite for large |e| beta
    one_m_f = 0.5 * (1.0 + np.tanh(0.5 * beta * e))
    gm_diag = -np.exp(-np.outer(tau, e)) * one_m_f
    GM = np.einsum("ak,tk,bk->tab", V, gm_diag, V.conj())
    rho = (V * f) @ V.conj().T
    mix = None
    if t is not None:
        fe = f[None, :] * np.exp(np.outer(tau, e))  # [N, k]
        ph = np.exp(-1j * np.outer(t, e))            # [T, k]
        mix = 1j * np.einsum("ak,rk,jk,bk->rjab", V, ph, fe, V.conj())
    return GM.astype(np.complex128), rho.astype(np.complex128), mix


def half_filled_rho(h):
    M = h.shape[0]
    _, V = np.linalg.eigh(h)
    occ = V[:, : M // 2]
    return (occ @ occ.conj().T).astype(np.complex128)


def propagators(h, t):
    """e^{-i h t_r} for every grid time (the free evolution)."""
    e, V = np.linalg.eigh(h)
    ph = np.exp(-1j * np.outer(t, e))                 # [N, M]
    return np.einsum("ak,rk,bk->rab", V, ph, V.conj())  # [N, M, M]


def free_triangles(h, rho0, t, n_rows=None):
    """Non-interacting history: G^<(t,t') = i A(t) rho0 A(t')^+,
    G^R(t,t') = -i A(t) A(t')^+ with A(t) = e^{-iht}; rows 0..n_rows-1."""
    n_rows = len(t) if n_rows is None else n_rows
    A = propagators(h, t[:n_rows])
    M = h.shape[0]
    L = np.zeros((tri_size(n_rows), M, M), np.complex128)
    R = np.zeros_like(L)
    Ar = np.einsum("rab,bc->rac", A, rho0)
    for r in range(n_rows):
        p = tri_index(r, 0)
        L[p:p + r + 1] = 1j * np.einsum("ab,cdb->cad", Ar[r], A[: r + 1].conj())
        R[p:p + r + 1] = -1j * np.einsum("ab,cdb->cad", A[r], A[: r + 1].conj())
        R[p + r] = -1j * np.eye(M)
    return L, R


def free_triangles_torch(h, rho0, t, n_rows, device, chunk_blocks=None, out=None):
    """``free_triangles`` built with torch on ``device`` (large histories),
    a few batched products per chunk of rows; ``out`` = (L, R) fills the
    first tri(n_rows) blocks of existing tensors instead of new ones."""
    A = torch.from_numpy(propagators(h, t[:n_rows])).to(device)
    rho = torch.from_numpy(rho0).to(device)
    M = h.shape[0]
    ntri = tri_size(n_rows)
    if chunk_blocks is None:  # about 512 MB per temporary
        chunk_blocks = max(4096, (1 << 29) // (M * M * 16))
    if out is None:
        L = torch.empty((ntri, M, M), dtype=torch.complex128, device=device)
        R = torch.empty_like(L)
    else:
        L, R = out
    Ar = A @ rho
    Ah = A.conj().transpose(1, 2).contiguous()
    r0 = 0
    while r0 < n_rows:
        r1 = r0 + 1
        while r1 < n_rows and tri_size(r1 + 1) - tri_size(r0) <= chunk_blocks:
            r1 += 1
        p0, p1 = tri_size(r0), tri_size(r1)
        idx = torch.arange(p0, p1, device=device)
        r = ((torch.sqrt(8.0 * idx.double() + 1.0) - 1.0) / 2.0).floor().long()
        r = torch.where(r * (r + 1) // 2 > idx, r - 1, r)
        r = torch.where((r + 1) * (r + 2) // 2 <= idx, r + 1, r)
        c = idx - r * (r + 1) // 2
        L[p0:p1] = 1j * torch.bmm(Ar[r], Ah[c])
        R[p0:p1] = -1j * torch.bmm(A[r], Ah[c])
        r0 = r1
    diag = torch.tensor([tri_index(q, q) for q in range(n_rows)], device=device)
    R[diag] = -1j * torch.eye(M, dtype=torch.complex128, device=device)
    return L, R


def free_rhs_rows(h, L, R, rows):
    """Exact t-derivatives of the non-interacting history, used as frozen
    right-hand-side rows at a restart: d/dt G^s(t_j, t_c) = -i h G^s(t_j, t_c)
    for s = <, > (G^> = G^R + G^<), as [2, j+1, M, M] per row j."""
    out = {}
    for j in rows:
        p = tri_index(j, 0)
        Gl = L[p:p + j + 1]
        Gg = R[p:p + j + 1] + Gl
        out[j] = np.stack([-1j * np.einsum("ab,cbd->cad", h, Gl),
                           -1j * np.einsum("ab,cbd->cad", h, Gg)])
    return out


def random_triangles(M, n_rows, seed, scale=1.0):
    """Seeded random complex histories (stress data) with R(r,r) = -i*1."""
    rng = np.random.default_rng(seed)
    ntri = tri_size(n_rows)
    L = scale * (rng.standard_normal((ntri, M, M)) + 1j * rng.standard_normal((ntri, M, M)))
    R = scale * (rng.standard_normal((ntri, M, M)) + 1j * rng.standard_normal((ntri, M, M)))
    for r in range(n_rows):
        R[tri_index(r, r)] = -1j * np.eye(M)
    return L.astype(np.complex128), R.astype(np.complex128)


def random_rows(M, n, seed, scale=1.0):
    """Seeded random self-energy rows S^<, S^> of row n: two [n+1, M, M]."""
    rng = np.random.default_rng(seed)
    shp = (n + 1, M, M)
    Sl = scale * (rng.standard_normal(shp) + 1j * rng.standard_normal(shp))
    Sg = scale * (rng.standard_normal(shp) + 1j * rng.standard_normal(shp))
    return Sl.astype(np.complex128), Sg.astype(np.complex128)


# ---------------------------------------------------------------- configs --
PULSE_CHAIN = {"E0": 0.5, "t0": 5.0, "sigma": 1.0, "omega": 2.0}

CONFIGS = {
    # Hubbard dimer, quench of U at t = 0 (Sec. 6 model family, M = 2 as the
    # H2/sto-6g system of Sec. 5).
    "dimer_m2_n64": dict(M=2, J=1.0, U=1.0, n_t=64, dt0=0.05, sig=0.3, h="chain", pulse=None),
    # open Hubbard chain with a Gaussian pulse (plain FP64 GPU workload)
    "chain_m8_n1024": dict(M=8, J=1.0, U=2.0, n_t=1024, dt0=0.02, sig=0.4, h="chain", pulse=PULSE_CHAIN),
    # GOE one-body matrix, precision-form workload
    "goe_m32_n1024": dict(M=32, J=None, U=1.5, n_t=1024, dt0=0.02, sig=0.4, h="goe", pulse=None),
    # differentiation workload: last 32 steps of a 512-point chain run
    "chain_m16_n512_w32": dict(M=16, J=1.0, U=2.0, n_t=512, dt0=0.02, sig=0.4, h="chain",
                               pulse=PULSE_CHAIN, window=32),
}


def build_model(cfg, seed):
    """(h0, U vector, site potential, pulse) of a config."""
    M = cfg["M"]
    h = chain_h(M, cfg["J"]) if cfg["h"] == "chain" else goe_h(M, 1000 + seed)
    U = np.full(M, cfg["U"], dtype=np.float64)
    return h, U, site_potential(M), cfg["pulse"]


def batch_model(sys):
    """Grid and model of one batched system: an open chain (J = 1) with
    local U, the site potential, no pulse, on its own seeded grid
    (dt_n = 0.02 exp(0.4 z_n), orders 1..5)."""
    t, order = grid(sys["n_t"], 0.02, 0.4, sys["grid_seed"])
    M = sys["M"]
    return t, order, chain_h(M, sys["J"]), np.full(M, sys["U"]), site_potential(M), None


def batch_systems(n_sys, seed):
    """Batched workload: n_sys independent Hubbard-type chains with M in
    {4,8,12,16,24}, history length N_t uniform in [256,1536], U uniform in
    [0.5,3], J = 1, each on its own seeded grid."""
    rng = np.random.default_rng(seed)
    Ms = rng.choice(np.array([4, 8, 12, 16, 24]), size=n_sys)
    Ns = rng.integers(256, 1537, size=n_sys)
    Us = rng.uniform(0.5, 3.0, size=n_sys)
    out = []
    for i in range(n_sys):
        out.append(dict(M=int(Ms[i]), n_t=int(Ns[i]), U=float(Us[i]), J=1.0,
                        grid_seed=int(seed * 1000 + i)))
    return out


def restart_state(h, rho0, t, order, n_start, n_rows, device=None):
    """Frozen state of a restart at row n_start: the non-interacting
    history (rows 0..n_rows-1; rows >= n_start are overwritten by the
    steps) and the right-hand-side rows the stepper needs on entry,
    j in [n_start - K, n_start) with K the largest order up to n_rows.
    ``device`` None gives numpy triangles, else torch tensors there."""
    K = max(1, int(np.max(order[1:n_rows]))) if n_rows > 1 else 1
    rows = list(range(max(0, n_start - K), n_start))
    if device is None:
        L, R = free_triangles(h, rho0, t, n_rows)
        Ln, Rn = L, R
    else:
        L, R = free_triangles_torch(h, rho0, t, n_rows, device)
        lo, hi = tri_index(rows[0], 0) if rows else 0, tri_index(n_start, 0)
        Ln = np.zeros((hi, h.shape[0], h.shape[0]), np.complex128)
        Rn = np.zeros_like(Ln)
        Ln[lo:hi] = L[lo:hi].cpu().numpy()
        Rn[lo:hi] = R[lo:hi].cpu().numpy()
    return L, R, free_rhs_rows(h, Ln, Rn, rows)
