"""Python binding of libkbe: the GB300 hot path of the adaptive
Kadanoff-Baym solver (arXiv 2405.08737).

Argument marshalling only.  Every step of the path runs in the library's
CUDA kernels; PyTorch provides device memory and streams.  There is no CPU
fallback: if the compiled library is missing, importing the handles raises.

Layouts (see include/kbe.h): complex128 tensors, two-time arrays
``[tri(N), M, M]`` with block ``r*(r+1)//2 + c`` for ``r >= c``;
self-energy rows ``[n+1, M, M]``; history slices ``[2, n+1, M, M]``;
right-hand-side ring ``[KBE_RING_ROWS, 2, n_max, M, M]``.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkbe.so")

KBE_OK, KBE_EINVAL, KBE_ERANGE, KBE_ENOMEM, KBE_ECUDA, KBE_ENUMERIC, KBE_ETIMEOUT, KBE_ESTATE = range(8)
KBE_MAX_ORDER = 12
KBE_RING_ROWS = 13
KBE_FP64 = 0
KBE_SPLIT_BF16 = 1
KBE_DF64 = 2
PRECISIONS = {"fp64": KBE_FP64, "split": KBE_SPLIT_BF16, "df64": KBE_DF64}

_lib = None


class KBEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("kbe status %d: %s" % (status, msg))
        self.status = status


def lib():
    """The loaded libkbe (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libkbe.so is not built (run __graft_entry__.build() or "
                               "python -m paper_2405_08737_gb300.build); there is no fallback")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.kbe_create.argtypes = [i, i, ctypes.POINTER(vp)]
        L.kbe_destroy.argtypes = [vp]
        L.kbe_last_error.argtypes = [vp]
        L.kbe_last_error.restype = ctypes.c_char_p
        L.kbe_last_launch_count.argtypes = [vp]
        L.kbe_set_grid.argtypes = [vp, vp, vp, i]
        L.kbe_grid_weights.argtypes = [vp, vp, i, i, vp]
        L.kbe_local_weights.argtypes = [vp, i, d, d, vp]
        L.kbe_set_model.argtypes = [vp, vp, vp, vp, vp]
        L.kbe_set_interaction.argtypes = [vp, vp]
        L.kbe_run_controlled.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.kbe_set_thermal.argtypes = [vp, d, i, i, vp]
        L.kbe_copy_mixed.argtypes = [vp, i, vp, i, vp]
        L.kbe_selfenergy_slice.argtypes = [vp, i, vp, vp, vp, vp, vp]
        L.kbe_selfenergy_all.argtypes = [vp, i, vp, vp, vp, vp, vp]
        L.kbe_history_slice.argtypes = [vp, i, i, vp, vp, vp, vp, vp, vp]
        L.kbe_rhs_row.argtypes = [vp, i, i, vp, vp, vp, vp, vp, vp, vp]
        L.kbe_init_uncorrelated.argtypes = [vp, vp, vp, vp, vp]
        L.kbe_debug_withhold_split.argtypes = [vp, ctypes.c_longlong, ctypes.c_longlong]
        L.kbe_debug_withhold_run.argtypes = [vp, ctypes.c_int, ctypes.c_longlong]
        L.kbe_set_split_planes.argtypes = [vp, i]
        L.kbe_step_predict.argtypes = [vp, i, vp, vp, vp, vp]
        L.kbe_step_sweep_band.argtypes = [vp, i, i, i, vp, vp, vp, vp, vp, vp]
        L.kbe_step_sweep_finish.argtypes = [vp, i, vp, vp, vp, vp, vp]
        L.kbe_step.argtypes = [vp, i, i, i, vp, vp, vp, vp, vp, vp, vp]
        L.kbe_run_steps.argtypes = [vp, i, i, i, i, vp, vp, vp, vp, vp, vp, vp]
        L.kbe_step_rows.argtypes = [vp, i, i, i, vp, vp, vp, vp, vp, vp, i, i, vp]
        L.kbe_step_host.argtypes = [vp, i, i, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.kbe_history_slice_band.argtypes = [vp, i, i, i, vp, vp, vp, vp, vp, vp]
        L.kbe_adjoint_slice.argtypes = [vp, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, i, vp]
        L.kbe_adjoint_selfenergy_slice.argtypes = [vp, i, vp, vp, vp, vp, vp, vp, vp, vp]
        L.kbe_step_adjoint.argtypes = [vp, i, i, i, vp, vp, vp, i, i, vp, vp, i, vp, vp, vp, vp]
        L.kbe_batch_create.argtypes = [vp, i, ctypes.POINTER(vp)]
        L.kbe_batch_destroy.argtypes = [vp]
        L.kbe_batch_last_error.argtypes = [vp]
        L.kbe_batch_last_error.restype = ctypes.c_char_p
        L.kbe_batch_last_launch_count.argtypes = [vp]
        L.kbe_batch_bind.argtypes = [vp, i, vp, vp, vp, vp, vp, vp]
        L.kbe_batch_step.argtypes = [vp, vp, i, i, vp]
        L.kbe_batch_set_policy.argtypes = [vp, i, i]
        L.kbe_batch_get_policy.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.kbe_batch_autotune.argtypes = [vp, vp, i, vp, ctypes.POINTER(i), ctypes.POINTER(i),
                                         ctypes.POINTER(d)]
        L.kbe_batch_sync_status.argtypes = [vp, vp]
        L.kbe_sync_status.argtypes = [vp, vp]
        L.kbe_reset_cache.argtypes = [vp]
        L.kbe_set_adaptive_orders.argtypes = [vp, i]
        L.kbe_get_history_orders.argtypes = [vp, vp, i]
        L.kbe_set_profiling.argtypes = [vp, i]
        L.kbe_read_profiling.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(d)]
        _lib = L
    return _lib


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _raise(status, ctx=None):
    if status != KBE_OK:
        msg = lib().kbe_last_error(ctx).decode()
        raise KBEError(status, msg)


# ------------------------------------------------------------- host weights
def grid_weights(t, order, n):
    """Composite weight row w_{n,0..n} (host FP64, Sec. 3.2)."""
    t = np.ascontiguousarray(t, np.float64)
    order = np.ascontiguousarray(order, np.int32)
    row = np.zeros(n + 1)
    _raise(lib().kbe_grid_weights(_np_ptr(t), _np_ptr(order), len(t), n, _np_ptr(row)))
    return row


def local_weights(tau, lo, hi):
    """Weights of the degree-(len(tau)-1) interpolatory rule over [lo, hi]."""
    tau = np.ascontiguousarray(tau, np.float64)
    w = np.zeros(len(tau))
    _raise(lib().kbe_local_weights(_np_ptr(tau), len(tau) - 1, lo, hi, _np_ptr(w)))
    return w


def tri_size(n):
    return n * (n + 1) // 2


# --------------------------------------------------------------- context
class Context:
    """A kbe_ctx for ``norb`` orbitals and up to ``n_max`` time points."""

    def __init__(self, norb, n_max):
        import torch  # noqa: F401  (device memory and streams)
        self.M = int(norb)
        self.n_max = int(n_max)
        h = ctypes.c_void_p()
        _raise(lib().kbe_create(self.M, self.n_max, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().kbe_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- helpers
    def _check(self, status):
        if status != KBE_OK:
            raise KBEError(status, lib().kbe_last_error(self._h).decode())

    @staticmethod
    def _stream(stream):
        import torch
        s = torch.cuda.current_stream() if stream is None else stream
        return ctypes.c_void_p(s.cuda_stream)

    @staticmethod
    def _host(x, nbytes):
        """Pointer to a contiguous complex128 host tensor of at least nbytes."""
        import torch
        if not isinstance(x, torch.Tensor) or x.is_cuda:
            raise TypeError("expected a host (CPU) tensor")
        if x.dtype != torch.complex128 or not x.is_contiguous():
            raise TypeError("expected a contiguous complex128 tensor")
        if x.numel() * 16 < nbytes:
            raise ValueError("host tensor of %d bytes, %d needed" % (x.numel() * 16, nbytes))
        return ctypes.c_void_p(x.data_ptr())

    def _dev(self, x, shape=None):
        import torch
        if not isinstance(x, torch.Tensor) or not x.is_cuda:
            raise TypeError("expected a CUDA tensor")
        if x.dtype != torch.complex128:
            raise TypeError("expected complex128, got %s" % x.dtype)
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        if shape is not None and tuple(x.shape[: len(shape)]) != tuple(shape):
            raise ValueError("bad shape %s, expected leading %s" % (tuple(x.shape), tuple(shape)))
        return ctypes.c_void_p(x.data_ptr())

    @property
    def last_launch_count(self):
        return int(lib().kbe_last_launch_count(self._h))

    # -- allocation helpers (PyTorch owns the memory)
    def empty_triangle(self, n_rows=None):
        import torch
        n = self.n_max if n_rows is None else n_rows
        return torch.zeros((tri_size(n), self.M, self.M), dtype=torch.complex128, device="cuda")

    def empty_rows(self):
        import torch
        return torch.zeros((self.n_max, self.M, self.M), dtype=torch.complex128, device="cuda")

    def empty_slice(self):
        import torch
        return torch.zeros((2, self.n_max, self.M, self.M), dtype=torch.complex128, device="cuda")

    def empty_row_store(self, n_rows):
        import torch
        return torch.zeros((n_rows, 2, self.n_max, self.M, self.M), dtype=torch.complex128, device="cuda")

    def empty_ring(self):
        import torch
        return torch.zeros((KBE_RING_ROWS, 2, self.n_max, self.M, self.M), dtype=torch.complex128, device="cuda")

    # -- API
    def set_grid(self, t, order):
        t = np.ascontiguousarray(t, np.float64)
        order = np.ascontiguousarray(order, np.int32)
        self.t = t
        self.order = order
        self._check(lib().kbe_set_grid(self._h, _np_ptr(t), _np_ptr(order), len(t)))

    def set_model(self, h0, U, v, pulse=None):
        h0 = np.ascontiguousarray(h0, np.complex128)
        U = np.ascontiguousarray(U, np.float64)
        v = np.ascontiguousarray(v, np.float64)
        p = np.array([0.0, 0.0, 1.0, 0.0]) if pulse is None else np.array(
            [pulse["E0"], pulse["t0"], pulse["sigma"], pulse["omega"]], np.float64)
        self._check(lib().kbe_set_model(self._h, _np_ptr(h0), _np_ptr(U), _np_ptr(v), _np_ptr(p)))

    def set_interaction(self, U4):
        """General real four-index interaction U4[i, f, d, e] = U_ifde for
        Eq. (SE) and Eq. (eps); None returns to the model's local U."""
        if U4 is None:
            self._check(lib().kbe_set_interaction(self._h, None))
            return
        U4 = np.ascontiguousarray(U4, np.float64)
        if U4.shape != (self.M,) * 4:
            raise ValueError("U4 must have shape (M, M, M, M)")
        self._check(lib().kbe_set_interaction(self._h, _np_ptr(U4)))

    def set_thermal(self, beta, GM, k_tau=5):
        """Thermal branch (Sec. 2, Eq. KBE3) with the Matsubara function
        GM [n_tau, M, M] on the uniform tau grid of [0, beta]; None turns it
        off.  Sets the mixed row of t = 0 from G^M."""
        if GM is None:
            self._check(lib().kbe_set_thermal(self._h, ctypes.c_double(0.0), 0, 0, None))
            return
        GM = np.ascontiguousarray(GM, np.complex128)
        if GM.ndim != 3 or GM.shape[1:] != (self.M, self.M):
            raise ValueError("GM must have shape (n_tau, M, M)")
        self.n_tau = GM.shape[0]
        self._check(lib().kbe_set_thermal(self._h, ctypes.c_double(beta), self.n_tau, k_tau, _np_ptr(GM)))

    def mixed_rows(self, n_rows, stream=None):
        """Copy of the mixed rows G^|(t_r, tau_k), r < n_rows: [n_rows, n_tau, M, M]."""
        import torch
        n_tau = max(getattr(self, "n_tau", 0), 1)  # without a thermal branch the call reports KBE_ESTATE
        out = torch.empty((n_rows, n_tau, self.M, self.M), dtype=torch.complex128, device="cuda")
        self._check(lib().kbe_copy_mixed(self._h, n_rows, self._dev(out), 0, self._stream(stream)))
        return out

    def set_mixed_rows(self, rows, stream=None):
        """Load mixed rows [n_rows, n_tau, M, M] (device) into the context."""
        self._check(lib().kbe_copy_mixed(self._h, rows.shape[0], self._dev(rows), 1, self._stream(stream)))

    def selfenergy_slice(self, n, L, R, Sl, Sg, stream=None):
        self._check(lib().kbe_selfenergy_slice(self._h, n, self._dev(L), self._dev(R), self._dev(Sl),
                                               self._dev(Sg), self._stream(stream)))

    def selfenergy_all(self, n_rows, L, R, Sl, Sg, stream=None):
        self._check(lib().kbe_selfenergy_all(self._h, n_rows, self._dev(L), self._dev(R), self._dev(Sl),
                                             self._dev(Sg), self._stream(stream)))

    def history_slice(self, n, L, R, Sl, Sg, out, precision="fp64", stream=None):
        self._check(lib().kbe_history_slice(self._h, n, PRECISIONS[precision], self._dev(L), self._dev(R),
                                            self._dev(Sl), self._dev(Sg), self._dev(out), self._stream(stream)))

    def history_slice_band(self, n, row_lo, row_hi, L, R, Sl, Sg, out, stream=None):
        """One device's share of the FP64 slice of row n: the contributions
        of the stored rows [row_lo, row_hi) (kbe_history_slice_band)."""
        self._check(lib().kbe_history_slice_band(self._h, n, int(row_lo), int(row_hi), self._dev(L), self._dev(R),
                                                 self._dev(Sl), self._dev(Sg), self._dev(out), self._stream(stream)))

    def init_uncorrelated(self, rho0, L, R, stream=None):
        """kbe_init_uncorrelated: block (0,0) of L = i rho0, of R = -i 1."""
        rho = np.ascontiguousarray(np.asarray(rho0, np.complex128).reshape(self.M, self.M))
        self._check(lib().kbe_init_uncorrelated(self._h, _np_ptr(rho), self._dev(L), self._dev(R),
                                                self._stream(stream)))

    def rhs_row(self, j, L, R, Sl, Sg, I_work, F_ring, precision="fp64", stream=None):
        self._check(lib().kbe_rhs_row(self._h, j, PRECISIONS[precision], self._dev(L), self._dev(R),
                                      self._dev(Sl), self._dev(Sg), self._dev(I_work), self._dev(F_ring),
                                      self._stream(stream)))

    def step(self, n, L, R, Sl, Sg, I_work, F_ring, P=2, precision="fp64", stream=None):
        self._check(lib().kbe_step(self._h, n, P, PRECISIONS[precision], self._dev(L), self._dev(R),
                                   self._dev(Sl), self._dev(Sg), self._dev(I_work), self._dev(F_ring),
                                   self._stream(stream)))

    def run_steps(self, n_first, n_last, L, R, Sl, Sg, I_work, F_ring, P=2, precision="fp64", stream=None):
        """kbe_run_steps: the steps of rows n_first..n_last in one call."""
        self._check(lib().kbe_run_steps(self._h, int(n_first), int(n_last), P, PRECISIONS[precision],
                                        self._dev(L), self._dev(R), self._dev(Sl), self._dev(Sg),
                                        self._dev(I_work), self._dev(F_ring), self._stream(stream)))

    # -- the phases of a KBE_FP64 step (one system split by row bands)
    def step_predict(self, n, L, R, F_ring, stream=None):
        self._check(lib().kbe_step_predict(self._h, n, self._dev(L), self._dev(R), self._dev(F_ring),
                                           self._stream(stream)))

    def step_sweep_band(self, n, row_lo, row_hi, L, R, Sl, Sg, I_part, stream=None):
        self._check(lib().kbe_step_sweep_band(self._h, n, int(row_lo), int(row_hi), self._dev(L), self._dev(R),
                                              self._dev(Sl), self._dev(Sg), self._dev(I_part),
                                              self._stream(stream)))

    def step_sweep_finish(self, n, L, R, I, F_ring, stream=None):
        self._check(lib().kbe_step_sweep_finish(self._h, n, self._dev(L), self._dev(R), self._dev(I),
                                                self._dev(F_ring), self._stream(stream)))

    def step_host(self, n, L_host, R_host, F_host, L, R, Sl, Sg, I_work, F_ring, L_row_host, R_row_host, P=2,
                  precision="fp64", stream=None):
        """kbe_step_host: rows 0..n-1 of L, R and the ring F come from host
        tensors (page-locked for asynchronous copies) and row n of L, R is
        copied back to L_row_host, R_row_host; the upload overlaps the first
        history slice."""
        blk = self.M * self.M * 16
        row = (n + 1) * blk
        self._check(lib().kbe_step_host(self._h, n, P, PRECISIONS[precision],
                                        self._host(L_host, tri_size(n) * blk), self._host(R_host, tri_size(n) * blk),
                                        self._host(F_host, KBE_RING_ROWS * 2 * self.n_max * blk),
                                        self._dev(L), self._dev(R), self._dev(Sl), self._dev(Sg), self._dev(I_work),
                                        self._dev(F_ring), self._host(L_row_host, row), self._host(R_row_host, row),
                                        self._stream(stream)))

    def step_rows(self, n, L, R, Sl, Sg, I_work, F_rows, j0, P=2, precision="fp64", stream=None):
        """kbe_step with right-hand-side row j in slot j - j0 of the row store F_rows."""
        self._check(lib().kbe_step_rows(self._h, n, P, PRECISIONS[precision], self._dev(L), self._dev(R),
                                        self._dev(Sl), self._dev(Sg), self._dev(I_work), self._dev(F_rows),
                                        int(j0), int(F_rows.shape[0]), self._stream(stream)))

    # -- reverse mode
    def adjoint_slice(self, n, L, R, Sl, Sg, dI, dSl, dSg, dL, dR, row_lo, stream=None):
        """Vector-Jacobian product of the history slice of row n: dSl, dSg
        are overwritten, dL, dR (rows row_lo.. of a triangle) incremented."""
        self._check(lib().kbe_adjoint_slice(self._h, n, self._dev(L), self._dev(R), self._dev(Sl), self._dev(Sg),
                                            self._dev(dI), self._dev(dSl), self._dev(dSg), self._dev(dL),
                                            self._dev(dR), int(row_lo), self._stream(stream)))

    def adjoint_selfenergy_slice(self, n, L, R, dSl, dSg, dL_row, dR_row, dU, stream=None):
        """Vector-Jacobian product of the self-energy row n: dL_row, dR_row
        and dU (CUDA float64 [M]) incremented."""
        self._check(lib().kbe_adjoint_selfenergy_slice(self._h, n, self._dev(L), self._dev(R), self._dev(dSl),
                                                       self._dev(dSg), self._dev(dL_row), self._dev(dR_row),
                                                       self._real_dev(dU), self._stream(stream)))

    def step_adjoint(self, n, P, L, R, F_rows, j0, dL, dR, row_lo, dF_rows, dU, dE0, precision="fp64",
                     stream=None):
        """Reverse sweep of the step n taken by step_rows with the same
        precision ("fp64" or "df64"; see kbe.h)."""
        self._check(lib().kbe_step_adjoint(self._h, n, P, PRECISIONS[precision], self._dev(L), self._dev(R),
                                           self._dev(F_rows), int(j0),
                                           int(F_rows.shape[0]), self._dev(dL), self._dev(dR), int(row_lo),
                                           self._dev(dF_rows), self._real_dev(dU), self._real_dev(dE0),
                                           self._stream(stream)))

    @staticmethod
    def _real_dev(x):
        import torch
        if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("expected a contiguous CUDA float64 tensor")
        return ctypes.c_void_p(x.data_ptr())

    def set_adaptive_orders(self, K):
        """Choose the history quadrature order of each step on the device
        (Sec. 3.2), up to K (0: the grid's orders)."""
        self._check(lib().kbe_set_adaptive_orders(self._h, int(K)))

    def history_orders(self, n=None):
        """History order per interval 0..n-1 (the chosen ones in adaptive mode)."""
        n = self.n_max if n is None else int(n)
        out = np.zeros(n, np.int32)
        self._check(lib().kbe_get_history_orders(self._h, _np_ptr(out), n))
        return out

    def reset_cache(self):
        """Forget the split path's digit planes kept between steps."""
        self._check(lib().kbe_reset_cache(self._h))

    def run_controlled(self, rho0, rtol, atol, dt0, t_end, q_max=12, k_hist=5, K_sel=0, h_max=0.0,
                       precision="fp64", stream=None):
        """Adaptive time stepping (Sec. 3.1, kbe_run_controlled) from the
        uncorrelated state rho0 to t_end; the run chooses the grid.  Returns
        a dict: ``t``, ``q`` (order per step), ``korder`` (history order per
        interval), ``n`` (rows), ``stats`` (steps, error-test failures,
        convergence failures, right-hand-side evaluations, reconstructed
        blocks), the device triangles ``L``, ``R`` and ``status`` (KBE_OK, or
        KBE_ERANGE when n_max rows filled first)."""
        import torch
        M = self.M
        L, R = self.empty_triangle(), self.empty_triangle()
        L[0].copy_(1j * torch.as_tensor(np.asarray(rho0, np.complex128), device="cuda"))
        R[0].copy_(-1j * torch.eye(M, dtype=torch.complex128, device="cuda"))
        Sl, Sg, I, F = self.empty_rows(), self.empty_rows(), self.empty_slice(), self.empty_ring()
        opts = np.array([rtol, atol, dt0, h_max, t_end], np.float64)
        iopts = np.array([q_max, k_hist, K_sel, PRECISIONS[precision]], np.int32)
        t = np.zeros(self.n_max)
        q = np.zeros(self.n_max, np.int32)
        ko = np.zeros(self.n_max, np.int32)
        n_rows = ctypes.c_int()
        stats = np.zeros(5, np.int32)
        st = lib().kbe_run_controlled(self._h, _np_ptr(opts), _np_ptr(iopts), self._dev(L), self._dev(R),
                                      self._dev(Sl), self._dev(Sg), self._dev(I), self._dev(F), _np_ptr(t),
                                      _np_ptr(q), _np_ptr(ko), ctypes.byref(n_rows), _np_ptr(stats),
                                      self._stream(stream))
        if st not in (KBE_OK, KBE_ERANGE):
            self._check(st)
        n = n_rows.value
        return {"t": t[:n], "q": q[:n], "korder": ko[:n], "n": n, "stats": tuple(int(x) for x in stats),
                "L": L, "R": R, "status": int(st)}

    def set_split_planes(self, keep):
        """kbe_set_split_planes: keep (True) or drop (False) the digit-plane cache of the split path."""
        self._check(lib().kbe_set_split_planes(self._h, 1 if keep else 0))

    def debug_withhold_run(self, barrier, spin_limit):
        """Failure-path test of the next cooperative run launch (kbe_debug_withhold_run)."""
        self._check(lib().kbe_debug_withhold_run(self._h, int(barrier), int(spin_limit)))

    def debug_withhold_split(self, unit, spin_limit):
        """Failure-path test of the next split contraction (kbe_debug_withhold_split)."""
        self._check(lib().kbe_debug_withhold_split(self._h, int(unit), int(spin_limit)))

    def set_profiling(self, enable):
        """Record CUDA events around each contraction kernel (clears old records)."""
        self._check(lib().kbe_set_profiling(self._h, 1 if enable else 0))

    def read_profiling(self):
        """(number of contraction kernels timed, their total milliseconds)."""
        n = ctypes.c_int()
        ms = ctypes.c_double()
        self._check(lib().kbe_read_profiling(self._h, ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value

    def sync_status(self, stream=None):
        """Synchronize and raise if a kernel flagged a problem."""
        self._check(lib().kbe_sync_status(self._h, self._stream(stream)))


class Run:
    """Device state of one run: triangles, self-energy rows, history slice
    and the right-hand-side ring, plus the calls that advance it."""

    def __init__(self, ctx):
        self.ctx = ctx
        self.L = ctx.empty_triangle()
        self.R = ctx.empty_triangle()
        self.Sl = ctx.empty_rows()
        self.Sg = ctx.empty_rows()
        self.I = ctx.empty_slice()
        self.F = ctx.empty_ring()

    def init_uncorrelated(self, rho0, stream=None):
        """Row 0 from G^<(0,0) = i rho0, G^R(0,0) = -i (kbe_init_uncorrelated),
        and its right-hand side."""
        self.ctx.init_uncorrelated(rho0, self.L, self.R, stream=stream)
        self.ctx.rhs_row(0, self.L, self.R, self.Sl, self.Sg, self.I, self.F, stream=stream)

    def step(self, n, P=2, precision="fp64", stream=None):
        self.ctx.step(n, self.L, self.R, self.Sl, self.Sg, self.I, self.F, P=P, precision=precision,
                      stream=stream)

    def run_steps(self, n_first, n_last, P=2, precision="fp64", stream=None):
        self.ctx.run_steps(n_first, n_last, self.L, self.R, self.Sl, self.Sg, self.I, self.F, P=P,
                           precision=precision, stream=stream)

    def step_host(self, n, L_host, R_host, F_host, L_row_host, R_row_host, P=2, precision="fp64", stream=None):
        """One step with the history and ring uploaded from host tensors and
        the new row downloaded (Context.step_host on this run's buffers)."""
        self.ctx.step_host(n, L_host, R_host, F_host, self.L, self.R, self.Sl, self.Sg, self.I, self.F,
                           L_row_host, R_row_host, P=P, precision=precision, stream=stream)


# ---------------------------------------------------------------- batching
class Batch:
    """Independent systems advanced by one batched KBE step (kbe_batch_*).

    ``runs`` is a list of Run objects (each on its own Context with grid and
    model set); their device state is bound to the batch."""

    def __init__(self, runs):
        self.runs = list(runs)
        arr = (ctypes.c_void_p * len(self.runs))(*[r.ctx._h.value for r in self.runs])
        h = ctypes.c_void_p()
        _raise(lib().kbe_batch_create(arr, len(self.runs), ctypes.byref(h)))
        self._h = h
        for i, r in enumerate(self.runs):
            self._check(lib().kbe_batch_bind(self._h, i, r.ctx._dev(r.L), r.ctx._dev(r.R), r.ctx._dev(r.Sl),
                                             r.ctx._dev(r.Sg), r.ctx._dev(r.I), r.ctx._dev(r.F)))

    def _check(self, status):
        if status != KBE_OK:
            raise KBEError(status, lib().kbe_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().kbe_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _rows(rows):
        r = np.ascontiguousarray(rows, np.int32)
        return r, _np_ptr(r)

    def step(self, rows, P=2, precision="fp64", stream=None):
        r, p = self._rows(rows)
        self._check(lib().kbe_batch_step(self._h, p, P, PRECISIONS[precision], Context._stream(stream)))

    @property
    def last_launch_count(self):
        return int(lib().kbe_batch_last_launch_count(self._h))

    def set_policy(self, block, item_work_log2):
        self._check(lib().kbe_batch_set_policy(self._h, block, item_work_log2))

    def policy(self):
        b, w = ctypes.c_int(), ctypes.c_int()
        self._check(lib().kbe_batch_get_policy(self._h, ctypes.byref(b), ctypes.byref(w)))
        return b.value, w.value

    def autotune(self, rows, reps=2, stream=None):
        """Time the candidate tile policies at ``rows``; keep and return the
        fastest as (block, item_work_log2, ms)."""
        r, p = self._rows(rows)
        b, w, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        self._check(lib().kbe_batch_autotune(self._h, p, reps, Context._stream(stream), ctypes.byref(b),
                                             ctypes.byref(w), ctypes.byref(ms)))
        return b.value, w.value, ms.value

    def sync_status(self, stream=None):
        self._check(lib().kbe_batch_sync_status(self._h, Context._stream(stream)))


# ------------------------------------------------------------ reverse mode
class Window:
    """A window of KBE steps n_start..n_end-1 restarted from frozen rows,
    as a function of the interaction U (per orbital) and the pulse
    amplitude E0, with its reverse sweep.

    Rows 0..n_start-1 of ``L``/``R`` (CUDA triangles of at least n_end
    rows) and the right-hand-side rows j0..n_start-1 in ``F_frozen``
    (mapping j -> [2, j+1, M, M]) are constants.  ``forward`` runs the
    window through the library's stepper (``precision`` "fp64" or "df64")
    keeping every right-hand-side row (the checkpoints), and returns the
    final diagonal block L(n_end-1, n_end-1); ``backward`` sweeps
    kbe_step_adjoint from the last step down and returns (dU, dE0) for a
    cotangent of that block.
    """

    def __init__(self, ctx, L, R, F_frozen, n_start, n_end, h0, v, pulse, P=2, precision="fp64"):
        import torch
        if precision not in ("fp64", "df64"):
            raise ValueError("precision must be 'fp64' or 'df64'")
        self.ctx, self.P, self.precision = ctx, int(P), precision
        self.n_start, self.n_end = int(n_start), int(n_end)
        self.h0 = np.ascontiguousarray(h0, np.complex128)
        self.v = np.ascontiguousarray(v, np.float64)
        self.pulse = dict(pulse) if pulse is not None else dict(E0=0.0, t0=0.0, sigma=1.0, omega=0.0)
        self.L, self.R = L, R
        self.j0 = min(F_frozen) if F_frozen else self.n_start
        self.F = ctx.empty_row_store(self.n_end - self.j0)
        for j, f in F_frozen.items():
            self.F[j - self.j0, :, : j + 1].copy_(torch.as_tensor(np.asarray(f), device="cuda"))
        self.Sl, self.Sg, self.I = ctx.empty_rows(), ctx.empty_rows(), ctx.empty_slice()
        self._state = None

    def _set_params(self, U, E0):
        p = dict(self.pulse, E0=float(E0))
        self.ctx.set_model(self.h0, np.asarray(U, np.float64), self.v, p)

    def forward(self, U, E0, stream=None):
        U = np.array(U, np.float64)
        self._set_params(U, E0)
        for n in range(self.n_start, self.n_end):
            self.ctx.step_rows(n, self.L, self.R, self.Sl, self.Sg, self.I, self.F, self.j0, P=self.P,
                               precision=self.precision, stream=stream)
        self._state = (U.tobytes(), float(E0))
        p = tri_size(self.n_end) - 1
        return self.L[p].clone()

    def backward(self, grad_block, U, E0, stream=None):
        import torch
        U = np.array(U, np.float64)
        if self._state != (U.tobytes(), float(E0)):
            self.forward(U, E0, stream=stream)   # the rows must be those of (U, E0)
        self._set_params(U, E0)
        M, lo = self.ctx.M, self.n_start
        base = tri_size(lo)
        nblk = tri_size(self.n_end) - base
        dL = torch.zeros((nblk, M, M), dtype=torch.complex128, device="cuda")
        dR = torch.zeros_like(dL)
        dL[tri_size(self.n_end) - 1 - base].copy_(torch.as_tensor(grad_block, dtype=torch.complex128))
        dF = torch.zeros_like(self.F)
        dU = torch.zeros(M, dtype=torch.float64, device="cuda")
        dE0 = torch.zeros(1, dtype=torch.float64, device="cuda")
        for n in range(self.n_end - 1, self.n_start - 1, -1):
            self.ctx.step_adjoint(n, self.P, self.L, self.R, self.F, self.j0, dL, dR, lo, dF, dU, dE0,
                                  precision=self.precision, stream=stream)
        return dU, dE0[0]


def _window_function():
    import torch

    class WindowFunction(torch.autograd.Function):
        """Final diagonal block of a Window as a differentiable function of
        (U, E0); the backward pass runs the library's adjoint kernels."""

        @staticmethod
        def forward(fctx, U, E0, window):
            fctx.window = window
            fctx.save_for_backward(U, E0)
            return window.forward(U.detach().cpu().numpy(), float(E0))

        @staticmethod
        def backward(fctx, grad):
            U, E0 = fctx.saved_tensors
            dU, dE0 = fctx.window.backward(grad.contiguous(), U.detach().cpu().numpy(), float(E0))
            return dU.to(U.device, U.dtype), dE0.to(E0.device, E0.dtype).reshape(E0.shape), None

    return WindowFunction


def window_final_block(U, E0, window):
    """Differentiable L(n_end-1, n_end-1) of ``window`` (a Window) for the
    float64 tensors U [M] and E0 (scalar)."""
    global _WF
    if _WF is None:
        _WF = _window_function()
    return _WF.apply(U, E0, window)


_WF = None
