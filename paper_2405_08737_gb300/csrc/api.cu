// api.cu -- the C ABI of libkbe (declared in include/kbe.h): argument
// validation, device workspace, and the launch sequences of each call.

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "kbe_internal.h"

using namespace kbe;

namespace {

thread_local std::string g_create_err;

kbe_status fail(kbe_ctx* ctx, kbe_status st, const std::string& msg) {
  if (ctx) ctx->err = msg; else g_create_err = msg;
  return st;
}

kbe_status cuda_fail(kbe_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, KBE_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool aligned16(const void* p) { return p && (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

WeightsView weights_view(const kbe_ctx* ctx) {
  return WeightsView{ctx->d_wbar, ctx->d_band, ctx->band_w};
}

template <class T> cudaError_t dev_alloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T) + 16);
}

void release(kbe_ctx* ctx) {
  for (cudaEvent_t ev : ctx->ev_pool) cudaEventDestroy(ev);
  ctx->ev_pool.clear();
  for (cudaEvent_t& ev : ctx->up_ev) {
    if (ev) cudaEventDestroy(ev);
    ev = nullptr;
  }
  if (ctx->up_start) cudaEventDestroy(ctx->up_start);
  if (ctx->up_stream) cudaStreamDestroy(ctx->up_stream);
  ctx->up_start = nullptr;
  ctx->up_stream = nullptr;
  cudaFree(ctx->d_wbar); cudaFree(ctx->d_band); cudaFree(ctx->d_corr); cudaFree(ctx->d_pred);
  cudaFree(ctx->d_h0); cudaFree(ctx->d_U); cudaFree(ctx->d_v); cudaFree(ctx->d_eps);
  cudaFree(ctx->d_part); cudaFree(ctx->d_status); cudaFree(ctx->d_split); cudaFree(ctx->d_adj);
  cudaFree(ctx->d_runbar);
  ctx->d_runbar = nullptr;
  cudaFree(ctx->d_planes);
  cudaFree(ctx->d_hist);
  cudaFree(ctx->d_korder);
  cudaFree(ctx->d_Ut); cudaFree(ctx->d_Xt); cudaFree(ctx->d_HF);
  ctx->d_Ut = ctx->d_Xt = ctx->d_HF = nullptr;
  cudaFree(ctx->d_ctl);
  ctx->d_ctl = nullptr;
  ctx->ctl_bytes = 0;
  cudaFree(ctx->d_th);
  ctx->d_th = nullptr;
  ctx->thermal = false;
  ctx->dense = false;
  ctx->d_hist = nullptr;
  ctx->d_korder = nullptr;
  ctx->d_planes = nullptr;
  ctx->planes_layout = SplitPlanes{};
  ctx->planes_L = ctx->planes_R = nullptr;
  ctx->planes_rows = 0;
  ctx->d_split = nullptr;
  ctx->d_adj = nullptr;
  ctx->adj_bytes = 0;
  ctx->d_wbar = ctx->d_band = ctx->d_corr = ctx->d_pred = nullptr;
  ctx->d_h0 = ctx->d_U = ctx->d_v = ctx->d_eps = ctx->d_part = nullptr;
  ctx->d_status = nullptr;
}

// set the device the context was created on
kbe_status use_device(kbe_ctx* ctx) {
  cudaError_t e = cudaSetDevice(ctx->device);
  return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "cudaSetDevice");
}

kbe_status check_row_call(kbe_ctx* ctx, int n) {
  if (!ctx->grid_set) return fail(ctx, KBE_ESTATE, "no grid: call kbe_set_grid first");
  if (n < 0 || n >= ctx->grid.n_t) return fail(ctx, KBE_ERANGE, "row n outside the grid");
  return KBE_OK;
}

// Next event pair of the measurement pool (nullptr when profiling is off).
bool next_events(kbe_ctx* ctx, cudaEvent_t* b, cudaEvent_t* e) {
  *b = *e = nullptr;
  if (!ctx->profiling) return true;
  while (ctx->ev_pool.size() < 2 * (ctx->ev_used + 1)) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) return false;
    ctx->ev_pool.push_back(ev);
  }
  *b = ctx->ev_pool[2 * ctx->ev_used];
  *e = ctx->ev_pool[2 * ctx->ev_used + 1];
  ++ctx->ev_used;
  return true;
}

// History slice of row n.  `stepping` is set by the KBE step: rows below n
// of L, R are then final, so digit planes encoded for them by earlier slices
// of the same arrays are reused (the split path re-encodes only units that
// involve rows >= the cached row count).
struct Staged;
kbe_status history(kbe_ctx* ctx, int n, int precision, const void* L, const void* R, const void* Sl,
                   const void* Sg, void* I_out, cudaStream_t s, int* launches, bool stepping = false,
                   const Staged* staged = nullptr);

// Rows arriving in chunks (kbe_step_host): chunk k is complete once ev[k]
// has fired, and the output columns [c_lo[k], c_hi[k]) read only rows of
// chunks 0..k.
struct Staged {
  int k = 0;
  int c_lo[16], c_hi[16];
  cudaEvent_t ev[16];
};

kbe_status history(kbe_ctx* ctx, int n, int precision, const void* L, const void* R, const void* Sl,
                   const void* Sg, void* I_out, cudaStream_t s, int* launches, bool stepping,
                   const Staged* staged) {
  if (precision == KBE_SPLIT_BF16) {
    if (!ctx->d_split) return fail(ctx, KBE_EINVAL, "split precision needs 1 <= norb <= 32");
    SplitLaunch l{ctx->M, n, (const double*)L, (const double*)R, (const double*)Sl, (const double*)Sg,
                  weights_view(ctx), (double*)I_out, ctx->d_split, ctx->split_bytes, ctx->d_status};
    if (!next_events(ctx, &l.ev_begin, &l.ev_end)) return fail(ctx, KBE_ECUDA, "profiling: cudaEventCreate");
    if (ctx->split_planes && !ctx->d_planes && !ctx->planes_failed) {
      SplitPlanes lay;
      if (!split_planes_layout(ctx->M, ctx->n_max, &lay) || cudaMalloc(&ctx->d_planes, lay.bytes) != cudaSuccess) {
        cudaGetLastError();
        ctx->d_planes = nullptr;
        ctx->planes_failed = true;  // not enough memory: convert inside the contraction kernel instead
      } else {
        ctx->planes_layout = lay;
        ctx->planes_rows = 0;
        ctx->planes_L = ctx->planes_R = nullptr;
      }
    }
    l.withhold = ctx->dbg_withhold;
    l.spin_limit = ctx->dbg_spin;
    ctx->dbg_withhold = -1;  // one launch only
    ctx->dbg_spin = 0;
    cudaError_t e;
    if (ctx->split_planes && ctx->d_planes) {
      int r0 = 0;
      if (stepping && ctx->planes_L == L && ctx->planes_R == R && ctx->planes_rows <= n) r0 = ctx->planes_rows;
      e = launch_history_split2(l, ctx->planes_layout, ctx->d_planes, r0, s, launches);
      if (e == cudaSuccess) {  // rows below n are final during a step; otherwise nothing is kept
        ctx->planes_L = stepping ? L : nullptr;
        ctx->planes_R = stepping ? R : nullptr;
        ctx->planes_rows = stepping ? n : 0;
      } else {
        ctx->planes_L = ctx->planes_R = nullptr;
        ctx->planes_rows = 0;
      }
    } else {
      e = launch_history_split(l, s, launches);
    }
    return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "split history slice launch");
  }
  if (precision != KBE_FP64 && precision != KBE_DF64) return fail(ctx, KBE_EINVAL, "unknown precision");
  HistoryArgs a{ctx->M, n, (const double*)L, (const double*)R, (const double*)Sl, (const double*)Sg,
                weights_view(ctx), (double*)I_out, ctx->d_part, ctx->part_bytes, ctx->d_status};
  cudaError_t e;
  if (precision == KBE_DF64) {
    if (!next_events(ctx, &a.ev_begin, &a.ev_end)) return fail(ctx, KBE_ECUDA, "profiling: cudaEventCreate");
    e = launch_history_df(a, s, launches);
    return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "history slice launch");
  }
  if (staged) {  // the column ranges contract as their rows arrive (no timing events: they would hold the waits)
    e = launch_history_f64_ranges(a, staged->k, staged->c_lo, staged->c_hi, staged->ev, s, launches);
    return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "history slice launch");
  }
  if (!next_events(ctx, &a.ev_begin, &a.ev_end)) return fail(ctx, KBE_ECUDA, "profiling: cudaEventCreate");
  e = launch_history_f64(a, s, launches);
  return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "history slice launch");
}

// Self-energy of n_blocks blocks from first_block (launch_sigma geometry),
// with the context's interaction: the local U or the dense tensor.
cudaError_t sigma_blocks(kbe_ctx* ctx, int64_t first_block, int64_t n_blocks, int64_t diag_rel, const void* L,
                         const void* R, void* Sl, void* Sg, cudaStream_t s) {
  if (ctx->dense)
    return launch_sigma_dense(ctx->M, first_block, n_blocks, diag_rel, (const double*)L, (const double*)R,
                              ctx->d_Ut, ctx->d_Xt, (double*)Sl, (double*)Sg, ctx->d_status, s);
  return launch_sigma(ctx->M, first_block, n_blocks, diag_rel, (const double*)L, (const double*)R, ctx->d_U,
                      (double*)Sl, (double*)Sg, ctx->d_status, s);
}

StepArgs step_args(kbe_ctx* ctx, int n, void* L, void* R, const void* I, void* F) {
  const HostGrid& g = ctx->grid;
  StepArgs a{};
  a.M = ctx->M;
  a.n = n;
  a.K = g.K;
  a.kn = n > 0 ? g.order[n] : 1;
  a.field = ctx->model.field(g.t[n]);
  a.L = (double*)L;
  a.R = (double*)R;
  a.F = (double*)F;
  a.n_max = ctx->n_max;
  a.f_base = 0;
  a.f_rows = kRing;
  a.I = (const double*)I;
  a.h0 = ctx->d_h0;
  a.U = ctx->d_U;
  a.HF = ctx->dense ? ctx->d_HF : nullptr;
  a.v = ctx->d_v;
  a.eps = ctx->d_eps;
  a.corr = ctx->d_corr + (size_t)n * kMaxOrder * kWTab;
  a.pred = ctx->d_pred + (size_t)n * kMaxOrder * kWTab;
  a.status = ctx->d_status;
  return a;
}


// ------------------------------------------------------- thermal branch --
struct ThermalLayout {
  double *GM, *left, *Smix, *Smw, *Aw, *Fx, *Gx;
  float4 *Smwf, *Awf;
};

// doubles of the tau-weight table, padded so that the complex arrays after
// it start on 256-byte boundaries (the kernels load them as double2)
size_t thermal_left_doubles(size_t N) { return (N * N + 31) / 32 * 32; }

ThermalLayout thermal_layout(kbe_ctx* ctx) {
  const size_t MM = (size_t)ctx->M * ctx->M, N = ctx->th_N;
  double* w = ctx->d_th;
  ThermalLayout t;
  t.GM = w;    w += N * MM * 2;
  t.left = w;  w += thermal_left_doubles(N);
  t.Smix = w;  w += N * MM * 2;
  t.Smw = w;   w += N * MM * 2;
  t.Aw = w;    w += (size_t)ctx->n_max * MM * 2;
  t.Fx = w;    w += (size_t)kRing * N * MM * 2;
  t.Gx = w;    w += (size_t)ctx->n_max * N * MM * 2;
  t.Smwf = reinterpret_cast<float4*>(w);  w += N * MM * 2;
  t.Awf = reinterpret_cast<float4*>(w);
  return t;
}

ThermalArgs thermal_args(kbe_ctx* ctx, const StepArgs& a, const void* Sl, const void* Sg, void* I) {
  const ThermalLayout t = thermal_layout(ctx);
  ThermalArgs x;
  x.M = ctx->M;
  x.N = ctx->th_N;
  x.n = a.n;
  x.kn = a.kn;
  x.U = ctx->d_U;
  x.Sl = (const double*)Sl;
  x.Sg = (const double*)Sg;
  x.w = weights_view(ctx);
  x.eps = ctx->d_eps;
  x.GM = t.GM;
  x.left = t.left;
  x.Gx = t.Gx;
  x.Smix = t.Smix;
  x.Smw = t.Smw;
  x.Aw = t.Aw;
  x.Smwf = t.Smwf;
  x.Awf = t.Awf;
  x.df = 0;
  x.Fx = t.Fx;
  x.I = (double*)I;
  x.corr = a.corr;
  x.pred = a.pred;
  x.status = ctx->d_status;
  return x;
}

// tau weights of the thermal branch: row j integrates over [0, tau_j]; each
// interval takes the interpolatory rule (Eq. weights, LU-solved) through
// kap + 1 = min(k, j) + 1 consecutive nodes containing it, centred where
// possible and kept inside [0, tau_j]
kbe_status thermal_weights(int N, double beta, int k, std::vector<double>* left, std::string* err) {
  std::vector<double> tau(N);
  for (int i = 0; i < N; ++i) tau[i] = beta * i / (N - 1);
  left->assign((size_t)N * N, 0.0);
  double w[kWTab];
  for (int j = 1; j < N; ++j) {
    const int kap = std::min(k, j);
    for (int l = 1; l <= j; ++l) {
      const int s0 = std::max(0, std::min(l - 1 - (kap - 1) / 2, j - kap));
      kbe_status st = local_weights(tau.data() + s0, kap, tau[l - 1], tau[l], w, err);
      if (st != KBE_OK) return st;
      for (int i = 0; i <= kap; ++i) (*left)[(size_t)j * N + s0 + i] += w[i];
    }
  }
  return KBE_OK;
}

// the thermal kernels of one sweep after the history slice (Sigma^|, mixed
// term into I), and the mixed right-hand side after the Fock matrix
cudaError_t thermal_sweep_a(kbe_ctx* ctx, const ThermalArgs& x, cudaStream_t s) {
  cudaError_t e = launch_th_sigma(x, s);
  if (e == cudaSuccess) e = launch_th_mixed(x, s);
  return e;
}

// One KBE step (predictor, then P rounds of self-energy, history slice,
// Fock matrix, right-hand side and corrector).  F rows are addressed as
// slot (j - f_base) % f_rows.  With save != nullptr, row n of L and R is
// copied to save[p] before round p and to save[P] at the end
// (save[p] = [2][n+1][M][M]: L row, then R row).
// With staged != nullptr the history rows and F arrive in chunks (kbe_step_host):
// the predictor waits for chunk 0 (F and the rows next to n), and the first
// FP64 history slice contracts its column ranges as their rows arrive.
kbe_status step_impl(kbe_ctx* ctx, int n, int P, int precision, void* L, void* R, void* Sl, void* Sg, void* I_work,
                     void* F, int f_base, int f_rows, cudaStream_t s, double* save, int* count_out,
                     const Staged* staged = nullptr) {
  StepArgs a = step_args(ctx, n, L, R, I_work, F);
  a.f_base = f_base;
  a.f_rows = f_rows;
  const size_t MM = (size_t)ctx->M * ctx->M;
  const size_t row_doubles = (size_t)(n + 1) * MM * 2;
  double* Lrow = (double*)L + tri(n, 0) * MM * 2;
  double* Rrow = (double*)R + tri(n, 0) * MM * 2;
  auto keep = [&](int p) -> cudaError_t {
    if (!save) return cudaSuccess;
    double* dst = save + (size_t)p * 2 * row_doubles;
    cudaError_t e = cudaMemcpyAsync(dst, Lrow, row_doubles * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dst + row_doubles, Rrow, row_doubles * sizeof(double), cudaMemcpyDeviceToDevice, s);
    return e;
  };
  int count = 0, nl = 0;
  cudaError_t e = cudaSuccess;
  if (staged && (e = cudaStreamWaitEvent(s, staged->ev[0], 0)) != cudaSuccess)
    return cuda_fail(ctx, e, "kbe_step: wait for the uploaded rows");
  const bool pipelined = staged && precision == KBE_FP64 && ctx->adaptive_K == 0 && !ctx->thermal;
  if (staged && !pipelined && (e = cudaStreamWaitEvent(s, staged->ev[staged->k - 1], 0)) != cudaSuccess)
    return cuda_fail(ctx, e, "kbe_step: wait for the uploaded rows");
  e = launch_predictor(a, s);
  ++count;
  if (e == cudaSuccess && ctx->thermal) {
    e = launch_th_adams(thermal_args(ctx, a, Sl, Sg, I_work), false, s);
    ++count;
  }
  *count_out = count;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "kbe_step: predictor");
  for (int it = 0; it < P; ++it) {
    if ((e = keep(it)) != cudaSuccess) return cuda_fail(ctx, e, "kbe_step: iterate copy");
    e = sigma_blocks(ctx, tri(n, 0), n + 1, n, L, R, Sl, Sg, s);
    *count_out = ++count;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kbe_step: self-energy");
    if (ctx->adaptive_K > 0) {  // history order of interval n from this sweep's rows (Sec. 3.2)
      SelectArgs sa{ctx->M, n, ctx->adaptive_K, (const double*)L, (const double*)R, (const double*)Sl,
                    (const double*)Sg, ctx->d_hist + (size_t)n * kMaxOrder * kWTab, ctx->d_band, ctx->d_wbar,
                    ctx->band_w, ctx->d_korder};
      sa.u = ctx->d_hist + (size_t)ctx->n_max * kMaxOrder * kWTab;
      int ns = 0;
      e = launch_select_order(sa, s, &ns);
      *count_out = (count += ns);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "kbe_step: history order selection");
    }
    kbe_status st = history(ctx, n, precision, L, R, Sl, Sg, I_work, s, &nl, true,
                            pipelined && it == 0 ? staged : nullptr);
    *count_out = (count += nl);
    if (st != KBE_OK) return st;
    if (ctx->thermal) {
      ThermalArgs x = thermal_args(ctx, a, Sl, Sg, I_work);
      x.df = precision != KBE_FP64;  // the thermal sums in double-float with the faster contractions
      if ((e = thermal_sweep_a(ctx, x, s)) != cudaSuccess || (e = launch_fock(a, s)) != cudaSuccess ||
          (e = launch_rhs_corrector(a, s)) != cudaSuccess || (e = launch_th_rhs(x, s)) != cudaSuccess ||
          (e = launch_th_adams(x, true, s)) != cudaSuccess) {
        *count_out = count + 7;
        return cuda_fail(ctx, e, "kbe_step: thermal corrector");
      }
      *count_out = (count += 7);
      continue;
    }
    if ((e = launch_fock(a, s)) != cudaSuccess || (e = launch_rhs_corrector(a, s)) != cudaSuccess) {
      *count_out = count + 3;
      return cuda_fail(ctx, e, "kbe_step: corrector");
    }
    *count_out = (count += 3);
  }
  if ((e = keep(P)) != cudaSuccess) return cuda_fail(ctx, e, "kbe_step: iterate copy");
  return KBE_OK;
}

kbe_status check_step_call(kbe_ctx* ctx, int n, int P, int precision, const void* L, const void* R, const void* Sl,
                           const void* Sg, const void* I_work, const void* F) {
  kbe_status st = check_row_call(ctx, n);
  if (st != KBE_OK) return st;
  if (n < 1) return fail(ctx, KBE_ERANGE, "kbe_step: n must be >= 1 (row 0 is the initial state)");
  if (P < 1 || P > 16) return fail(ctx, KBE_EINVAL, "kbe_step: P outside [1, 16]");
  if (!ctx->model.set) return fail(ctx, KBE_ESTATE, "no model: call kbe_set_model first");
  if (!aligned16(L) || !aligned16(R) || !aligned16(Sl) || !aligned16(Sg) || !aligned16(I_work) || !aligned16(F))
    return fail(ctx, KBE_EINVAL, "kbe_step: NULL or misaligned pointer");
  if (precision != KBE_FP64 && precision != KBE_SPLIT_BF16 && precision != KBE_DF64)
    return fail(ctx, KBE_EINVAL, "kbe_step: unknown precision");
  if (ctx->adaptive_K > 0) {
    if (n > ctx->adaptive_rows)
      return fail(ctx, KBE_ESTATE, "kbe_step: adaptive history orders need the steps in order (row " +
                                       std::to_string(ctx->adaptive_rows) + " is next)");
    ctx->adaptive_rows = n + 1;  // rows above n are stepped again
  }
  return use_device(ctx);
}

// Rows of a right-hand-side row store needed by step n: n - k_n .. n.
kbe_status check_row_store(kbe_ctx* ctx, int n, int j0, int n_rows) {
  if (n_rows < 1 || j0 < 0) return fail(ctx, KBE_EINVAL, "row store: n_rows < 1 or j0 < 0");
  if (n - ctx->grid.order[n] < j0) return fail(ctx, KBE_ERANGE, "row store: step n needs rows from n - k_n < j0");
  if (n - j0 >= n_rows) return fail(ctx, KBE_ERANGE, "row store: row n is beyond the store (n - j0 >= n_rows)");
  return KBE_OK;
}

// Reverse-mode workspace: 13 + 2 (P + 1) rows of n_max M^2 complex.
constexpr int kAdjFixedRows = 13;
kbe_status adjoint_workspace(kbe_ctx* ctx, int P) {
  const size_t row = (size_t)ctx->n_max * ctx->M * ctx->M * 16;
  const size_t need = (kAdjFixedRows + 2 * (size_t)(P + 1)) * row;
  if (ctx->adj_bytes >= need) return KBE_OK;
  cudaFree(ctx->d_adj);
  ctx->d_adj = nullptr;
  ctx->adj_bytes = 0;
  cudaError_t e = cudaMalloc(&ctx->d_adj, need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, e == cudaErrorMemoryAllocation ? KBE_ENOMEM : KBE_ECUDA,
                std::string("adjoint workspace: ") + cudaGetErrorString(e));
  }
  ctx->adj_bytes = need;
  return KBE_OK;
}


// ------------------------------------------------- adaptive time stepping --
// Host side of kbe_run_controlled (Sec. 3.1): the step/order controller in
// FP64 on the host, every vector operation on the device.

// integral over [t_{n-1}, t_n] of prod_i (t - nodes_i): the polynomial in
// u = (t - t_{n-1}) / h is expanded in monomials and integrated over [0, 1]
double error_integral(const double* t, int n, const int* nodes, int cnt) {
  const double h = t[n] - t[n - 1];
  double c[kWTab + 2] = {1.0};
  int deg = 0;
  for (int i = 0; i < cnt; ++i) {  // multiply by (u - u_i)
    const double ui = (t[nodes[i]] - t[n - 1]) / h;
    c[deg + 1] = 0.0;
    for (int k = deg + 1; k >= 1; --k) c[k] = c[k - 1] - ui * c[k];
    c[0] = -ui * c[0];
    ++deg;
  }
  double s = 0.0;
  for (int k = 0; k <= deg; ++k) s += c[k] / (k + 1);
  return s * std::pow(h, cnt + 1);
}

// divided-difference coefficients over t_n, t_{n-1}, ..., t_{n-qq}
void divdiff_coeffs(const double* t, int n, int qq, double* alpha) {
  for (int i = 0; i <= qq; ++i) {
    double d = 1.0;
    for (int k = 0; k <= qq; ++k)
      if (k != i) d *= t[n - i] - t[n - k];
    alpha[i] = 1.0 / d;
  }
}

struct CtlRun {
  kbe_ctx* ctx;
  cudaStream_t s;
  int M, n_max, precision, K_sel, k_hist, bw;
  void *L, *R, *Sl, *Sg, *I, *F;
  double *Sring, *eps_ring, *ypred, *ycur, *partial, *out;
  int nfev = 0, nrecon = 0, launches = 0;
};

kbe_status ctl_workspace(kbe_ctx* ctx) {
  const size_t MM = (size_t)ctx->M * ctx->M, nm = ctx->n_max;
  const size_t need = (kRing * 2 * nm * MM + kRing * MM + 4 * nm * MM) * 16 +
                      (2 * (size_t)ctl_partial_count(ctx->n_max, ctx->M) + 4) * sizeof(double);
  if (ctx->ctl_bytes >= need) return KBE_OK;
  cudaFree(ctx->d_ctl);
  ctx->d_ctl = nullptr;
  ctx->ctl_bytes = 0;
  cudaError_t e = cudaMalloc(&ctx->d_ctl, need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, e == cudaErrorMemoryAllocation ? KBE_ENOMEM : KBE_ECUDA,
                std::string("kbe_run_controlled: workspace: ") + cudaGetErrorString(e));
  }
  ctx->ctl_bytes = need;
  return KBE_OK;
}

// right-hand side row n from the current row n (Sigma, order choice, slice, eps, F)
kbe_status ctl_feval(CtlRun& r, int n) {
  kbe_ctx* ctx = r.ctx;
  cudaError_t e = sigma_blocks(ctx, tri(n, 0), n + 1, n, r.L, r.R, r.Sl, r.Sg, r.s);
  ++r.launches;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "kbe_run_controlled: self-energy");
  if (r.K_sel > 0 && n > 0) {
    SelectArgs sa{ctx->M, n, r.K_sel, (const double*)r.L, (const double*)r.R, (const double*)r.Sl,
                  (const double*)r.Sg, ctx->d_hist + (size_t)n * kMaxOrder * kWTab, ctx->d_band, ctx->d_wbar,
                  ctx->band_w, ctx->d_korder};
    sa.u = ctx->d_hist + (size_t)ctx->n_max * kMaxOrder * kWTab;
    int ns = 0;
    if ((e = launch_select_order(sa, r.s, &ns)) != cudaSuccess) return cuda_fail(ctx, e, "kbe_run_controlled: order");
    r.launches += ns;
  }
  int nl = 0;
  kbe_status st = history(ctx, n, r.precision, r.L, r.R, r.Sl, r.Sg, r.I, r.s, &nl, true);
  r.launches += nl;
  if (st != KBE_OK) return st;
  StepArgs a = step_args(ctx, n, r.L, r.R, r.I, r.F);
  if ((e = launch_fock(a, r.s)) != cudaSuccess || (e = launch_rhs(a, r.s)) != cudaSuccess)
    return cuda_fail(ctx, e, "kbe_run_controlled: right-hand side");
  r.launches += 2;
  ++r.nfev;
  return KBE_OK;
}

// self-energy row and Fock matrix of the accepted row n into the rings
kbe_status ctl_store(CtlRun& r, int n) {
  kbe_ctx* ctx = r.ctx;
  const size_t srow = (size_t)r.n_max * ctx->M * ctx->M * 2;  // doubles per s-row
  double* slot = r.Sring + (size_t)(n % kRing) * 2 * srow;
  cudaError_t e = sigma_blocks(ctx, tri(n, 0), n + 1, n, r.L, r.R, slot, slot + srow, r.s);
  StepArgs a = step_args(ctx, n, r.L, r.R, r.I, r.F);
  a.eps = r.eps_ring + (size_t)(n % kRing) * ctx->M * ctx->M * 2;
  if (e == cudaSuccess) e = launch_fock(a, r.s);
  r.launches += 2;
  return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "kbe_run_controlled: accepted row");
}

kbe_status ctl_read(CtlRun& r, double* host) {
  cudaError_t e = cudaMemcpyAsync(host, r.out, 2 * sizeof(double), cudaMemcpyDeviceToHost, r.s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(r.s);
  return e == cudaSuccess ? KBE_OK : cuda_fail(r.ctx, e, "kbe_run_controlled: norm read");
}

// weights of interval n for the history quadrature: band row n and the
// settled entry n - bw (fixed orders), or the local weights of every order
// for the device's order choice
kbe_status ctl_interval_weights(CtlRun& r, int n) {
  kbe_ctx* ctx = r.ctx;
  HostGrid& g = ctx->grid;
  double w[kWTab];
  cudaError_t e;
  if (r.K_sel > 0) {
    std::vector<double> hist((size_t)kMaxOrder * kWTab, 0.0);
    for (int k = 1; k <= std::min(r.K_sel, n); ++k) {
      kbe_status st = local_weights(g.t.data() + n - k, k, g.t[n - 1], g.t[n], w, &ctx->err);
      if (st != KBE_OK) return st;
      for (int j = 0; j <= k; ++j) hist[(size_t)(k - 1) * kWTab + j] = w[j];
    }
    e = cudaMemcpyAsync(ctx->d_hist + (size_t)n * kMaxOrder * kWTab, hist.data(), hist.size() * sizeof(double),
                        cudaMemcpyHostToDevice, r.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r.s);  // the host buffer is released on return
    return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "kbe_run_controlled: weights upload");
  }
  const int bw = r.bw, kap = std::min(r.k_hist, n);
  kbe_status st = local_weights(g.t.data() + n - kap, kap, g.t[n - 1], g.t[n], w, &ctx->err);
  if (st != KBE_OK) return st;
  // band row n from row n-1 (row recursion of Sec. 3.2) plus the local weights
  for (int d = 0; d < bw; ++d) {
    const int m = n - d;
    double v = 0.0;
    if (m >= 0) {
      if (d >= 1) v = g.band[(size_t)(n - 1) * bw + (d - 1)];
      if (d <= kap) v += w[kap - d];
    }
    g.band[(size_t)n * bw + d] = v;
  }
  if (n - bw >= 0) g.wbar[n - bw] = g.band[(size_t)(n - 1) * bw + (bw - 1)];
  e = cudaMemcpyAsync(ctx->d_band + (size_t)n * bw, g.band.data() + (size_t)n * bw, bw * sizeof(double),
                      cudaMemcpyHostToDevice, r.s);
  if (e == cudaSuccess && n - bw >= 0)
    e = cudaMemcpyAsync(ctx->d_wbar + (n - bw), g.wbar.data() + (n - bw), sizeof(double), cudaMemcpyHostToDevice,
                        r.s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(r.s);  // a retry rewrites these host entries
  return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "kbe_run_controlled: weights upload");
}

}  // namespace

void kbe::set_global_error(const char* msg) { g_create_err = msg; }

int kbe::sm_count() {
  constexpr int kDevs = 64;
  static std::atomic<int> cached[kDevs] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevs) {
    cudaGetLastError();
    return 1;
  }
  int v = cached[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
    cudaGetLastError();
    return 1;
  }
  cached[dev].store(v, std::memory_order_relaxed);
  return v;
}

extern "C" {

kbe_status kbe_create(int norb, int n_max, kbe_ctx** out) {
  if (!out) return fail(nullptr, KBE_EINVAL, "kbe_create: out is NULL");
  *out = nullptr;
  if (norb < 1 || norb > kMaxNorb) return fail(nullptr, KBE_EINVAL, "kbe_create: norb outside [1, 64]");
  if (n_max < 1 || n_max > (1 << 20)) return fail(nullptr, KBE_EINVAL, "kbe_create: n_max outside [1, 2^20]");
  kbe_ctx* ctx = new (std::nothrow) kbe_ctx();
  if (!ctx) return fail(nullptr, KBE_ENOMEM, "kbe_create: host allocation failed");
  ctx->M = norb;
  ctx->n_max = n_max;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e != cudaSuccess) { delete ctx; return fail(nullptr, KBE_ECUDA, std::string("kbe_create: ") + cudaGetErrorString(e)); }
  const size_t MM = (size_t)norb * norb;
  const size_t row = (size_t)n_max * MM;  // complex entries of one s-row
  // prep rows and chunk partials of the FP64 slice (history_f64_split): small
  // rows take up to kMaxSplitSmall chunks
  ctx->part_bytes = (3 + 2 * (size_t)(row <= (size_t)kRunMaxRow ? kMaxSplitSmall : kMaxSplit)) * row * 16;
  if ((e = dev_alloc(&ctx->d_part, ctx->part_bytes / sizeof(double))) != cudaSuccess ||
      (e = dev_alloc(&ctx->d_wbar, (size_t)n_max)) != cudaSuccess ||
      (e = dev_alloc(&ctx->d_band, (size_t)n_max * (kMaxOrder + 1))) != cudaSuccess ||
      (e = dev_alloc(&ctx->d_corr, (size_t)n_max * kMaxOrder * kWTab)) != cudaSuccess ||
      (e = dev_alloc(&ctx->d_pred, (size_t)n_max * kMaxOrder * kWTab)) != cudaSuccess ||
      (e = dev_alloc(&ctx->d_h0, 2 * MM)) != cudaSuccess ||
      (e = dev_alloc(&ctx->d_U, (size_t)norb)) != cudaSuccess ||
      (e = dev_alloc(&ctx->d_v, (size_t)norb)) != cudaSuccess ||
      (e = dev_alloc(&ctx->d_eps, 2 * MM)) != cudaSuccess ||
      (e = dev_alloc(&ctx->d_status, 1)) != cudaSuccess || (e = dev_alloc(&ctx->d_runbar, 1)) != cudaSuccess) {
    release(ctx);
    delete ctx;
    cudaGetLastError();
    return fail(nullptr, e == cudaErrorMemoryAllocation ? KBE_ENOMEM : KBE_ECUDA,
                std::string("kbe_create: device allocation: ") + cudaGetErrorString(e));
  }
  ctx->split_bytes = split_workspace_bytes(norb, n_max);
  if (ctx->split_bytes > 0 && (e = cudaMalloc(&ctx->d_split, ctx->split_bytes)) != cudaSuccess) {
    release(ctx);
    delete ctx;
    cudaGetLastError();
    return fail(nullptr, e == cudaErrorMemoryAllocation ? KBE_ENOMEM : KBE_ECUDA,
                std::string("kbe_create: split workspace: ") + cudaGetErrorString(e));
  }
  if ((e = cudaMemset(ctx->d_status, 0, sizeof(int))) != cudaSuccess) {
    release(ctx);
    delete ctx;
    return fail(nullptr, KBE_ECUDA, std::string("kbe_create: ") + cudaGetErrorString(e));
  }
  *out = ctx;
  return KBE_OK;
}

kbe_status kbe_destroy(kbe_ctx* ctx) {
  if (!ctx) return KBE_OK;
  cudaSetDevice(ctx->device);
  release(ctx);
  delete ctx;
  return KBE_OK;
}

const char* kbe_last_error(const kbe_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

int kbe_last_launch_count(const kbe_ctx* ctx) { return ctx ? ctx->last_launches : 0; }

kbe_status kbe_grid_weights(const double* t, const int* order, int n_t, int n, double* row) {
  if (!row) return fail(nullptr, KBE_EINVAL, "kbe_grid_weights: row is NULL");
  HostGrid g;
  std::string err;
  kbe_status st = build_grid(t, order, n_t, &g, &err);
  if (st != KBE_OK) return fail(nullptr, st, err);
  if (n < 0 || n >= n_t) return fail(nullptr, KBE_EINVAL, "kbe_grid_weights: n outside [0, n_t)");
  const int bw = g.K + 1;
  for (int m = 0; m <= n; ++m) row[m] = (n - m < bw) ? g.band[(size_t)n * bw + (n - m)] : g.wbar[m];
  return KBE_OK;
}

kbe_status kbe_local_weights(const double* tau, int k, double lo, double hi, double* w) {
  std::string err;
  kbe_status st = local_weights(tau, k, lo, hi, w, &err);
  if (st != KBE_OK) return fail(nullptr, st, "kbe_local_weights: " + err);
  return KBE_OK;
}

kbe_status kbe_set_grid(kbe_ctx* ctx, const double* t, const int* order, int n_t) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  if (n_t > ctx->n_max) return fail(ctx, KBE_EINVAL, "kbe_set_grid: n_t > n_max");
  HostGrid g;
  kbe_status st = build_grid(t, order, n_t, &g, &ctx->err);
  if (st != KBE_OK) return st;
  if ((st = use_device(ctx)) != KBE_OK) return st;
  const int bw = g.K + 1;
  // the band array is laid out with the grid's own width
  cudaError_t e;
  if ((e = cudaMemcpy(ctx->d_wbar, g.wbar.data(), n_t * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(ctx->d_band, g.band.data(), (size_t)n_t * bw * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(ctx->d_corr, g.corr.data(), g.corr.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(ctx->d_pred, g.pred.data(), g.pred.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(ctx, e, "kbe_set_grid: upload");
  ctx->grid = std::move(g);
  ctx->grid_set = true;
  ctx->band_w = ctx->grid.K + 1;
  ctx->adaptive_K = 0;
  ctx->adaptive_rows = 0;
  ctx->planes_L = ctx->planes_R = nullptr;  // cached digit planes depend on the band of the weights
  ctx->planes_rows = 0;
  return KBE_OK;
}

kbe_status kbe_set_model(kbe_ctx* ctx, const double* h0, const double* U, const double* v, const double* pulse) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  if (!h0 || !U || !v || !pulse) return fail(ctx, KBE_EINVAL, "kbe_set_model: NULL argument");
  const int M = ctx->M;
  for (int i = 0; i < 2 * M * M; ++i)
    if (!std::isfinite(h0[i])) return fail(ctx, KBE_EINVAL, "kbe_set_model: non-finite h0");
  for (int i = 0; i < M; ++i)
    if (!std::isfinite(U[i]) || !std::isfinite(v[i])) return fail(ctx, KBE_EINVAL, "kbe_set_model: non-finite U or v");
  for (int i = 0; i < 4; ++i)
    if (!std::isfinite(pulse[i])) return fail(ctx, KBE_EINVAL, "kbe_set_model: non-finite pulse");
  if (!(pulse[2] > 0.0)) return fail(ctx, KBE_EINVAL, "kbe_set_model: pulse sigma must be > 0");
  kbe_status st = use_device(ctx);
  if (st != KBE_OK) return st;
  Model& md = ctx->model;
  md.h0.assign(h0, h0 + 2 * M * M);
  md.U.assign(U, U + M);
  md.v.assign(v, v + M);
  md.E0 = pulse[0]; md.t0 = pulse[1]; md.sigma = pulse[2]; md.omega = pulse[3];
  cudaError_t e;
  if ((e = cudaMemcpy(ctx->d_h0, h0, 2 * M * M * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(ctx->d_U, U, M * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(ctx->d_v, v, M * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(ctx, e, "kbe_set_model: upload");
  md.set = true;
  return KBE_OK;
}

kbe_status kbe_set_thermal(kbe_ctx* ctx, double beta, int n_tau, int k_tau, const double* GM) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  if (!GM) {
    ctx->thermal = false;
    return KBE_OK;
  }
  if (ctx->dense) return fail(ctx, KBE_EINVAL, "kbe_set_thermal: the thermal branch needs the local interaction");
  if (!(beta > 0.0) || !std::isfinite(beta) || n_tau < 2 || n_tau > 4096 || k_tau < 1 || k_tau > kMaxOrder)
    return fail(ctx, KBE_EINVAL, "kbe_set_thermal: need beta > 0, 2 <= n_tau <= 4096, 1 <= k_tau <= 12");
  const int M = ctx->M;
  const size_t MM = (size_t)M * M, N = n_tau;
  for (size_t i = 0; i < 2 * N * MM; ++i)
    if (!std::isfinite(GM[i])) return fail(ctx, KBE_EINVAL, "kbe_set_thermal: non-finite G^M");
  std::vector<double> left;
  kbe_status st = thermal_weights(n_tau, beta, k_tau, &left, &ctx->err);
  if (st != KBE_OK) return st;
  if ((st = use_device(ctx)) != KBE_OK) return st;
  const size_t doubles = 2 * N * MM + thermal_left_doubles(N) + 4 * N * MM + 2 * (size_t)ctx->n_max * MM +
                         2 * (size_t)kRing * N * MM + 2 * (size_t)ctx->n_max * N * MM + 2 * N * MM +
                         2 * (size_t)ctx->n_max * MM;  // + the double-float copies of Smw and Aw
  cudaFree(ctx->d_th);
  ctx->d_th = nullptr;
  ctx->thermal = false;
  cudaError_t e = dev_alloc(&ctx->d_th, doubles);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->d_th = nullptr;
    return fail(ctx, e == cudaErrorMemoryAllocation ? KBE_ENOMEM : KBE_ECUDA, "kbe_set_thermal: allocation");
  }
  ctx->th_N = n_tau;
  ctx->th_k = k_tau;
  ctx->th_beta = beta;
  if ((e = cudaMemset(ctx->d_th, 0, doubles * sizeof(double))) != cudaSuccess)
    return cuda_fail(ctx, e, "kbe_set_thermal: clear");
  const ThermalLayout t = thermal_layout(ctx);
  // initial mixed row G^|(0, tau_j) = -i G^M(beta - tau_j)
  std::vector<double> row0(2 * N * MM);
  for (size_t j = 0; j < N; ++j)
    for (size_t k = 0; k < MM; ++k) {
      const double* g = GM + 2 * ((N - 1 - j) * MM + k);
      row0[2 * (j * MM + k)] = g[1];
      row0[2 * (j * MM + k) + 1] = -g[0];
    }
  if ((e = cudaMemcpy(t.GM, GM, 2 * N * MM * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(t.left, left.data(), N * N * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(t.Gx, row0.data(), row0.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(ctx, e, "kbe_set_thermal: upload");
  ctx->thermal = true;
  return KBE_OK;
}

kbe_status kbe_copy_mixed(kbe_ctx* ctx, int n_rows, void* buf, int to_context, void* stream) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  if (!ctx->thermal) return fail(ctx, KBE_ESTATE, "kbe_copy_mixed: no thermal branch (kbe_set_thermal)");
  if (n_rows < 1 || n_rows > ctx->n_max) return fail(ctx, KBE_EINVAL, "kbe_copy_mixed: n_rows outside [1, n_max]");
  if (!aligned16(buf)) return fail(ctx, KBE_EINVAL, "kbe_copy_mixed: NULL or misaligned pointer");
  kbe_status st = use_device(ctx);
  if (st != KBE_OK) return st;
  const size_t bytes = (size_t)n_rows * ctx->th_N * ctx->M * ctx->M * 16;
  double* Gx = thermal_layout(ctx).Gx;
  cudaError_t e = to_context ? cudaMemcpyAsync(Gx, buf, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream)
                             : cudaMemcpyAsync(buf, Gx, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
  return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "kbe_copy_mixed");
}

kbe_status kbe_set_interaction(kbe_ctx* ctx, const double* U4) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  if (!U4) {
    ctx->dense = false;
    return KBE_OK;
  }
  const int M = ctx->M;
  if (ctx->thermal) return fail(ctx, KBE_EINVAL, "kbe_set_interaction: the thermal branch needs the local interaction");
  if (M > kDenseMaxM) return fail(ctx, KBE_ERANGE, "kbe_set_interaction: norb above KBE_DENSE_MAX_NORB");
  const size_t M4 = (size_t)M * M * M * M;
  for (size_t k = 0; k < M4; ++k)
    if (!std::isfinite(U4[k])) return fail(ctx, KBE_EINVAL, "kbe_set_interaction: non-finite tensor entry");
  kbe_status st = use_device(ctx);
  if (st != KBE_OK) return st;
  auto at = [M](int p, int q, int r, int t) { return (((size_t)p * M + q) * M + r) * M + t; };
  std::vector<double> Ut(M4), Xt(M4), HF(M4);
  for (int i = 0; i < M; ++i)
    for (int f = 0; f < M; ++f)
      for (int d = 0; d < M; ++d)
        for (int e = 0; e < M; ++e) {
          Ut[at(d, i, e, f)] = U4[at(i, f, d, e)];
          // (j,a,b,c) := (i,f,d,e): UEx_jabc = 2 U_jbac - U_jabc, stored at [b][j][a][c]
          Xt[at(d, i, f, e)] = 2.0 * U4[at(i, d, f, e)] - U4[at(i, f, d, e)];
          // (i,j,b,a) := (i,f,d,e): HF[(i,j)][(b,a)] = U_iabj - 2 U_ijba
          HF[at(i, f, d, e)] = U4[at(i, e, d, f)] - 2.0 * U4[at(i, f, d, e)];
        }
  cudaError_t e = cudaSuccess;
  if (!ctx->d_Ut) {
    if ((e = dev_alloc(&ctx->d_Ut, M4)) != cudaSuccess || (e = dev_alloc(&ctx->d_Xt, M4)) != cudaSuccess ||
        (e = dev_alloc(&ctx->d_HF, M4)) != cudaSuccess) {
      cudaFree(ctx->d_Ut); cudaFree(ctx->d_Xt); cudaFree(ctx->d_HF);
      ctx->d_Ut = ctx->d_Xt = ctx->d_HF = nullptr;
      cudaGetLastError();
      return fail(ctx, e == cudaErrorMemoryAllocation ? KBE_ENOMEM : KBE_ECUDA, "kbe_set_interaction: allocation");
    }
  }
  if ((e = cudaMemcpy(ctx->d_Ut, Ut.data(), M4 * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(ctx->d_Xt, Xt.data(), M4 * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(ctx->d_HF, HF.data(), M4 * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = dense_sigma_prepare(M)) != cudaSuccess)
    return cuda_fail(ctx, e, "kbe_set_interaction: upload");
  ctx->dense = true;
  return KBE_OK;
}

kbe_status kbe_selfenergy_slice(kbe_ctx* ctx, int n, const void* L, const void* R, void* Sl, void* Sg,
                                void* stream) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  kbe_status st = check_row_call(ctx, n);
  if (st != KBE_OK) return st;
  if (!ctx->model.set) return fail(ctx, KBE_ESTATE, "no model: call kbe_set_model first");
  if (!aligned16(L) || !aligned16(R) || !aligned16(Sl) || !aligned16(Sg))
    return fail(ctx, KBE_EINVAL, "kbe_selfenergy_slice: NULL or misaligned pointer");
  if ((st = use_device(ctx)) != KBE_OK) return st;
  cudaError_t e = sigma_blocks(ctx, tri(n, 0), n + 1, n, L, R, Sl, Sg, (cudaStream_t)stream);
  ctx->last_launches = 1;
  return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "kbe_selfenergy_slice");
}

kbe_status kbe_selfenergy_all(kbe_ctx* ctx, int n_rows, const void* L, const void* R, void* Sl, void* Sg,
                              void* stream) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  if (n_rows < 1 || n_rows > ctx->n_max) return fail(ctx, KBE_EINVAL, "kbe_selfenergy_all: n_rows outside [1, n_max]");
  if (!ctx->model.set) return fail(ctx, KBE_ESTATE, "no model: call kbe_set_model first");
  if (!aligned16(L) || !aligned16(R) || !aligned16(Sl) || !aligned16(Sg))
    return fail(ctx, KBE_EINVAL, "kbe_selfenergy_all: NULL or misaligned pointer");
  kbe_status st = use_device(ctx);
  if (st != KBE_OK) return st;
  cudaError_t e = sigma_blocks(ctx, 0, tri(n_rows, 0), -1, L, R, Sl, Sg, (cudaStream_t)stream);
  ctx->last_launches = 1;
  return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "kbe_selfenergy_all");
}

kbe_status kbe_history_slice(kbe_ctx* ctx, int n, int precision, const void* L, const void* R, const void* Sl,
                             const void* Sg, void* I_out, void* stream) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  kbe_status st = check_row_call(ctx, n);
  if (st != KBE_OK) return st;
  if (!aligned16(L) || !aligned16(R) || !aligned16(Sl) || !aligned16(Sg) || !aligned16(I_out))
    return fail(ctx, KBE_EINVAL, "kbe_history_slice: NULL or misaligned pointer");
  if ((st = use_device(ctx)) != KBE_OK) return st;
  int nl = 0;
  st = history(ctx, n, precision, L, R, Sl, Sg, I_out, (cudaStream_t)stream, &nl);
  ctx->last_launches = nl;
  return st;
}

kbe_status kbe_history_slice_band(kbe_ctx* ctx, int n, int row_lo, int row_hi, const void* L, const void* R,
                                  const void* Sl, const void* Sg, void* I_out, void* stream) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  kbe_status st = check_row_call(ctx, n);
  if (st != KBE_OK) return st;
  if (row_lo < 0 || row_hi < row_lo) return fail(ctx, KBE_EINVAL, "kbe_history_slice_band: need 0 <= row_lo <= row_hi");
  if (!aligned16(L) || !aligned16(R) || !aligned16(Sl) || !aligned16(Sg) || !aligned16(I_out))
    return fail(ctx, KBE_EINVAL, "kbe_history_slice_band: NULL or misaligned pointer");
  if ((st = use_device(ctx)) != KBE_OK) return st;
  HistoryArgs a{ctx->M, n, (const double*)L, (const double*)R, (const double*)Sl, (const double*)Sg,
                weights_view(ctx), (double*)I_out, ctx->d_part, ctx->part_bytes, ctx->d_status};
  a.band_lo = row_lo;
  a.band_hi = row_hi;
  int nl = 0;
  cudaError_t e = launch_history_f64(a, (cudaStream_t)stream, &nl);
  ctx->last_launches = nl;
  return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "kbe_history_slice_band: launch");
}

// ------------------------------------------------------------ step phases --
// The phases of a KBE_FP64 step for callers that form the history slice
// themselves (one system split by row bands across devices: the bands'
// partial slices sum to the slice).
static kbe_status check_phase(kbe_ctx* ctx, int n, const char* who) {
  kbe_status st = check_row_call(ctx, n);
  if (st != KBE_OK) return st;
  if (n < 1) return fail(ctx, KBE_ERANGE, std::string(who) + ": n must be >= 1");
  if (!ctx->model.set) return fail(ctx, KBE_ESTATE, "no model: call kbe_set_model first");
  if (ctx->adaptive_K > 0 || ctx->thermal)
    return fail(ctx, KBE_ESTATE, std::string(who) + ": adaptive history orders and the thermal branch need kbe_step");
  return use_device(ctx);
}

kbe_status kbe_step_predict(kbe_ctx* ctx, int n, void* L, void* R, void* F_ring, void* stream) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  kbe_status st = check_phase(ctx, n, "kbe_step_predict");
  if (st != KBE_OK) return st;
  if (!aligned16(L) || !aligned16(R) || !aligned16(F_ring))
    return fail(ctx, KBE_EINVAL, "kbe_step_predict: NULL or misaligned pointer");
  StepArgs a = step_args(ctx, n, L, R, nullptr, F_ring);
  cudaError_t e = launch_predictor(a, (cudaStream_t)stream);
  ctx->last_launches = 1;
  return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "kbe_step_predict");
}

kbe_status kbe_step_sweep_band(kbe_ctx* ctx, int n, int row_lo, int row_hi, const void* L, const void* R,
                               void* S_less, void* S_great, void* I_part, void* stream) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  kbe_status st = check_phase(ctx, n, "kbe_step_sweep_band");
  if (st != KBE_OK) return st;
  if (row_lo < 0 || row_hi < row_lo) return fail(ctx, KBE_EINVAL, "kbe_step_sweep_band: need 0 <= row_lo <= row_hi");
  if (!aligned16(L) || !aligned16(R) || !aligned16(S_less) || !aligned16(S_great) || !aligned16(I_part))
    return fail(ctx, KBE_EINVAL, "kbe_step_sweep_band: NULL or misaligned pointer");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = sigma_blocks(ctx, tri(n, 0), n + 1, n, L, R, S_less, S_great, s);
  if (e != cudaSuccess) { ctx->last_launches = 1; return cuda_fail(ctx, e, "kbe_step_sweep_band: self-energy"); }
  HistoryArgs a{ctx->M, n, (const double*)L, (const double*)R, (const double*)S_less, (const double*)S_great,
                weights_view(ctx), (double*)I_part, ctx->d_part, ctx->part_bytes, ctx->d_status};
  a.band_lo = row_lo;
  a.band_hi = row_hi;
  if (!next_events(ctx, &a.ev_begin, &a.ev_end)) return fail(ctx, KBE_ECUDA, "profiling: cudaEventCreate");
  int nl = 0;
  e = launch_history_f64(a, s, &nl);
  ctx->last_launches = 1 + nl;
  return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "kbe_step_sweep_band: history slice");
}

kbe_status kbe_step_sweep_finish(kbe_ctx* ctx, int n, void* L, void* R, const void* I, void* F_ring, void* stream) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  kbe_status st = check_phase(ctx, n, "kbe_step_sweep_finish");
  if (st != KBE_OK) return st;
  if (!aligned16(L) || !aligned16(R) || !aligned16(I) || !aligned16(F_ring))
    return fail(ctx, KBE_EINVAL, "kbe_step_sweep_finish: NULL or misaligned pointer");
  cudaStream_t s = (cudaStream_t)stream;
  StepArgs a = step_args(ctx, n, L, R, I, F_ring);
  cudaError_t e = launch_fock(a, s);
  if (e == cudaSuccess) e = launch_rhs_corrector(a, s);
  ctx->last_launches = 3;
  return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "kbe_step_sweep_finish");
}

kbe_status kbe_set_split_planes(kbe_ctx* ctx, int keep) {
  if (!ctx) return KBE_EINVAL;
  if (keep != 0 && keep != 1) return fail(ctx, KBE_EINVAL, "kbe_set_split_planes: keep must be 0 or 1");
  ctx->split_planes = keep != 0;
  if (!keep && ctx->d_planes) {
    if (use_device(ctx) == KBE_OK) {
      cudaDeviceSynchronize();  // no launch may still read the buffer
      cudaFree(ctx->d_planes);
    }
    ctx->d_planes = nullptr;
  }
  ctx->planes_L = ctx->planes_R = nullptr;
  ctx->planes_rows = 0;
  ctx->planes_failed = false;
  return KBE_OK;
}

kbe_status kbe_debug_withhold_run(kbe_ctx* ctx, int barrier, long long spin_limit) {
  if (!ctx) return KBE_EINVAL;
  if (barrier < 0 || spin_limit < 1) return fail(ctx, KBE_EINVAL, "kbe_debug_withhold_run: barrier < 0 or spin_limit < 1");
  ctx->dbg_run_withhold = barrier;
  ctx->dbg_run_spin = spin_limit;
  return KBE_OK;
}

kbe_status kbe_debug_withhold_split(kbe_ctx* ctx, long long unit, long long spin_limit) {
  if (!ctx) return KBE_EINVAL;
  if (unit < 0 || spin_limit < 1) return fail(ctx, KBE_EINVAL, "kbe_debug_withhold_split: unit < 0 or spin_limit < 1");
  ctx->dbg_withhold = unit;
  ctx->dbg_spin = spin_limit;
  return KBE_OK;
}

kbe_status kbe_init_uncorrelated(kbe_ctx* ctx, const double* rho0, void* L, void* R, void* stream) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  if (!rho0) return fail(ctx, KBE_EINVAL, "kbe_init_uncorrelated: NULL rho0");
  if (!aligned16(L) || !aligned16(R)) return fail(ctx, KBE_EINVAL, "kbe_init_uncorrelated: NULL or misaligned pointer");
  const int MM = ctx->M * ctx->M;
  for (int i = 0; i < 2 * MM; ++i)
    if (!std::isfinite(rho0[i])) return fail(ctx, KBE_EINVAL, "kbe_init_uncorrelated: non-finite rho0");
  kbe_status st = use_device(ctx);
  if (st != KBE_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // rho0 is staged in the Fock-matrix buffer, which the next right-hand side overwrites
  cudaError_t e = cudaMemcpyAsync(ctx->d_eps, rho0, (size_t)MM * 16, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_init_row0(ctx->M, ctx->d_eps, (double*)L, (double*)R, s);
  ctx->last_launches = 1;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "kbe_init_uncorrelated");
  return KBE_OK;
}

kbe_status kbe_rhs_row(kbe_ctx* ctx, int j, int precision, const void* L, const void* R, void* Sl, void* Sg,
                       void* I_work, void* F_ring, void* stream) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  kbe_status st = check_row_call(ctx, j);
  if (st != KBE_OK) return st;
  if (!ctx->model.set) return fail(ctx, KBE_ESTATE, "no model: call kbe_set_model first");
  if (!aligned16(L) || !aligned16(R) || !aligned16(Sl) || !aligned16(Sg) || !aligned16(I_work) || !aligned16(F_ring))
    return fail(ctx, KBE_EINVAL, "kbe_rhs_row: NULL or misaligned pointer");
  if ((st = use_device(ctx)) != KBE_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  int count = 0, nl = 0;
  cudaError_t e = sigma_blocks(ctx, tri(j, 0), j + 1, j, L, R, Sl, Sg, s);
  ++count;
  if (e != cudaSuccess) { ctx->last_launches = count; return cuda_fail(ctx, e, "kbe_rhs_row: self-energy"); }
  st = history(ctx, j, precision, L, R, Sl, Sg, I_work, s, &nl);
  count += nl;
  if (st != KBE_OK) { ctx->last_launches = count; return st; }
  StepArgs a = step_args(ctx, j, (void*)L, (void*)R, I_work, F_ring);
  if (ctx->thermal) {  // Sigma^| and the mixed term, the row's F, then the mixed right-hand side
    ThermalArgs x = thermal_args(ctx, a, Sl, Sg, I_work);
    x.df = precision != KBE_FP64;
    if ((e = thermal_sweep_a(ctx, x, s)) != cudaSuccess || (e = launch_fock(a, s)) != cudaSuccess ||
        (e = launch_rhs(a, s)) != cudaSuccess || (e = launch_th_rhs(x, s)) != cudaSuccess) {
      ctx->last_launches = count + 5;
      return cuda_fail(ctx, e, "kbe_rhs_row: thermal right-hand side");
    }
    ctx->last_launches = count + 5;
    return KBE_OK;
  }
  if ((e = launch_fock(a, s)) != cudaSuccess || (e = launch_rhs(a, s)) != cudaSuccess) {
    ctx->last_launches = count + 2;
    return cuda_fail(ctx, e, "kbe_rhs_row: right-hand side");
  }
  ctx->last_launches = count + 2;
  return KBE_OK;
}

kbe_status kbe_step(kbe_ctx* ctx, int n, int P, int precision, void* L, void* R, void* Sl, void* Sg, void* I_work,
                    void* F_ring, void* stream) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  kbe_status st = check_step_call(ctx, n, P, precision, L, R, Sl, Sg, I_work, F_ring);
  if (st != KBE_OK) return st;
  int count = 0;
  st = step_impl(ctx, n, P, precision, L, R, Sl, Sg, I_work, F_ring, 0, kRing, (cudaStream_t)stream, nullptr, &count);
  ctx->last_launches = count;
  return st;
}

// The steps of rows n_first..n_last, one after another on the stream.
// (Capturing them into one CUDA graph was measured on the 63-step dimer run:
// 5.77 ms against 5.61 ms launched one by one; its steps are bound on the
// device, at about 6 microseconds per small kernel, not by the launches.)
kbe_status kbe_run_steps(kbe_ctx* ctx, int n_first, int n_last, int P, int precision, void* L, void* R, void* Sl,
                         void* Sg, void* I_work, void* F_ring, void* stream) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  if (n_first < 1 || n_last < n_first) return fail(ctx, KBE_EINVAL, "kbe_run_steps: need 1 <= n_first <= n_last");
  kbe_status st = check_row_call(ctx, n_last);  // the whole range on the grid
  if (st != KBE_OK) return st;
  // the rest as kbe_step of the first row (with adaptive orders: the rows in order from the next one)
  st = check_step_call(ctx, n_first, P, precision, L, R, Sl, Sg, I_work, F_ring);
  if (st != KBE_OK) return st;
  if (ctx->adaptive_K > 0) ctx->adaptive_rows = n_last + 1;  // the rows above n_first are stepped here
  int total = 0;
  // Plain FP64 steps with the local interaction and fixed orders: runs of
  // small rows go to the cooperative kernel, up to kRunMaxSteps rows per launch.
  const bool coop = precision == KBE_FP64 && !ctx->dense && ctx->adaptive_K == 0 && !ctx->thermal &&
                    !ctx->profiling && !ctx->run_coop_refused;
  const int64_t MM = (int64_t)ctx->M * ctx->M;
  int n = n_first;
  while (n <= n_last && st == KBE_OK) {
    if (coop && (int64_t)(n + 1) * MM <= kRunMaxRow) {
      RunSmallHost h{};
      h.base = step_args(ctx, n, L, R, I_work, F_ring);
      h.Sl = (double*)Sl;
      h.Sg = (double*)Sg;
      h.I = (double*)I_work;
      h.w = weights_view(ctx);
      h.part = ctx->d_part;
      h.corr0 = ctx->d_corr;
      h.pred0 = ctx->d_pred;
      h.bar = ctx->d_runbar;
      h.spin = ctx->dbg_run_spin > 0 ? ctx->dbg_run_spin : 1ll << 24;  // polls: about a second or more
      h.withhold = ctx->dbg_run_withhold;
      ctx->dbg_run_spin = 0;  // one launch only
      ctx->dbg_run_withhold = -1;
      h.P = P;
      while (h.nsteps < kRunMaxSteps && n <= n_last && (int64_t)(n + 1) * MM <= kRunMaxRow) {
        const int i = h.nsteps;
        if (!history_f64_split(ctx->M, n, ctx->part_bytes, 0x7fffffff, &h.nchunk[i], &h.chunk_len[i]))
          return fail(ctx, KBE_ENOMEM, "kbe_run_steps: history workspace too small");
        h.n[i] = n;
        h.kn[i] = ctx->grid.order[n];
        h.field[i] = ctx->model.field(ctx->grid.t[n]);
        ++h.nsteps;
        ++n;
      }
      int count = 0;
      const cudaError_t e = launch_run_small(h, (cudaStream_t)stream, &count);
      total += count;
      if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported) {
        // fewer SMs available than the device has (e.g. a partitioned GPU): these rows and all later ones
        // take the per-kernel step (the launch error is not sticky)
        cudaGetLastError();
        ctx->run_coop_refused = true;
        for (int i = 0; i < h.nsteps && st == KBE_OK; ++i) {
          int c = 0;
          st = step_impl(ctx, h.n[i], P, precision, L, R, Sl, Sg, I_work, F_ring, 0, kRing, (cudaStream_t)stream,
                         nullptr, &c);
          total += c;
        }
      } else if (e != cudaSuccess) {
        st = cuda_fail(ctx, e, "kbe_run_steps: cooperative run launch");
      }
      continue;
    }
    int count = 0;
    st = step_impl(ctx, n, P, precision, L, R, Sl, Sg, I_work, F_ring, 0, kRing, (cudaStream_t)stream, nullptr,
                   &count);
    total += count;
    ++n;
  }
  ctx->last_launches = total;
  return st;
}

kbe_status kbe_step_host(kbe_ctx* ctx, int n, int P, int precision, const void* L_host, const void* R_host,
                         const void* F_host, void* L, void* R, void* Sl, void* Sg, void* I_work, void* F_ring,
                         void* L_row_host, void* R_row_host, void* stream) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  kbe_status st = check_step_call(ctx, n, P, precision, L, R, Sl, Sg, I_work, F_ring);
  if (st != KBE_OK) return st;
  if (!L_host || !R_host || !F_host || !L_row_host || !R_row_host)
    return fail(ctx, KBE_EINVAL, "kbe_step_host: NULL host pointer");
  cudaError_t e = cudaSuccess;
  if (!ctx->up_stream) {
    e = cudaStreamCreateWithFlags(&ctx->up_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->up_start, cudaEventDisableTiming);
    for (cudaEvent_t& ev : ctx->up_ev)
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kbe_step_host: copy stream");
  }
  // one copy stream: two concurrent host-to-device copies (L and R) were
  // measured slower (e2e step 26.0 ms instead of 23.9 ms)
  const cudaStream_t s = (cudaStream_t)stream, cs = ctx->up_stream;
  const size_t blk = (size_t)ctx->M * ctx->M * 16;  // bytes of one block
  // rows n-1 down to 0 in chunks (row r holds r + 1 blocks); the columns of
  // each chunk are contracted while the next ones are copied.  Every column
  // reads a block of each row above it, so the longest rows come first and
  // the step waits for the first chunk alone.  The chunks' bytes grow
  // geometrically (shares 1 : q : q^2 ...), so that the first is small and
  // each later one arrives while the columns before it are contracted.
  // Measured on the e2e step of chain_m8_n1024 (row 1023, M = 8): 5 chunks
  // with q = 1.8 22.7 ms; 4 or 6 chunks with q = 1.5-2.0 22.8-23.1 ms; 4
  // equal chunks 23.6 ms; the upload before the step 27.0 ms.  Each column
  // range is one more launch of the contraction.
  Staged sg;
  sg.k = std::min(5, n);
  const double q = 1.8;
  double share_sum = 0.0, share = 1.0;
  for (int k = 0; k < sg.k; ++k, share *= q) share_sum += share;
  double share_acc = 0.0;
  share = 1.0;
  int hi = n;
  for (int k = 0; k < sg.k; ++k, share *= q) {
    share_acc += share;
    const double target = (double)tri(n, 0) * std::max(0.0, 1.0 - share_acc / share_sum);  // blocks below the chunk
    int lo = k + 1 == sg.k ? 0 : (int)std::floor((std::sqrt(8.0 * target + 1.0) - 1.0) / 2.0);
    lo = std::max(0, std::min(lo, hi - 1));
    sg.c_lo[k] = lo;
    sg.c_hi[k] = k == 0 ? n + 1 : hi;
    hi = lo;
  }
  sg.c_lo[sg.k - 1] = 0;
  // the copies start after the work already queued on the stream (the
  // buffers may still be in use) and never overwrite row n
  if ((e = cudaEventRecord(ctx->up_start, s)) != cudaSuccess || (e = cudaStreamWaitEvent(cs, ctx->up_start, 0)))
    return cuda_fail(ctx, e, "kbe_step_host: copy stream");
  const size_t ring_bytes = (size_t)kRing * 2 * ctx->n_max * blk;
  e = cudaMemcpyAsync(F_ring, F_host, ring_bytes, cudaMemcpyHostToDevice, cs);
  for (int k = 0; k < sg.k && e == cudaSuccess; ++k) {
    const int r_lo = sg.c_lo[k], r_hi = k == 0 ? n : sg.c_hi[k];
    const size_t off = (size_t)tri(r_lo, 0) * blk, bytes = (size_t)(tri(r_hi, 0) - tri(r_lo, 0)) * blk;
    if (bytes > 0) {
      e = cudaMemcpyAsync((char*)L + off, (const char*)L_host + off, bytes, cudaMemcpyHostToDevice, cs);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync((char*)R + off, (const char*)R_host + off, bytes, cudaMemcpyHostToDevice, cs);
    }
    if (e == cudaSuccess) e = cudaEventRecord(sg.ev[k] = ctx->up_ev[k], cs);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "kbe_step_host: upload");
  // rows 0..n-1 were rewritten: digit planes cached from earlier steps are stale
  ctx->planes_L = ctx->planes_R = nullptr;
  ctx->planes_rows = 0;
  int count = 0;
  st = step_impl(ctx, n, P, precision, L, R, Sl, Sg, I_work, F_ring, 0, kRing, s, nullptr, &count, &sg);
  ctx->last_launches = count;
  if (st != KBE_OK) return st;
  const size_t row_bytes = (size_t)(n + 1) * blk;
  e = cudaMemcpyAsync(L_row_host, (const char*)L + (size_t)tri(n, 0) * blk, row_bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(R_row_host, (const char*)R + (size_t)tri(n, 0) * blk, row_bytes, cudaMemcpyDeviceToHost, s);
  return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "kbe_step_host: row download");
}

kbe_status kbe_step_rows(kbe_ctx* ctx, int n, int P, int precision, void* L, void* R, void* Sl, void* Sg,
                         void* I_work, void* F_rows, int j0, int n_rows, void* stream) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  if (ctx->thermal) return fail(ctx, KBE_ESTATE, "kbe_step_rows: the thermal branch steps with kbe_step");
  kbe_status st = check_step_call(ctx, n, P, precision, L, R, Sl, Sg, I_work, F_rows);
  if (st != KBE_OK) return st;
  if ((st = check_row_store(ctx, n, j0, n_rows)) != KBE_OK) return st;
  int count = 0;
  st = step_impl(ctx, n, P, precision, L, R, Sl, Sg, I_work, F_rows, j0, n_rows, (cudaStream_t)stream, nullptr,
                 &count);
  ctx->last_launches = count;
  return st;
}

kbe_status kbe_adjoint_slice(kbe_ctx* ctx, int n, const void* L, const void* R, const void* S_less,
                             const void* S_great, const void* dI, void* dS_less, void* dS_great, void* dL, void* dR,
                             int row_lo, void* stream) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  kbe_status st = check_row_call(ctx, n);
  if (st != KBE_OK) return st;
  if (row_lo < 0 || row_lo > n) return fail(ctx, KBE_ERANGE, "kbe_adjoint_slice: row_lo outside [0, n]");
  if (!aligned16(L) || !aligned16(R) || !aligned16(S_less) || !aligned16(S_great) || !aligned16(dI) ||
      !aligned16(dS_less) || !aligned16(dS_great) || !aligned16(dL) || !aligned16(dR))
    return fail(ctx, KBE_EINVAL, "kbe_adjoint_slice: NULL or misaligned pointer");
  if ((st = use_device(ctx)) != KBE_OK) return st;
  const int64_t MM = (int64_t)ctx->M * ctx->M;
  const int64_t row_n = (tri(n, 0) - tri(row_lo, 0)) * MM * 2;
  AdjHistArgs h{ctx->M, n, row_lo, (const double*)L, (const double*)R, (const double*)S_less,
                (const double*)S_great, (const double*)dI, weights_view(ctx), (double*)dS_less, (double*)dS_great,
                (double*)dL, (double*)dR, (double*)dL + row_n, (double*)dR + row_n, ctx->d_part, ctx->part_bytes};
  int nl = 0;
  cudaError_t e = launch_adjoint_history(h, (cudaStream_t)stream, &nl);
  ctx->last_launches = nl;
  return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "kbe_adjoint_slice");
}

kbe_status kbe_adjoint_selfenergy_slice(kbe_ctx* ctx, int n, const void* L, const void* R, const void* dS_less,
                                        const void* dS_great, void* dL_row, void* dR_row, double* dU, void* stream) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  kbe_status st = check_row_call(ctx, n);
  if (st != KBE_OK) return st;
  if (!ctx->model.set) return fail(ctx, KBE_ESTATE, "no model: call kbe_set_model first");
  if (ctx->dense || ctx->thermal)
    return fail(ctx, KBE_ESTATE, "kbe_adjoint_selfenergy_slice: needs the local interaction and no thermal branch");
  if (!aligned16(L) || !aligned16(R) || !aligned16(dS_less) || !aligned16(dS_great) || !aligned16(dL_row) ||
      !aligned16(dR_row) || !dU || (reinterpret_cast<uintptr_t>(dU) & 7u))
    return fail(ctx, KBE_EINVAL, "kbe_adjoint_selfenergy_slice: NULL or misaligned pointer");
  if ((st = use_device(ctx)) != KBE_OK) return st;
  const int64_t MM = (int64_t)ctx->M * ctx->M;
  AdjSigmaArgs a{ctx->M, n, (const double*)L + tri(n, 0) * MM * 2, (const double*)R + tri(n, 0) * MM * 2, ctx->d_U,
                 (const double*)dS_less, (const double*)dS_great, (double*)dL_row, (double*)dR_row, ctx->d_part,
                 dU};
  int nl = 0;
  cudaError_t e = launch_adjoint_sigma(a, (cudaStream_t)stream, &nl);
  ctx->last_launches = nl;
  return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "kbe_adjoint_selfenergy_slice");
}

kbe_status kbe_step_adjoint(kbe_ctx* ctx, int n, int P, int precision, void* L, void* R, void* F_rows, int j0,
                            int n_rows, void* dL, void* dR, int row_lo, void* dF_rows, double* dU, double* dE0,
                            void* stream) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  if (precision != KBE_FP64 && precision != KBE_DF64)
    return fail(ctx, KBE_EINVAL, "kbe_step_adjoint: precision must be KBE_FP64 or KBE_DF64");
  if (!aligned16(dL) || !aligned16(dR) || !aligned16(dF_rows) || !dU || !dE0 ||
      (reinterpret_cast<uintptr_t>(dU) & 7u) || (reinterpret_cast<uintptr_t>(dE0) & 7u))
    return fail(ctx, KBE_EINVAL, "kbe_step_adjoint: NULL or misaligned pointer");
  if (!ctx->grid_set) return fail(ctx, KBE_ESTATE, "no grid: call kbe_set_grid first");
  if (ctx->dense || ctx->thermal)
    return fail(ctx, KBE_ESTATE, "kbe_step_adjoint: needs the local interaction and no thermal branch");
  if (n < 1 || n >= ctx->grid.n_t) return fail(ctx, KBE_ERANGE, "kbe_step_adjoint: n outside [1, n_t)");
  if (row_lo < 0 || row_lo > n) return fail(ctx, KBE_ERANGE, "kbe_step_adjoint: row_lo outside [0, n]");
  if (P < 1 || P > 16) return fail(ctx, KBE_EINVAL, "kbe_step_adjoint: P outside [1, 16]");
  if (!ctx->model.set) return fail(ctx, KBE_ESTATE, "no model: call kbe_set_model first");
  kbe_status st = adjoint_workspace(ctx, P);
  if (st != KBE_OK) return st;
  const int64_t MM = (int64_t)ctx->M * ctx->M;
  const size_t rowd = (size_t)ctx->n_max * MM * 2;  // doubles of one workspace row
  double* w = ctx->d_adj;
  double* Sl = w;            double* Sg = w + rowd;
  double* Iw = w + 2 * rowd;  // [2][n+1][M][M]
  double* dSl = w + 4 * rowd; double* dSg = w + 5 * rowd;
  double* gL = w + 6 * rowd;  double* gR = w + 7 * rowd;
  double* Ib = w + 8 * rowd;  // [2][n+1][M][M]
  double* Fs = w + 10 * rowd; // [2][n_max][M][M]
  double* epsb = w + 12 * rowd;
  double* save = w + kAdjFixedRows * rowd;
  st = check_step_call(ctx, n, P, precision, L, R, Sl, Sg, Iw, F_rows);
  if (st != KBE_OK) return st;
  if ((st = check_row_store(ctx, n, j0, n_rows)) != KBE_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  int count = 0, nl = 0;
  // forward again from the stored rows, keeping the iterates of row n (the
  // same kernels as the forward step, so the same iterates)
  st = step_impl(ctx, n, P, precision, L, R, Sl, Sg, Iw, F_rows, j0, n_rows, s, save, &count);
  if (st != KBE_OK) { ctx->last_launches = count; return st; }
  const size_t row_bytes = (size_t)(n + 1) * MM * 16;
  const int64_t base = tri(row_lo, 0);
  double* Lrow = (double*)L + tri(n, 0) * MM * 2;
  double* Rrow = (double*)R + tri(n, 0) * MM * 2;
  const double* dLn = (const double*)dL + (tri(n, 0) - base) * MM * 2;
  const double* dRn = (const double*)dR + (tri(n, 0) - base) * MM * 2;
  const int64_t fs = (int64_t)rowd;          // doubles between s = < and s = > in an F row
  const int64_t fstride = 2 * fs;
  double* Fn = (double*)dF_rows + (int64_t)(n - j0) * fstride;
  const HostGrid& g = ctx->grid;
  StepArgs a = step_args(ctx, n, L, R, Iw, F_rows);
  a.f_base = j0;
  a.f_rows = n_rows;
  const double shape = ctx->model.shape(g.t[n]);
  cudaError_t e = cudaSuccess;
  auto check = [&](const char* where) -> kbe_status {
    if (e != cudaSuccess) { ctx->last_launches = count; return cuda_fail(ctx, e, where); }
    return KBE_OK;
  };
  // cotangent of the final row n
  e = cudaMemcpyAsync(gL, dLn, row_bytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(gR, dRn, row_bytes, cudaMemcpyDeviceToDevice, s);
  if ((st = check("kbe_step_adjoint: copy")) != KBE_OK) return st;
  AdjLinArgs lin{ctx->M, n, a.kn, 1, a.corr, gL, gR, (double*)dL, (double*)dR, base, n - 1 >= row_lo ? 1 : 0,
                 (double*)dF_rows, j0, fstride, fs, nullptr};
  for (int p = P - 1; p >= 0; --p) {
    // row n := iterate p, then its self-energy row and Fock matrix
    const double* it = save + (size_t)p * 2 * (row_bytes / 8);
    e = cudaMemcpyAsync(Lrow, it, row_bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Rrow, it + row_bytes / 8, row_bytes, cudaMemcpyDeviceToDevice, s);
    if ((st = check("kbe_step_adjoint: restore")) != KBE_OK) return st;
    e = launch_sigma(ctx->M, tri(n, 0), n + 1, n, (const double*)L, (const double*)R, ctx->d_U, Sl, Sg,
                     ctx->d_status, s);
    ++count;
    if (e == cudaSuccess) e = launch_fock(a, s);
    ++count;
    if ((st = check("kbe_step_adjoint: self-energy")) != KBE_OK) return st;
    // corrector: cotangent of iterate p+1 -> row n-1, stored F rows, F row n of round p
    double* Fcur = Fn;
    if (p != P - 1) {
      Fcur = Fs;
      e = cudaMemsetAsync(Fs, 0, (size_t)fstride * sizeof(double), s);
      if ((st = check("kbe_step_adjoint: clear")) != KBE_OK) return st;
    }
    lin.corrector = 1;
    lin.wtab = a.corr;
    lin.Fb_cur = Fcur;
    e = launch_adjoint_lin(lin, s, &nl);
    count += nl;
    if (e == cudaSuccess) e = cudaMemsetAsync(gL, 0, row_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(gR, 0, row_bytes, s);
    if ((st = check("kbe_step_adjoint: corrector")) != KBE_OK) return st;
    // right-hand side -> slice cotangent, row n, U, E0
    AdjRhsArgs r{ctx->M, n, ctx->d_eps, Fcur, fs, Lrow, Rrow, ctx->d_U, ctx->d_v, shape, Ib, gL, gR, epsb, dU, dE0};
    e = launch_adjoint_rhs(r, s, &nl);
    count += nl;
    if ((st = check("kbe_step_adjoint: right-hand side")) != KBE_OK) return st;
    // history slice -> Sigma row, rows row_lo..n-1, row n
    AdjHistArgs h{ctx->M, n, row_lo, (const double*)L, (const double*)R, Sl, Sg, Ib, weights_view(ctx), dSl, dSg,
                  (double*)dL, (double*)dR, gL, gR, ctx->d_part, ctx->part_bytes};
    h.df = precision == KBE_DF64;  // the step's own arithmetic for its longest reverse sum
    e = launch_adjoint_history(h, s, &nl);
    count += nl;
    if ((st = check("kbe_step_adjoint: history slice")) != KBE_OK) return st;
    // self-energy -> row n, U
    AdjSigmaArgs sg{ctx->M, n, Lrow, Rrow, ctx->d_U, dSl, dSg, gL, gR, ctx->d_part, dU};
    e = launch_adjoint_sigma(sg, s, &nl);
    count += nl;
    if ((st = check("kbe_step_adjoint: self-energy")) != KBE_OK) return st;
  }
  // predictor: cotangent of iterate 0 -> row n-1 and stored F rows
  lin.corrector = 0;
  lin.wtab = a.pred;
  lin.Fb_cur = nullptr;
  e = launch_adjoint_lin(lin, s, &nl);
  count += nl;
  if ((st = check("kbe_step_adjoint: predictor")) != KBE_OK) return st;
  // leave row n as the forward step left it
  const double* fin = save + (size_t)P * 2 * (row_bytes / 8);
  e = cudaMemcpyAsync(Lrow, fin, row_bytes, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(Rrow, fin + row_bytes / 8, row_bytes, cudaMemcpyDeviceToDevice, s);
  if ((st = check("kbe_step_adjoint: restore")) != KBE_OK) return st;
  ctx->last_launches = count;
  return KBE_OK;
}

kbe_status kbe_set_adaptive_orders(kbe_ctx* ctx, int K) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  if (!ctx->grid_set) return fail(ctx, KBE_ESTATE, "no grid: call kbe_set_grid first");
  if (K < 0 || K > kMaxOrder) return fail(ctx, KBE_ERANGE, "kbe_set_adaptive_orders: K outside [0, 12]");
  kbe_status st = use_device(ctx);
  if (st != KBE_OK) return st;
  const HostGrid& g = ctx->grid;
  cudaError_t e = cudaSuccess;
  ctx->planes_L = ctx->planes_R = nullptr;  // the band width changes
  ctx->planes_rows = 0;
  if (K == 0) {  // back to the grid's orders
    const int bw = g.K + 1;
    if ((e = cudaMemcpy(ctx->d_wbar, g.wbar.data(), g.n_t * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(ctx->d_band, g.band.data(), (size_t)g.n_t * bw * sizeof(double), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
      return cuda_fail(ctx, e, "kbe_set_adaptive_orders: upload");
    ctx->adaptive_K = 0;
    ctx->band_w = bw;
    return KBE_OK;
  }
  const size_t tab = (size_t)ctx->n_max * kMaxOrder * kWTab;
  if (!ctx->d_hist && (e = cudaMalloc(&ctx->d_hist, hist_doubles(ctx->n_max, ctx->M) * sizeof(double))) != cudaSuccess)
    return cuda_fail(ctx, e, "kbe_set_adaptive_orders: allocation");
  if (!ctx->d_korder && (e = cudaMalloc(&ctx->d_korder, ctx->n_max * sizeof(int))) != cudaSuccess)
    return cuda_fail(ctx, e, "kbe_set_adaptive_orders: allocation");
  // local weights of every order k <= min(K, n) for each interval n (host FP64, Eq. weights)
  std::vector<double> hist(tab, 0.0);
  double w[kWTab];
  for (int n = 1; n < g.n_t; ++n)
    for (int k = 1; k <= (K < n ? K : n); ++k) {
      st = local_weights(g.t.data() + n - k, k, g.t[n - 1], g.t[n], w, &ctx->err);
      if (st != KBE_OK) return st;
      for (int j = 0; j <= k; ++j) hist[((size_t)n * kMaxOrder + (k - 1)) * kWTab + j] = w[j];
    }
  const int bw = K + 1;
  if ((e = cudaMemcpy(ctx->d_hist, hist.data(), tab * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemset(ctx->d_band, 0, (size_t)ctx->n_max * bw * sizeof(double))) != cudaSuccess ||
      (e = cudaMemset(ctx->d_wbar, 0, ctx->n_max * sizeof(double))) != cudaSuccess ||
      (e = cudaMemset(ctx->d_korder, 0, ctx->n_max * sizeof(int))) != cudaSuccess)
    return cuda_fail(ctx, e, "kbe_set_adaptive_orders: upload");
  ctx->adaptive_K = K;
  ctx->band_w = bw;
  ctx->adaptive_rows = 1;  // row 0 has no interval
  return KBE_OK;
}

kbe_status kbe_get_history_orders(kbe_ctx* ctx, int* orders, int n) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  if (!orders || n < 0 || n > ctx->n_max) return fail(ctx, KBE_EINVAL, "kbe_get_history_orders: bad arguments");
  if (ctx->adaptive_K == 0) {
    for (int l = 0; l < n; ++l) orders[l] = l == 0 ? 0 : (ctx->grid.order[l] < l ? ctx->grid.order[l] : l);
    return KBE_OK;
  }
  kbe_status st = use_device(ctx);
  if (st != KBE_OK) return st;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(orders, ctx->d_korder, n * sizeof(int), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "kbe_get_history_orders");
}

kbe_status kbe_reset_cache(kbe_ctx* ctx) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  ctx->planes_L = ctx->planes_R = nullptr;
  ctx->planes_rows = 0;
  return KBE_OK;
}

kbe_status kbe_set_profiling(kbe_ctx* ctx, int enable) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  ctx->profiling = enable != 0;
  ctx->ev_used = 0;
  return KBE_OK;
}

kbe_status kbe_read_profiling(kbe_ctx* ctx, int* count, double* total_ms) {
  if (!ctx || !count || !total_ms) return KBE_EINVAL;
  ctx->last_launches = 0;
  kbe_status st = use_device(ctx);
  if (st != KBE_OK) return st;
  double tot = 0.0;
  for (size_t i = 0; i < ctx->ev_used; ++i) {
    cudaError_t e = cudaEventSynchronize(ctx->ev_pool[2 * i + 1]);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ctx->ev_pool[2 * i], ctx->ev_pool[2 * i + 1]);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kbe_read_profiling");
    tot += ms;
  }
  *count = (int)ctx->ev_used;
  *total_ms = tot;
  return KBE_OK;
}

kbe_status kbe_run_controlled(kbe_ctx* ctx, const double* opts, const int* iopts, void* L, void* R, void* Sl,
                              void* Sg, void* I_work, void* F_ring, double* t_out, int* q_out, int* korder_out,
                              int* n_rows, int* stats, void* stream) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  if (!opts || !iopts || !t_out || !q_out || !korder_out || !n_rows || !stats)
    return fail(ctx, KBE_EINVAL, "kbe_run_controlled: NULL host argument");
  if (!aligned16(L) || !aligned16(R) || !aligned16(Sl) || !aligned16(Sg) || !aligned16(I_work) || !aligned16(F_ring))
    return fail(ctx, KBE_EINVAL, "kbe_run_controlled: NULL or misaligned device pointer");
  if (!ctx->model.set) return fail(ctx, KBE_ESTATE, "no model: call kbe_set_model first");
  if (ctx->thermal) return fail(ctx, KBE_ESTATE, "kbe_run_controlled: runs without the thermal branch");
  const double rtol = opts[0], atol = opts[1], h0 = opts[2], h_max = opts[3], t_end = opts[4];
  const int q_max = iopts[0], k_hist = iopts[1], K_sel = iopts[2], precision = iopts[3];
  for (int i = 0; i < 5; ++i)
    if (!std::isfinite(opts[i])) return fail(ctx, KBE_EINVAL, "kbe_run_controlled: non-finite option");
  if (!(rtol >= 0.0) || !(atol > 0.0) || !(h0 > 0.0) || !(h_max >= 0.0) || !(t_end > 0.0))
    return fail(ctx, KBE_EINVAL, "kbe_run_controlled: need rtol >= 0, atol > 0, h0 > 0, h_max >= 0, t_end > 0");
  if (q_max < 1 || q_max > kMaxOrder || k_hist < 1 || k_hist > kMaxOrder || K_sel < 0 || K_sel > kMaxOrder)
    return fail(ctx, KBE_EINVAL, "kbe_run_controlled: q_max, k_hist in [1, 12], K_sel in [0, 12]");
  if (precision != KBE_FP64 && precision != KBE_SPLIT_BF16 && precision != KBE_DF64)
    return fail(ctx, KBE_EINVAL, "kbe_run_controlled: unknown precision");
  if (ctx->n_max < 2) return fail(ctx, KBE_EINVAL, "kbe_run_controlled: n_max < 2");
  kbe_status st = use_device(ctx);
  if (st != KBE_OK) return st;
  if ((st = ctl_workspace(ctx)) != KBE_OK) return st;
  const int M = ctx->M, MM = M * M, n_max = ctx->n_max;
  cudaError_t e = cudaSuccess;
  if (K_sel > 0) {
    if (!ctx->d_hist && (e = cudaMalloc(&ctx->d_hist, hist_doubles(ctx->n_max, ctx->M) * sizeof(double))) != cudaSuccess)
      return cuda_fail(ctx, e, "kbe_run_controlled: allocation");
    if (!ctx->d_korder && (e = cudaMalloc(&ctx->d_korder, n_max * sizeof(int))) != cudaSuccess)
      return cuda_fail(ctx, e, "kbe_run_controlled: allocation");
  }
  CtlRun r;
  r.ctx = ctx;
  r.s = (cudaStream_t)stream;
  r.M = M; r.n_max = n_max; r.precision = precision; r.K_sel = K_sel; r.k_hist = k_hist;
  r.bw = (K_sel > 0 ? K_sel : k_hist) + 1;
  r.L = L; r.R = R; r.Sl = Sl; r.Sg = Sg; r.I = I_work; r.F = F_ring;
  {
    double* w = (double*)ctx->d_ctl;
    const size_t srow = (size_t)n_max * MM * 2;
    r.Sring = w;               w += (size_t)kRing * 2 * srow;
    r.eps_ring = w;            w += (size_t)kRing * MM * 2;
    r.ypred = w;               w += 2 * srow;
    r.ycur = w;                w += 2 * srow;
    r.out = w;                 w += 4;
    r.partial = w;
  }
  // the growing grid: point 0 now, point n per attempt of step n
  HostGrid& g = ctx->grid;
  g = HostGrid{};
  g.n_t = 1;
  g.K = r.bw - 1;
  g.t.assign(n_max, 0.0);
  g.order.assign(n_max, 0);
  g.wbar.assign(n_max, 0.0);
  g.band.assign((size_t)n_max * r.bw, 0.0);
  ctx->grid_set = true;
  ctx->band_w = r.bw;
  ctx->adaptive_K = K_sel;
  ctx->adaptive_rows = 1;
  ctx->planes_L = ctx->planes_R = nullptr;
  ctx->planes_rows = 0;
  if ((e = cudaMemsetAsync(ctx->d_band, 0, (size_t)n_max * r.bw * sizeof(double), r.s)) != cudaSuccess ||
      (e = cudaMemsetAsync(ctx->d_wbar, 0, n_max * sizeof(double), r.s)) != cudaSuccess ||
      (K_sel > 0 && (e = cudaMemsetAsync(ctx->d_korder, 0, n_max * sizeof(int), r.s)) != cudaSuccess))
    return cuda_fail(ctx, e, "kbe_run_controlled: reset");
  std::vector<int> qused(n_max, 0);
  int n_err = 0, n_conv = 0, n = 1, rc = 0;
  auto finish = [&](kbe_status status) -> kbe_status {
    ctx->last_launches = r.launches;
    stats[0] = n - 1; stats[1] = n_err; stats[2] = n_conv; stats[3] = r.nfev; stats[4] = r.nrecon;
    *n_rows = n;
    std::vector<int> ko(n_max, 0);
    if (K_sel > 0) {
      cudaError_t e2 = cudaStreamSynchronize(r.s);
      if (e2 == cudaSuccess) e2 = cudaMemcpy(ko.data(), ctx->d_korder, n_max * sizeof(int), cudaMemcpyDeviceToHost);
      if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "kbe_run_controlled: orders");
    } else {
      for (int l = 1; l < n; ++l) ko[l] = k_hist;
    }
    for (int i = 0; i < n_max; ++i) {
      t_out[i] = i < n ? g.t[i] : 0.0;
      q_out[i] = i < n ? qused[i] : 0;
      korder_out[i] = i < n ? ko[i] : 0;
    }
    if (status != KBE_OK) return status;
    // the context's grid becomes the accepted grid with the history orders used
    std::vector<double> tg(g.t.begin(), g.t.begin() + n);
    std::vector<int> og(ko.begin(), ko.begin() + n);
    cudaError_t e2 = cudaStreamSynchronize(r.s);
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "kbe_run_controlled: stream");
    kbe_status st2 = kbe_set_grid(ctx, tg.data(), og.data(), n);
    if (st2 != KBE_OK) return st2;
    ctx->last_launches = r.launches;
    if (rc == 1) return fail(ctx, KBE_ERANGE, "kbe_run_controlled: n_max rows filled before t_end");
    return KBE_OK;
  };
  // row 0: its right-hand side, self-energy and Fock matrix
  if ((st = ctl_feval(r, 0)) != KBE_OK || (st = ctl_store(r, 0)) != KBE_OK) return finish(st);
  double h = h0, eta_max = 1e4;
  int q = 1, qsteps = 0;
  double host[2];
  const double addon = 1e-6;
  while (g.t[n - 1] < t_end * (1.0 - 1e-14)) {
    if (n >= n_max) { rc = 1; break; }
    int nef = 0, ncf = 0;
    bool failed = false;
    double E = 0.0;
    const double N = (2.0 * n + 1.0) * MM;
    for (;;) {  // attempts of step n
      if (h_max > 0.0 && h > h_max) h = h_max;
      if (g.t[n - 1] + h > t_end) h = t_end - g.t[n - 1];
      if (q > n) q = n;
      g.t[n] = g.t[n - 1] + h;
      g.order[n] = k_hist;
      g.n_t = n + 1;
      if ((st = ctl_interval_weights(r, n)) != KBE_OK) return finish(st);
      CtlArgs a{};
      a.M = M; a.n = n; a.q = q; a.n_max = n_max;
      a.L = (double*)L; a.R = (double*)R; a.F = (const double*)F_ring;
      a.rtol = rtol; a.atol = atol;
      a.ypred = r.ypred; a.ycur = r.ycur; a.partial = r.partial; a.status = ctx->d_status;
      a.q1 = a.q2 = -1;
      if ((st = local_weights(g.t.data() + n - q, q - 1, g.t[n - 1], g.t[n], a.wp, &ctx->err)) != KBE_OK ||
          (st = local_weights(g.t.data() + n - q + 1, q - 1, g.t[n - 1], g.t[n], a.wc, &ctx->err)) != KBE_OK)
        return finish(st);
      int np[kWTab], nc[kWTab];
      for (int i = 1; i <= q; ++i) np[i - 1] = n - i;
      for (int i = 0; i < q; ++i) nc[i] = n - i;
      const double Ep = error_integral(g.t.data(), n, np, q), Ec = error_integral(g.t.data(), n, nc, q);
      const double Cm = Ec / (Ep - Ec);
      if ((e = launch_ctl_predict(a, r.s)) != cudaSuccess) return finish(cuda_fail(ctx, e, "kbe_run_controlled: predictor"));
      ++r.launches;
      bool conv = false;
      double Rr = 1.0, dprev = 0.0, esq = 0.0;
      for (int m = 1; m <= 3; ++m) {
        if ((st = ctl_feval(r, n)) != KBE_OK) return finish(st);
        if ((e = launch_ctl_correct(a, r.out, r.s)) != cudaSuccess)
          return finish(cuda_fail(ctx, e, "kbe_run_controlled: corrector"));
        r.launches += 2;
        if ((st = ctl_read(r, host)) != KBE_OK) return finish(st);
        const double d = std::sqrt(host[0] / N);
        esq = host[1];
        if (m > 1) Rr = std::max(0.3 * Rr, d / dprev);
        if (Rr * d * std::fabs(Cm) < 0.1) { conv = true; break; }
        if (m > 1 && d > 2.0 * dprev) break;
        dprev = d;
      }
      if (!conv) {
        ++n_conv; ++ncf; failed = true;
        if (ncf > 10) return finish(fail(ctx, KBE_ENUMERIC, "kbe_run_controlled: fixed-point iteration failed 10 times"));
        h *= 0.25;
        continue;
      }
      E = std::fabs(Cm) * std::sqrt(esq / N);
      if (E > 1.0) {
        ++n_err; ++nef; failed = true;
        if (nef > 7) return finish(fail(ctx, KBE_ENUMERIC, "kbe_run_controlled: error test failed 7 times"));
        if (nef >= 3) { q = 1; qsteps = 0; h *= 0.1; continue; }
        const double eta = 1.0 / (std::pow(6.0 * E, 1.0 / (q + 1)) + addon);
        h *= std::max(0.1, std::min(0.9, eta));
        continue;
      }
      break;
    }
    // accepted row n
    qused[n] = q;
    if ((st = ctl_store(r, n)) != KBE_OK) return finish(st);
    {
      ReconArgs rr{M, n, std::max(0, n - std::min(q + 1, 12)), n_max, (const double*)L, (const double*)R, r.Sring,
                   r.eps_ring, weights_view(ctx), (double*)F_ring, ctx->d_status};
      if ((e = launch_ctl_reconstruct(rr, r.s)) != cudaSuccess)
        return finish(cuda_fail(ctx, e, "kbe_run_controlled: reconstruction"));
      ++r.launches;
      r.nrecon += n - rr.jlo;
    }
    ++qsteps;
    double eta = E > 0.0 ? 1.0 / (std::pow(6.0 * E, 1.0 / (q + 1)) + addon) : eta_max;
    int qn = q;
    if (qsteps > q) {
      CtlArgs a{};
      a.M = M; a.n = n; a.q = q; a.n_max = n_max;
      a.L = (double*)L; a.R = (double*)R; a.F = (const double*)F_ring;
      a.rtol = rtol; a.atol = atol; a.partial = r.partial; a.status = ctx->d_status;
      a.q1 = q > 1 ? q - 1 : -1;
      a.q2 = (q < q_max && n - q - 1 >= 0) ? q + 1 : -1;
      double P1 = 0.0, P2 = 0.0;
      int nodes[kWTab + 1];
      for (int i = 0; i <= q; ++i) nodes[i] = n - i;
      if (a.q1 >= 0) { divdiff_coeffs(g.t.data(), n, a.q1, a.wp); P1 = std::fabs(error_integral(g.t.data(), n, nodes, a.q1)); }
      if (a.q2 >= 0) { divdiff_coeffs(g.t.data(), n, a.q2, a.wc); P2 = std::fabs(error_integral(g.t.data(), n, nodes, a.q2)); }
      if (a.q1 >= 0 || a.q2 >= 0) {
        if ((e = launch_ctl_divdiff(a, r.out, r.s)) != cudaSuccess)
          return finish(cuda_fail(ctx, e, "kbe_run_controlled: order estimates"));
        r.launches += 2;
        if ((st = ctl_read(r, host)) != KBE_OK) return finish(st);
        if (a.q1 >= 0) {
          const double Eq = P1 * std::sqrt(host[0] / N);
          const double e2 = Eq > 0.0 ? 1.0 / (std::pow(6.0 * Eq, 1.0 / q) + addon) : eta_max;
          if (e2 > eta) { eta = e2; qn = q - 1; }
        }
        if (a.q2 >= 0) {
          const double Eq = P2 * std::sqrt(host[1] / N);
          const double e2 = Eq > 0.0 ? 1.0 / (std::pow(10.0 * Eq, 1.0 / (q + 2)) + addon) : eta_max;
          if (e2 > eta) { eta = e2; qn = q + 1; }
        }
      }
    }
    if (qn != q) { q = qn; qsteps = 0; }
    if (eta < 1.5) eta = 1.0;
    else eta = std::min(eta, failed ? 1.0 : eta_max);
    h *= eta;
    eta_max = 10.0;
    ++n;
  }
  return finish(KBE_OK);
}

kbe_status kbe_sync_status(kbe_ctx* ctx, void* stream) {
  if (!ctx) return KBE_EINVAL;
  ctx->last_launches = 0;
  kbe_status st = use_device(ctx);
  if (st != KBE_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "kbe_sync_status: stream");
  int flag = 0;
  if ((e = cudaMemcpy(&flag, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(ctx, e, "kbe_sync_status: read");
  if ((e = cudaMemset(ctx->d_status, 0, sizeof(int))) != cudaSuccess)
    return cuda_fail(ctx, e, "kbe_sync_status: clear");
  if (flag & kStatusTimeout) return fail(ctx, KBE_ETIMEOUT, "a device wait ran out");
  if (flag & kStatusInternal) return fail(ctx, KBE_ECUDA, "a kernel found an inconsistent launch geometry");
  if (flag & kStatusNumeric) return fail(ctx, KBE_ENUMERIC, "a kernel produced a non-finite value");
  return KBE_OK;
}

}  // extern "C"
