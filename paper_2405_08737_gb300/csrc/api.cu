// api.cu -- the C ABI of libkbe (declared in include/kbe.h): argument
// validation, device workspace, and the launch sequences of each call.

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
  return WeightsView{ctx->d_wbar, ctx->d_band, ctx->grid.K + 1};
}

template <class T> cudaError_t dev_alloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T) + 16);
}

void release(kbe_ctx* ctx) {
  for (cudaEvent_t ev : ctx->ev_pool) cudaEventDestroy(ev);
  ctx->ev_pool.clear();
  cudaFree(ctx->d_wbar); cudaFree(ctx->d_band); cudaFree(ctx->d_corr); cudaFree(ctx->d_pred);
  cudaFree(ctx->d_h0); cudaFree(ctx->d_U); cudaFree(ctx->d_v); cudaFree(ctx->d_eps);
  cudaFree(ctx->d_part); cudaFree(ctx->d_status); cudaFree(ctx->d_split);
  ctx->d_split = nullptr;
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

kbe_status history(kbe_ctx* ctx, int n, int precision, const void* L, const void* R, const void* Sl,
                   const void* Sg, void* I_out, cudaStream_t s, int* launches) {
  if (precision == KBE_SPLIT_BF16) {
    if (!ctx->d_split) return fail(ctx, KBE_EINVAL, "split precision needs 1 <= norb <= 32");
    SplitLaunch l{ctx->M, n, (const double*)L, (const double*)R, (const double*)Sl, (const double*)Sg,
                  weights_view(ctx), (double*)I_out, ctx->d_split, ctx->split_bytes, ctx->d_status};
    if (!next_events(ctx, &l.ev_begin, &l.ev_end)) return fail(ctx, KBE_ECUDA, "profiling: cudaEventCreate");
    cudaError_t e = launch_history_split(l, s, launches);
    return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "split history slice launch");
  }
  if (precision != KBE_FP64) return fail(ctx, KBE_EINVAL, "unknown precision");
  HistoryArgs a{ctx->M, n, (const double*)L, (const double*)R, (const double*)Sl, (const double*)Sg,
                weights_view(ctx), (double*)I_out, ctx->d_part, ctx->part_bytes, ctx->d_status};
  if (!next_events(ctx, &a.ev_begin, &a.ev_end)) return fail(ctx, KBE_ECUDA, "profiling: cudaEventCreate");
  cudaError_t e = launch_history_f64(a, s, launches);
  return e == cudaSuccess ? KBE_OK : cuda_fail(ctx, e, "history slice launch");
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
  a.I = (const double*)I;
  a.h0 = ctx->d_h0;
  a.U = ctx->d_U;
  a.v = ctx->d_v;
  a.eps = ctx->d_eps;
  a.corr = ctx->d_corr + (size_t)n * kMaxOrder * kWTab;
  a.pred = ctx->d_pred + (size_t)n * kMaxOrder * kWTab;
  a.status = ctx->d_status;
  return a;
}

}  // namespace

void kbe::set_global_error(const char* msg) { g_create_err = msg; }

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
  ctx->part_bytes = (3 + 2 * (size_t)kMaxSplit) * row * 16;
  if ((e = dev_alloc(&ctx->d_part, ctx->part_bytes / sizeof(double))) != cudaSuccess ||
      (e = dev_alloc(&ctx->d_wbar, (size_t)n_max)) != cudaSuccess ||
      (e = dev_alloc(&ctx->d_band, (size_t)n_max * (kMaxOrder + 1))) != cudaSuccess ||
      (e = dev_alloc(&ctx->d_corr, (size_t)n_max * kMaxOrder * kWTab)) != cudaSuccess ||
      (e = dev_alloc(&ctx->d_pred, (size_t)n_max * kMaxOrder * kWTab)) != cudaSuccess ||
      (e = dev_alloc(&ctx->d_h0, 2 * MM)) != cudaSuccess ||
      (e = dev_alloc(&ctx->d_U, (size_t)norb)) != cudaSuccess ||
      (e = dev_alloc(&ctx->d_v, (size_t)norb)) != cudaSuccess ||
      (e = dev_alloc(&ctx->d_eps, 2 * MM)) != cudaSuccess ||
      (e = dev_alloc(&ctx->d_status, 1)) != cudaSuccess) {
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
  cudaError_t e = launch_sigma(ctx->M, tri(n, 0), n + 1, n, (const double*)L, (const double*)R, ctx->d_U,
                               (double*)Sl, (double*)Sg, ctx->d_status, (cudaStream_t)stream);
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
  cudaError_t e = launch_sigma(ctx->M, 0, tri(n_rows, 0), -1, (const double*)L, (const double*)R, ctx->d_U,
                               (double*)Sl, (double*)Sg, ctx->d_status, (cudaStream_t)stream);
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
  cudaError_t e = launch_sigma(ctx->M, tri(j, 0), j + 1, j, (const double*)L, (const double*)R, ctx->d_U,
                               (double*)Sl, (double*)Sg, ctx->d_status, s);
  ++count;
  if (e != cudaSuccess) { ctx->last_launches = count; return cuda_fail(ctx, e, "kbe_rhs_row: self-energy"); }
  st = history(ctx, j, precision, L, R, Sl, Sg, I_work, s, &nl);
  count += nl;
  if (st != KBE_OK) { ctx->last_launches = count; return st; }
  StepArgs a = step_args(ctx, j, (void*)L, (void*)R, I_work, F_ring);
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
  kbe_status st = check_row_call(ctx, n);
  if (st != KBE_OK) return st;
  if (n < 1) return fail(ctx, KBE_ERANGE, "kbe_step: n must be >= 1 (row 0 is the initial state)");
  if (P < 1 || P > 16) return fail(ctx, KBE_EINVAL, "kbe_step: P outside [1, 16]");
  if (!ctx->model.set) return fail(ctx, KBE_ESTATE, "no model: call kbe_set_model first");
  if (!aligned16(L) || !aligned16(R) || !aligned16(Sl) || !aligned16(Sg) || !aligned16(I_work) || !aligned16(F_ring))
    return fail(ctx, KBE_EINVAL, "kbe_step: NULL or misaligned pointer");
  if (precision != KBE_FP64 && precision != KBE_SPLIT_BF16) return fail(ctx, KBE_EINVAL, "kbe_step: unknown precision");
  if ((st = use_device(ctx)) != KBE_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  StepArgs a = step_args(ctx, n, L, R, I_work, F_ring);
  int count = 0, nl = 0;
  cudaError_t e = launch_predictor(a, s);
  ++count;
  if (e != cudaSuccess) { ctx->last_launches = count; return cuda_fail(ctx, e, "kbe_step: predictor"); }
  for (int it = 0; it < P; ++it) {
    e = launch_sigma(ctx->M, tri(n, 0), n + 1, n, (const double*)L, (const double*)R, ctx->d_U, (double*)Sl,
                     (double*)Sg, ctx->d_status, s);
    ++count;
    if (e != cudaSuccess) { ctx->last_launches = count; return cuda_fail(ctx, e, "kbe_step: self-energy"); }
    st = history(ctx, n, precision, L, R, Sl, Sg, I_work, s, &nl);
    count += nl;
    if (st != KBE_OK) { ctx->last_launches = count; return st; }
    if ((e = launch_fock(a, s)) != cudaSuccess || (e = launch_rhs_corrector(a, s)) != cudaSuccess) {
      ctx->last_launches = count + 3;
      return cuda_fail(ctx, e, "kbe_step: corrector");
    }
    count += 3;
  }
  ctx->last_launches = count;
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
  if (flag & kStatusNumeric) return fail(ctx, KBE_ENUMERIC, "a kernel produced a non-finite value");
  return KBE_OK;
}

}  // extern "C"
