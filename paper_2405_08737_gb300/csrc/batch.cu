// batch.cu -- many independent systems advanced by one batched KBE step.
//
// Each system is a context (its own orbital count M, grid, weights, model)
// with caller-owned state (L, R triangles, self-energy rows, history slice,
// right-hand-side ring).  One batched step advances every active system by
// one row n_i, with the same arithmetic as kbe_step:
//   plan -> predictor -> P x { self-energy, prep, history (persistent),
//                              reduce, Fock, right-hand side, corrector }.
// All kernels read the per-system descriptors from device memory and the
// rows of the step from a small device array, so the whole step is one
// CUDA graph that does not depend on the rows; a step is one H2D copy of the
// rows and one graph launch.
//
// The FP64 history contraction runs as one persistent kernel over a work
// list of (system, tile, history chunk) items: a tile is `block` consecutive
// output entries (c, a, b) of one system's slice, a chunk a contiguous range
// of history points m.  The chunk length follows from a target item work
// (2^item_work_log2 complex multiply-adds), so items of big and small
// systems cost about the same; items are taken in order of decreasing cost
// through an atomic counter.  (block, item_work_log2) is the tile policy; the
// autotuner times candidate policies on the batch itself.
//
// Elementwise kernels run grid-stride over the concatenation of all active
// systems' rows; a thread finds its system by binary search over the
// offsets the plan kernel wrote.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "row_kernels.cuh"

namespace kbe {
namespace {

struct BatchSys {
  int M, n_max, n_t, band_w;
  double* L;
  double* R;
  double* Sl;
  double* Sg;
  double* I;
  double* F;
  const double* wbar;
  const double* band;
  const double* corr;
  const double* pred;
  const double* h0;
  const double* U;
  const double* v;
  const int* order;     // [n_t]
  const double* field;  // [n_t]: E(t_n)
  double* eps;
  double* part;
  int64_t part_doubles;
  // written by the plan kernel
  int n;                // row of this step, -1 when inactive
  int nchunk, chunk_len, xblk;
};

struct BatchDev {
  int n_sys;
  int block;            // threads per history item (tile width in output entries)
  int item_work_log2;   // target complex multiply-adds per history item
  BatchSys* sys;
  const int* rows;
  int* rank_sys;        // [n_sys] system at rank r
  int64_t* elem_off;    // [n_sys + 1] (rank order)
  int64_t* item_off;    // [n_sys + 1] (rank order)
  unsigned long long* counter;
  int* status;
};

__device__ __forceinline__ int find_rank(const int64_t* off, int n, int64_t x) {
  int lo = 0, hi = n;  // off[lo] <= x < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ StepArgs step_of(const BatchSys& s, int* status) {
  StepArgs a;
  a.M = s.M;
  a.n = s.n;
  a.K = s.band_w - 1;
  a.kn = s.n > 0 ? s.order[s.n] : 1;
  a.field = s.field[s.n];
  a.L = s.L;
  a.R = s.R;
  a.F = s.F;
  a.n_max = s.n_max;
  a.f_base = 0;
  a.f_rows = kRing;
  a.I = s.I;
  a.h0 = s.h0;
  a.U = s.U;
  a.HF = nullptr;  // batches hold local interactions only
  a.v = s.v;
  a.eps = s.eps;
  a.corr = s.corr + (int64_t)s.n * kMaxOrder * kWTab;
  a.pred = s.pred + (int64_t)s.n * kMaxOrder * kWTab;
  a.status = status;
  return a;
}

// ------------------------------------------------------------------ plan --
// One block.  Per system: activity, history tiling, element and item counts;
// then ranks by decreasing item cost and the exclusive scans in rank order.
__global__ void batch_plan(BatchDev b) {
  extern __shared__ unsigned char sm_raw[];
  double* cost = reinterpret_cast<double*>(sm_raw);              // [n_sys]
  int64_t* elems = reinterpret_cast<int64_t*>(cost + b.n_sys);   // [n_sys]
  int64_t* items = elems + b.n_sys;                              // [n_sys]
  for (int i = threadIdx.x; i < b.n_sys; i += blockDim.x) {
    BatchSys& s = b.sys[i];
    const int n = b.rows[i];
    if (n < 1 || n >= s.n_t) {
      s.n = -1;
      s.nchunk = s.chunk_len = s.xblk = 0;
      cost[i] = -1.0;
      elems[i] = items[i] = 0;
      continue;
    }
    const int64_t MM = (int64_t)s.M * s.M;
    const int64_t outputs = (int64_t)(n + 1) * MM;
    const int64_t row = outputs;                  // complex entries of one s
    // chunk length from the target item work: block outputs x len points x ~3M MACs
    const double per_point = (double)b.block * 3.0 * s.M;
    int len = (int)fmin((double)(n + 1), fmax(1.0, ldexp(1.0, b.item_work_log2) / per_point));
    int nchunk = (n + 1 + len - 1) / len;
    if (nchunk > kMaxSplit) nchunk = kMaxSplit;
    // the prep rows and the partials must fit the system's workspace
    while (nchunk > 1 && (3 + 2 * (int64_t)nchunk) * row * 2 > s.part_doubles) --nchunk;
    len = (n + 1 + nchunk - 1) / nchunk;
    nchunk = (n + 1 + len - 1) / len;
    s.n = n;
    s.nchunk = nchunk;
    s.chunk_len = len;
    s.xblk = (int)((outputs + b.block - 1) / b.block);
    elems[i] = outputs;
    items[i] = (int64_t)s.xblk * nchunk;
    cost[i] = (double)len * (double)s.M;  // work of one item, up to the common factors
  }
  __syncthreads();
  // rank: decreasing cost, ties by index (inactive systems last)
  for (int i = threadIdx.x; i < b.n_sys; i += blockDim.x) {
    int r = 0;
    for (int j = 0; j < b.n_sys; ++j)
      r += (cost[j] > cost[i]) || (cost[j] == cost[i] && j < i);
    b.rank_sys[r] = i;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t e = 0, it = 0;
    for (int r = 0; r < b.n_sys; ++r) {
      const int i = b.rank_sys[r];
      b.elem_off[r] = e;
      b.item_off[r] = it;
      e += elems[i];
      it += items[i];
    }
    b.elem_off[b.n_sys] = e;
    b.item_off[b.n_sys] = it;
  }
}

// ------------------------------------------------------------ elementwise --
// Grid-stride over the active systems' row entries; `what` selects the body.
enum RowOp { kOpPredictor = 0, kOpSigma = 1, kOpPrep = 2, kOpRhs = 3, kOpCorrector = 4, kOpReduce = 5 };

template <int OP>
__global__ void __launch_bounds__(256) batch_rows(BatchDev b) {
  const int64_t total = b.elem_off[b.n_sys];
  bool ok = true;
  if (OP == kOpPrep && blockIdx.x == 0 && threadIdx.x == 0) *b.counter = 0ull;  // for the history launch
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = find_rank(b.elem_off, b.n_sys, e);
    const BatchSys& s = b.sys[b.rank_sys[r]];
    const int64_t lin = e - b.elem_off[r];
    const int MM = s.M * s.M;
    const int n = s.n;
    if (OP == kOpPredictor || OP == kOpCorrector) {
      rk::adams_entry(step_of(s, b.status), lin, OP == kOpCorrector);
    } else if (OP == kOpRhs) {
      ok &= rk::rhs_entry(step_of(s, b.status), lin);
    } else if (OP == kOpSigma) {
      const int64_t off = tri(n, 0) * MM;
      const int64_t blk = lin / MM;
      const int ab = (int)(lin - blk * MM);
      ok &= rk::sigma_entry(s.M, lin, ab, blk == n, rk::sigma_uu(s.M, ab, s.U),
                            reinterpret_cast<const double2*>(s.L) + off, reinterpret_cast<const double2*>(s.R) + off,
                            reinterpret_cast<double2*>(s.Sl), reinterpret_cast<double2*>(s.Sg));
    } else if (OP == kOpPrep) {
      const int64_t row = (int64_t)(n + 1) * MM;
      const WeightsView w{s.wbar, s.band, s.band_w};
      rk::history_prep_entry(MM, n, lin, s.Sl, s.Sg, w, s.part, s.part + 2 * row, s.part + 4 * row);
    } else {  // kOpReduce: both s of entry lin
      const int64_t row = (int64_t)(n + 1) * MM;
      double2* out = reinterpret_cast<double2*>(s.I);
      if (s.nchunk > 1) {
        const double2* part = reinterpret_cast<const double2*>(s.part + 6 * row);
        ok &= rk::history_reduce_entry(2 * row, s.nchunk, lin, part, out);
        ok &= rk::history_reduce_entry(2 * row, s.nchunk, lin + row, part, out);
      } else {
        const double2 x = out[lin], y = out[lin + row];
        ok &= isfinite(x.x) && isfinite(x.y) && isfinite(y.x) && isfinite(y.y);
      }
    }
  }
  if (!ok) atomicOr(b.status, kStatusNumeric);
}

__global__ void batch_fock(BatchDev b) {
  const BatchSys& s = b.sys[blockIdx.x];
  if (s.n < 1) return;
  const StepArgs a = step_of(s, b.status);
  for (int ab = threadIdx.x; ab < s.M * s.M; ab += blockDim.x) rk::fock_entry(a, ab);
}

// --------------------------------------------------------- history slice --
// Persistent: each block takes items from the counter until the list is done.
template <int BS>
__global__ void __launch_bounds__(BS) batch_history(BatchDev b) {
  __shared__ long long item_s;
  const long long total = b.item_off[b.n_sys];
  for (;;) {
    if (threadIdx.x == 0) item_s = (long long)atomicAdd(b.counter, 1ull);
    __syncthreads();
    const long long item = item_s;
    __syncthreads();
    if (item >= total) break;
    const int r = find_rank(b.item_off, b.n_sys, item);
    const BatchSys& s = b.sys[b.rank_sys[r]];
    const long long local = item - b.item_off[r];
    const int xb = (int)(local % s.xblk);
    const int chunk = (int)(local / s.xblk);
    const int MM = s.M * s.M;
    const int n = s.n;
    const int64_t row = (int64_t)(n + 1) * MM;
    const int64_t lin = (int64_t)xb * BS + threadIdx.x;
    if (lin < row) {
      rk::PartialArgs p{s.M, MM, n, s.chunk_len, s.L, s.R, s.Sl, s.Sg, s.part, s.part + 2 * row,
                        s.part + 4 * row, WeightsView{s.wbar, s.band, s.band_w},
                        s.nchunk == 1 ? s.I : s.part + 6 * row};
      rk::history_partial_entry(p, lin, chunk);
    }
  }
}

}  // namespace
}  // namespace kbe

// ------------------------------------------------------------- host side --
using namespace kbe;

struct kbe_batch {
  int n_sys = 0;
  int device = 0;
  std::string err;
  std::vector<kbe_ctx*> ctx;
  std::vector<BatchSys> sys;     // host mirror of the descriptors
  std::vector<char> bound;
  BatchDev dev{};
  void* d_mem = nullptr;         // descriptors, rows, ranks, offsets, counter, status
  int* d_order = nullptr;        // concatenated order tables
  double* d_field = nullptr;     // concatenated field tables
  bool dirty = true;             // descriptors need an upload
  int hist_blocks[2] = {0, 0};   // persistent grid for block = 128, 256
  // graph of one step for (P, precision, policy); split graphs also key on rows
  cudaGraphExec_t graph = nullptr;
  int g_P = 0, g_prec = -1, g_block = 0, g_work = 0;
  std::vector<int> g_rows;
  int g_count = 0;               // kernels in the step graph
  int last_launches = 0;
  // split precision: the work list of the fused contraction over every
  // active system (host plan, its device image) and the partial sums
  FusedPlanHost fplan;
  std::vector<int> fplan_rows;           // the rows the work list was built for
  std::vector<unsigned char> fplan_up;   // the image on the device
  void* d_fplan = nullptr;
  size_t fplan_bytes = 0;
  double* d_fpart = nullptr;
  size_t fpart_bytes = 0;
};

namespace {

kbe_status bfail(kbe_batch* b, kbe_status st, const std::string& msg) {
  if (b) b->err = msg; else set_global_error(msg.c_str());
  return st;
}

kbe_status bcuda(kbe_batch* b, cudaError_t e, const char* where) {
  return bfail(b, KBE_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void drop_graph(kbe_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->g_P = 0;
  b->g_prec = -1;
}


// Enqueue one batched step (rows already on the device).  Split precision
// runs the fused contraction over the work list built from the host rows
// (its image already uploaded).
cudaError_t enqueue_step(kbe_batch* b, int P, int precision, const int* rows_host, cudaStream_t s, int* count) {
  BatchDev d = b->dev;
  int nl = 0;
  batch_plan<<<1, 256, (size_t)b->n_sys * 24, s>>>(d);
  ++nl;
  batch_rows<kOpPredictor><<<sm_count() * 8, 256, 0, s>>>(d);
  ++nl;
  cudaError_t e = cudaGetLastError();
  for (int it = 0; it < P && e == cudaSuccess; ++it) {
    batch_rows<kOpSigma><<<sm_count() * 8, 256, 0, s>>>(d);
    ++nl;
    if (precision == KBE_FP64) {  // prep also clears the work counter
      batch_rows<kOpPrep><<<sm_count() * 8, 256, 0, s>>>(d);
      if (d.block == 128)
        batch_history<128><<<b->hist_blocks[0], 128, 0, s>>>(d);
      else
        batch_history<256><<<b->hist_blocks[1], 256, 0, s>>>(d);
      batch_rows<kOpReduce><<<sm_count() * 8, 256, 0, s>>>(d);
      nl += 3;
    } else if (precision == KBE_DF64) {  // each system's double-float slice in its context's workspace
      for (int i = 0; i < b->n_sys && e == cudaSuccess; ++i) {
        const int n = rows_host[i];
        const kbe_ctx* c = b->ctx[i];
        if (n < 1 || n >= c->grid.n_t) continue;
        const BatchSys& y = b->sys[i];
        HistoryArgs a{y.M, n, y.L, y.R, y.Sl, y.Sg, WeightsView{y.wbar, y.band, y.band_w}, y.I, c->d_part,
                      c->part_bytes, d.status};
        int k = 0;
        e = launch_history_df(a, s, &k);
        nl += k;
      }
    } else if (b->fplan.n_ent > 0) {  // one persistent tensor-core contraction over every active system's units
      int k = 0;
      e = launch_history_fused(b->fplan, b->d_fplan, b->d_fpart, d.status, s, &k);
      nl += k;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    batch_fock<<<b->n_sys, 256, 0, s>>>(d);
    batch_rows<kOpRhs><<<sm_count() * 8, 256, 0, s>>>(d);
    batch_rows<kOpCorrector><<<sm_count() * 8, 256, 0, s>>>(d);
    nl += 3;
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  *count = nl;
  return e;
}

kbe_status upload(kbe_batch* b) {
  if (!b->dirty) return KBE_OK;
  for (int i = 0; i < b->n_sys; ++i)
    if (!b->bound[i]) return bfail(b, KBE_ESTATE, "kbe_batch: system " + std::to_string(i) + " has no state bound");
  cudaError_t e = cudaMemcpy(b->dev.sys, b->sys.data(), b->sys.size() * sizeof(BatchSys), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bcuda(b, e, "kbe_batch: descriptor upload");
  b->dirty = false;
  return KBE_OK;
}

}  // namespace

extern "C" {

kbe_status kbe_batch_create(kbe_ctx* const* ctxs, int n_sys, kbe_batch** out) {
  if (!out) return bfail(nullptr, KBE_EINVAL, "kbe_batch_create: out is NULL");
  *out = nullptr;
  if (!ctxs || n_sys < 1 || n_sys > 1024) return bfail(nullptr, KBE_EINVAL, "kbe_batch_create: n_sys outside [1, 1024]");
  int dev0 = -1;
  for (int i = 0; i < n_sys; ++i) {
    const kbe_ctx* c = ctxs[i];
    if (!c) return bfail(nullptr, KBE_EINVAL, "kbe_batch_create: NULL context");
    if (!c->grid_set || !c->model.set)
      return bfail(nullptr, KBE_ESTATE, "kbe_batch_create: every context needs its grid and model set");
    if (c->adaptive_K > 0)
      return bfail(nullptr, KBE_EINVAL, "kbe_batch_create: batched steps use the grids' history orders");
    if (c->dense)
      return bfail(nullptr, KBE_EINVAL, "kbe_batch_create: batched steps use the local interaction");
    if (c->thermal)
      return bfail(nullptr, KBE_EINVAL, "kbe_batch_create: batched steps have no thermal branch");
    if (dev0 < 0) dev0 = c->device;
    if (c->device != dev0) return bfail(nullptr, KBE_EINVAL, "kbe_batch_create: contexts on different devices");
  }
  kbe_batch* b = new (std::nothrow) kbe_batch();
  if (!b) return bfail(nullptr, KBE_ENOMEM, "kbe_batch_create: host allocation failed");
  b->n_sys = n_sys;
  b->device = dev0;
  b->ctx.assign(ctxs, ctxs + n_sys);
  b->sys.resize(n_sys);
  b->bound.assign(n_sys, 0);
  cudaError_t e = cudaSetDevice(dev0);
  // device block: descriptors | rows | rank | elem_off | item_off | counter | status
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = (off + bytes + 255) / 256 * 256; return o; };
  const size_t o_sys = take(sizeof(BatchSys) * n_sys), o_rows = take(sizeof(int) * n_sys),
               o_rank = take(sizeof(int) * n_sys), o_eoff = take(sizeof(int64_t) * (n_sys + 1)),
               o_ioff = take(sizeof(int64_t) * (n_sys + 1)), o_cnt = take(sizeof(unsigned long long)),
               o_st = take(sizeof(int));
  size_t n_order = 0;
  for (int i = 0; i < n_sys; ++i) n_order += ctxs[i]->grid.n_t;
  if (e == cudaSuccess) e = cudaMalloc(&b->d_mem, off);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_order, n_order * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_field, n_order * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(b->d_mem, 0, off);
  if (e != cudaSuccess) {
    cudaFree(b->d_mem); cudaFree(b->d_order); cudaFree(b->d_field);
    delete b;
    cudaGetLastError();
    return bfail(nullptr, e == cudaErrorMemoryAllocation ? KBE_ENOMEM : KBE_ECUDA,
                 std::string("kbe_batch_create: ") + cudaGetErrorString(e));
  }
  char* base = static_cast<char*>(b->d_mem);
  b->dev.n_sys = n_sys;
  b->dev.block = 256;
  b->dev.item_work_log2 = 20;
  b->dev.sys = reinterpret_cast<BatchSys*>(base + o_sys);
  b->dev.rows = reinterpret_cast<int*>(base + o_rows);
  b->dev.rank_sys = reinterpret_cast<int*>(base + o_rank);
  b->dev.elem_off = reinterpret_cast<int64_t*>(base + o_eoff);
  b->dev.item_off = reinterpret_cast<int64_t*>(base + o_ioff);
  b->dev.counter = reinterpret_cast<unsigned long long*>(base + o_cnt);
  b->dev.status = reinterpret_cast<int*>(base + o_st);
  // per-system tables
  std::vector<int> order(n_order);
  std::vector<double> field(n_order);
  size_t at = 0;
  for (int i = 0; i < n_sys; ++i) {
    const kbe_ctx* c = ctxs[i];
    const int nt = c->grid.n_t;
    BatchSys& y = b->sys[i];
    std::memset(&y, 0, sizeof(y));
    y.M = c->M;
    y.n_max = c->n_max;
    y.n_t = nt;
    y.band_w = c->grid.K + 1;
    y.wbar = c->d_wbar;
    y.band = c->d_band;
    y.corr = c->d_corr;
    y.pred = c->d_pred;
    y.h0 = c->d_h0;
    y.U = c->d_U;
    y.v = c->d_v;
    y.eps = c->d_eps;
    y.part = c->d_part;
    y.part_doubles = (int64_t)(c->part_bytes / sizeof(double));
    y.order = b->d_order + at;
    y.field = b->d_field + at;
    y.n = -1;
    for (int j = 0; j < nt; ++j) {
      order[at + j] = c->grid.order[j];
      field[at + j] = c->model.field(c->grid.t[j]);
    }
    at += nt;
  }
  if ((e = cudaMemcpy(b->d_order, order.data(), n_order * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b->d_field, field.data(), n_order * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) {
    kbe_status st = bcuda(nullptr, e, "kbe_batch_create: table upload");
    cudaFree(b->d_mem); cudaFree(b->d_order); cudaFree(b->d_field);
    delete b;
    return st;
  }
  const int sms = sm_count();
  int occ128 = 1, occ256 = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ128, batch_history<128>, 128, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ256, batch_history<256>, 256, 0);
  b->hist_blocks[0] = sms * std::max(1, occ128);
  b->hist_blocks[1] = sms * std::max(1, occ256);
  cudaGetLastError();
  *out = b;
  return KBE_OK;
}

kbe_status kbe_batch_destroy(kbe_batch* b) {
  if (!b) return KBE_OK;
  cudaSetDevice(b->device);
  drop_graph(b);
  cudaFree(b->d_mem);
  cudaFree(b->d_order);
  cudaFree(b->d_field);
  cudaFree(b->d_fplan);
  cudaFree(b->d_fpart);
  delete b;
  return KBE_OK;
}

const char* kbe_batch_last_error(const kbe_batch* b) { return b ? b->err.c_str() : kbe_last_error(nullptr); }

int kbe_batch_last_launch_count(const kbe_batch* b) { return b ? b->last_launches : 0; }

kbe_status kbe_batch_bind(kbe_batch* b, int i, void* L, void* R, void* S_less, void* S_great, void* I_work,
                          void* F_ring) {
  if (!b) return KBE_EINVAL;
  if (i < 0 || i >= b->n_sys) return bfail(b, KBE_EINVAL, "kbe_batch_bind: system index out of range");
  for (const void* p : {(const void*)L, (const void*)R, (const void*)S_less, (const void*)S_great,
                        (const void*)I_work, (const void*)F_ring})
    if (!p || (reinterpret_cast<uintptr_t>(p) & 15u)) return bfail(b, KBE_EINVAL, "kbe_batch_bind: NULL or misaligned pointer");
  BatchSys& y = b->sys[i];
  y.L = (double*)L; y.R = (double*)R; y.Sl = (double*)S_less; y.Sg = (double*)S_great;
  y.I = (double*)I_work; y.F = (double*)F_ring;
  b->bound[i] = 1;
  b->dirty = true;
  drop_graph(b);  // split graphs hold the pointers
  b->fplan_rows.clear();  // and so does the split work list: rebuild it
  return KBE_OK;
}

kbe_status kbe_batch_set_policy(kbe_batch* b, int block, int item_work_log2) {
  if (!b) return KBE_EINVAL;
  if (block != 128 && block != 256) return bfail(b, KBE_EINVAL, "kbe_batch_set_policy: block must be 128 or 256");
  if (item_work_log2 < 10 || item_work_log2 > 40) return bfail(b, KBE_EINVAL, "kbe_batch_set_policy: item_work_log2 outside [10, 40]");
  if (block != b->dev.block || item_work_log2 != b->dev.item_work_log2) {
    b->dev.block = block;
    b->dev.item_work_log2 = item_work_log2;
    drop_graph(b);
  }
  return KBE_OK;
}

kbe_status kbe_batch_get_policy(const kbe_batch* b, int* block, int* item_work_log2) {
  if (!b || !block || !item_work_log2) return KBE_EINVAL;
  *block = b->dev.block;
  *item_work_log2 = b->dev.item_work_log2;
  return KBE_OK;
}

kbe_status kbe_batch_step(kbe_batch* b, const int* rows, int P, int precision, void* stream) {
  if (!b) return KBE_EINVAL;
  b->last_launches = 0;
  if (!rows) return bfail(b, KBE_EINVAL, "kbe_batch_step: rows is NULL");
  if (P < 1 || P > 16) return bfail(b, KBE_EINVAL, "kbe_batch_step: P outside [1, 16]");
  if (precision != KBE_FP64 && precision != KBE_SPLIT_BF16 && precision != KBE_DF64)
    return bfail(b, KBE_EINVAL, "kbe_batch_step: unknown precision");
  for (int i = 0; i < b->n_sys; ++i) {
    const kbe_ctx* c = b->ctx[i];
    if (rows[i] >= c->grid.n_t) return bfail(b, KBE_ERANGE, "kbe_batch_step: row beyond a system's grid");
    if (precision == KBE_SPLIT_BF16 && rows[i] >= 1 && !c->d_split)
      return bfail(b, KBE_EINVAL, "kbe_batch_step: split precision needs 1 <= norb <= 32 in every active system");
  }
  cudaError_t e = cudaSetDevice(b->device);
  if (e != cudaSuccess) return bcuda(b, e, "kbe_batch_step: cudaSetDevice");
  kbe_status st = upload(b);
  if (st != KBE_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // rows of this step (pageable copy: the host array may be reused on return)
  if ((e = cudaMemcpyAsync((void*)b->dev.rows, rows, sizeof(int) * b->n_sys, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return bcuda(b, e, "kbe_batch_step: rows upload");
  const bool same_rows = precision == KBE_FP64 ||
                         ((int)b->g_rows.size() == b->n_sys && std::equal(b->g_rows.begin(), b->g_rows.end(), rows));
  if (precision == KBE_SPLIT_BF16 && (e = split_prepare()) != cudaSuccess) return bcuda(b, e, "kbe_batch_step: split setup");
  if (precision == KBE_SPLIT_BF16 &&
      !((int)b->fplan_rows.size() == b->n_sys && std::equal(b->fplan_rows.begin(), b->fplan_rows.end(), rows))) {
    // the work list of these rows, before any capture
    b->fplan_rows.clear();
    std::vector<FusedSystem> fs;
    for (int i = 0; i < b->n_sys; ++i) {
      if (rows[i] < 1) continue;
      const BatchSys& y = b->sys[i];
      fs.push_back(FusedSystem{y.M, rows[i], y.L, y.R, y.Sl, y.Sg, WeightsView{y.wbar, y.band, y.band_w}, y.I,
                               b->ctx[i]->d_split});
    }
    if (fs.empty()) {
      b->fplan = FusedPlanHost{};
    } else {
      if (!fused_build(fs.data(), (int)fs.size(), &b->fplan))
        return bfail(b, KBE_EINVAL, "kbe_batch_step: split work list");
      const size_t need_plan = b->fplan.image.size(), need_part = fused_part_bytes(b->fplan);
      if (need_plan > b->fplan_bytes || need_part > b->fpart_bytes) {
        drop_graph(b);  // the graph holds the buffers' addresses
        if (need_plan > b->fplan_bytes) {
          cudaFree(b->d_fplan);
          b->d_fplan = nullptr;
          b->fplan_bytes = 0;
          b->fplan_up.clear();
          if ((e = cudaMalloc(&b->d_fplan, need_plan)) != cudaSuccess) {
            b->d_fplan = nullptr;
            return bfail(b, KBE_ENOMEM, "kbe_batch_step: split work list buffer");
          }
          b->fplan_bytes = need_plan;
        }
        if (need_part > b->fpart_bytes) {
          cudaFree(b->d_fpart);
          b->d_fpart = nullptr;
          b->fpart_bytes = 0;
          if ((e = cudaMalloc(&b->d_fpart, need_part)) != cudaSuccess) {
            b->d_fpart = nullptr;
            return bfail(b, KBE_ENOMEM, "kbe_batch_step: split partial sums");
          }
          b->fpart_bytes = need_part;
        }
      }
      if (b->fplan.image != b->fplan_up) {  // stream-ordered after the steps already queued
        if ((e = cudaMemcpyAsync(b->d_fplan, b->fplan.image.data(), b->fplan.image.size(), cudaMemcpyHostToDevice,
                                 s)) != cudaSuccess)
          return bcuda(b, e, "kbe_batch_step: split work list upload");
        b->fplan_up = b->fplan.image;
      }
    }
    b->fplan_rows.assign(rows, rows + b->n_sys);
  }
  if (!b->graph || b->g_P != P || b->g_prec != precision || b->g_block != b->dev.block ||
      b->g_work != b->dev.item_work_log2 || !same_rows) {
    drop_graph(b);
    cudaStream_t cs;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return bcuda(b, e, "kbe_batch_step: capture stream");
    cudaGraph_t g = nullptr;
    int count = 0;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t el = enqueue_step(b, P, precision, rows, cs, &count);
      e = cudaStreamEndCapture(cs, &g);
      if (el != cudaSuccess) e = el;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      cudaGetLastError();
      return bcuda(b, e, "kbe_batch_step: graph capture");
    }
    b->g_P = P;
    b->g_prec = precision;
    b->g_block = b->dev.block;
    b->g_work = b->dev.item_work_log2;
    b->g_rows.assign(rows, rows + b->n_sys);
    b->g_count = count;
  }
  b->last_launches = b->g_count;
  if ((e = cudaGraphLaunch(b->graph, s)) != cudaSuccess) return bcuda(b, e, "kbe_batch_step: graph launch");
  return KBE_OK;
}

kbe_status kbe_batch_autotune(kbe_batch* b, const int* rows, int reps, void* stream, int* block_out,
                              int* work_out, double* best_ms) {
  if (!b) return KBE_EINVAL;
  if (!rows || reps < 1 || reps > 100) return bfail(b, KBE_EINVAL, "kbe_batch_autotune: rows NULL or reps outside [1, 100]");
  for (int i = 0; i < b->n_sys; ++i)
    if (rows[i] >= b->ctx[i]->grid.n_t) return bfail(b, KBE_ERANGE, "kbe_batch_autotune: row beyond a system's grid");
  cudaError_t e = cudaSetDevice(b->device);
  if (e != cudaSuccess) return bcuda(b, e, "kbe_batch_autotune: cudaSetDevice");
  kbe_status st = upload(b);
  if (st != KBE_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((e = cudaMemcpyAsync((void*)b->dev.rows, rows, sizeof(int) * b->n_sys, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return bcuda(b, e, "kbe_batch_autotune: rows upload");
  // the slice of the current state: self-energy rows, then timed history slices
  BatchDev d = b->dev;
  batch_plan<<<1, 256, (size_t)b->n_sys * 24, s>>>(d);
  batch_rows<kOpSigma><<<sm_count() * 8, 256, 0, s>>>(d);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks[2] = {128, 256};
  double best = 1e300;
  int bb = b->dev.block, bw = b->dev.item_work_log2;
  for (int bi = 0; bi < 2 && e == cudaSuccess; ++bi) {
    for (int lw = 14; lw <= 26 && e == cudaSuccess; lw += 2) {
      d.block = blocks[bi];
      d.item_work_log2 = lw;
      double tot = 0.0;
      for (int r = 0; r <= reps && e == cudaSuccess; ++r) {  // r = 0 warms up
        batch_plan<<<1, 256, (size_t)b->n_sys * 24, s>>>(d);
        batch_rows<kOpPrep><<<sm_count() * 8, 256, 0, s>>>(d);
        cudaEventRecord(e0, s);
        if (d.block == 128) batch_history<128><<<b->hist_blocks[0], 128, 0, s>>>(d);
        else batch_history<256><<<b->hist_blocks[1], 256, 0, s>>>(d);
        cudaEventRecord(e1, s);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) tot += ms;
      }
      if (e == cudaSuccess && tot / reps < best) {
        best = tot / reps;
        bb = d.block;
        bw = lw;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return bcuda(b, e, "kbe_batch_autotune");
  st = kbe_batch_set_policy(b, bb, bw);
  if (st != KBE_OK) return st;
  if (block_out) *block_out = bb;
  if (work_out) *work_out = bw;
  if (best_ms) *best_ms = best;
  return KBE_OK;
}

kbe_status kbe_batch_sync_status(kbe_batch* b, void* stream) {
  if (!b) return KBE_EINVAL;
  cudaError_t e = cudaSetDevice(b->device);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return bcuda(b, e, "kbe_batch_sync_status");
  int flag = 0;
  if ((e = cudaMemcpy(&flag, b->dev.status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemset(b->dev.status, 0, sizeof(int))) != cudaSuccess)
    return bcuda(b, e, "kbe_batch_sync_status: status word");
  if (flag & kStatusTimeout) return bfail(b, KBE_ETIMEOUT, "a device wait ran out");
  if (flag & kStatusInternal) return bfail(b, KBE_ECUDA, "a kernel found an inconsistent launch geometry");
  if (flag & kStatusNumeric) return bfail(b, KBE_ENUMERIC, "a kernel produced a non-finite value");
  return KBE_OK;
}

}  // extern "C"
