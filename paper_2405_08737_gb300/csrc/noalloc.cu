// noalloc.cu -- a history slice that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code running inside another
// framework's memory pool or allocator hooks (where a nested allocation
// would re-enter the allocator or break its accounting), or embedded hosts
// that hand over fixed buffers only.  kbe_history_slice_noalloc() serves
// them: it needs no context, takes the grid on the host and the two-time
// data on the device, and keeps all of its scratch (weight tables, folded
// self-energy rows, split partials, status word) in one file-scope
// __device__ array of fixed size.  Every GPU that loads the library reserves that array until the
// process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call overwrites what it reads, and clears the status word.
// Calls whose kernels overlap on the GPU (different streams, no ordering)
// race on the array.

#include <cmath>
#include <mutex>

#include "kbe_internal.h"

namespace kbe {
namespace {

constexpr size_t kScratchDoubles = size_t(8) << 20;   // 64 MiB
constexpr int kNoallocMaxPoints = 8192;               // grid points
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// Host-side staging of the weight tables (no heap use on the success path).
double h_wbar[kNoallocMaxPoints];
double h_band[kNoallocMaxPoints * (kMaxOrder + 1)];
std::mutex h_mutex;

// Device address of g_noalloc_scratch, looked up once per device.
double* g_dev_scratch[kNoallocMaxDevices] = {nullptr};
std::mutex g_dev_mutex;

cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_dev_mutex);
  if (!g_dev_scratch[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_dev_scratch[dev] = static_cast<double*>(p);
  }
  *out = g_dev_scratch[dev];
  return cudaSuccess;
}

// Composite weights of Sec. 3.2 into the static host tables: settled
// vector and band of width K+1, same recursion and LU solves as the
// context path.  Returns the band width, or 0 on a bad grid.
int host_weights(const double* t, const int* order, int n_t, std::string* err) {
  int K = 1;
  for (int l = 1; l < n_t; ++l) {
    const int kap = order[l] < l ? order[l] : l;
    if (kap > K) K = kap;
  }
  const int bw = K + 1;
  for (int m = 0; m < n_t; ++m) h_wbar[m] = 0.0;
  for (int j = 0; j < n_t * bw; ++j) h_band[j] = 0.0;
  double w[kWTab];
  for (int c = 1; c < n_t; ++c) {
    const int kap = order[c] < c ? order[c] : c;
    if (local_weights(t + c - kap, kap, t[c - 1], t[c], w, err) != KBE_OK) return 0;
    for (int j = 0; j <= kap; ++j) h_wbar[c - kap + j] += w[j];
    for (int j = 0; j < bw && j <= c; ++j) h_band[c * bw + j] = h_wbar[c - j];
  }
  return bw;
}

}  // namespace
}  // namespace kbe

using namespace kbe;

extern "C" kbe_status kbe_history_slice_noalloc(int norb, int n, const double* t, const int* order, int n_t,
                                                const void* L, const void* R, const void* S_less,
                                                const void* S_great, void* I_out, void* stream) {
  // errors are reported through kbe_last_error(NULL)
  auto fail = [](kbe_status st, const char* msg) {
    set_global_error(msg);
    return st;
  };
  if (norb < 1 || norb > kMaxNorb) return fail(KBE_EINVAL, "kbe_history_slice_noalloc: norb outside [1, 64]");
  if (!t || !order) return fail(KBE_EINVAL, "kbe_history_slice_noalloc: NULL grid");
  if (n_t < 1 || n_t > kNoallocMaxPoints)
    return fail(KBE_EINVAL, "kbe_history_slice_noalloc: n_t outside [1, 8192] (the fixed scratch limit)");
  if (n < 0 || n >= n_t) return fail(KBE_ERANGE, "kbe_history_slice_noalloc: n outside [0, n_t)");
  auto al = [](const void* p) { return p && (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (!al(L) || !al(R) || !al(S_less) || !al(S_great) || !al(I_out))
    return fail(KBE_EINVAL, "kbe_history_slice_noalloc: NULL or misaligned device pointer");
  if (t[0] != 0.0) return fail(KBE_EINVAL, "kbe_history_slice_noalloc: t[0] must be 0");
  for (int l = 1; l < n_t; ++l) {
    if (!std::isfinite(t[l]) || !(t[l] > t[l - 1]))
      return fail(KBE_EINVAL, "kbe_history_slice_noalloc: t must be finite and strictly increasing");
    if (order[l] < 1 || order[l] > kMaxOrder)
      return fail(KBE_ERANGE, "kbe_history_slice_noalloc: order outside [1, 12]");
  }
  const int MM = norb * norb;
  const size_t row = (size_t)(n + 1) * MM;          // complex entries per s
  const size_t wdoubles = (size_t)n_t * (kMaxOrder + 2) + 64;  // wbar + band (+ status, padding)
  // the prep buffers (3 complex rows) must fit next to the weight tables
  if (wdoubles + 6 * row > kScratchDoubles)
    return fail(KBE_EINVAL, "kbe_history_slice_noalloc: (n+1)*norb^2 exceeds the 64 MiB scratch "
                            "(at most about 1.37e6 complex entries per row)");
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) return fail(KBE_ECUDA, "kbe_history_slice_noalloc: cudaGetSymbolAddress failed");
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(h_mutex);  // the host staging tables are shared
  std::string err;
  const int bw = host_weights(t, order, n_t, &err);
  if (bw == 0) return fail(KBE_EINVAL, "kbe_history_slice_noalloc: singular weight system");
  // layout: wbar [n_t] | band [n_t][bw] | status word | work (256-byte aligned)
  double* d_wbar = scratch;
  double* d_band = d_wbar + n_t;
  const size_t status_off = (size_t)n_t * (1 + bw);
  int* d_status = reinterpret_cast<int*>(scratch + status_off);
  const size_t used = (status_off + 1 + 31) / 32 * 32;
  double* d_work = scratch + used;
  // pageable host source: the copy is staged before cudaMemcpyAsync returns
  if ((e = cudaMemcpyAsync(d_wbar, h_wbar, n_t * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_band, h_band, (size_t)n_t * bw * sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(d_status, 0, sizeof(int), s)) != cudaSuccess)
    return fail(KBE_ECUDA, "kbe_history_slice_noalloc: staging the weight tables failed");
  HistoryArgs a{norb, n, (const double*)L, (const double*)R, (const double*)S_less, (const double*)S_great,
                WeightsView{d_wbar, d_band, bw}, (double*)I_out, d_work, (kScratchDoubles - used) * sizeof(double),
                d_status};
  int nl = 0;
  e = launch_history_f64(a, s, &nl);
  if (e != cudaSuccess) return fail(KBE_ECUDA, "kbe_history_slice_noalloc: launch failed");
  return KBE_OK;
}
