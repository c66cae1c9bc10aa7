// history_f64.cu -- FP64 history slice of Eq. (KBE2) (Sec. 2).
//
//   I^s(n,c) = sum_{m<=n} w_{n,m} Sigma^R(n,m) G^s(m,c)
//            + sum_{m<=c} w_{c,m} Sigma^s(n,m) G^A(m,c),      s in {<,>}
//
// with Sigma^R(n,m) = S^>(n,m) - S^<(n,m) (theta(0) = 1), G^A(m,c) =
// R(c,m)^+, and G^s(m,c) = -G^s(c,m)^+ above the diagonal (Sec. 2).
//
// GB300 design notes.  FP64 on this part runs at about 2 DFMA per clock per
// SM (1.2 TFLOP/s measured for the whole GPU; FP64 mma.sync measured lower,
// 1.05 TFLOP/s), so the contraction is bound by the FP64 pipe at every
// orbital count: 48 M^3 flops per 32 M^2 bytes of history is 1.5 M flop/B,
// far above the 0.18 flop/B balance point of 1.2 TFLOP/s over 6.8 TB/s.
// The kernel therefore spends its FP64 issue slots on complex multiply-adds
// only:
//   * a prep pass folds the weights into the self-energy row once:
//       A1[m] = w_{n,m} (S^> - S^<)[m]          (term 1, all m)
//       B^s[m] = wbar_m S^s[m]                    (term 2, settled weights)
//     so the main loop holds no weight products except in the K+1 band
//     points next to the diagonal, where w_{c,m} still differs from wbar_m;
//   * term 1 is split as A1 G^> = A1 G^< + A1 G^R (no G^< + G^R sums);
//   * one thread owns one output entry (c, a, b) for both s, with four
//     independent complex accumulators (8 FMA chains);
//   * the history index m is split into chunks across grid.y; partial sums
//     go to a workspace and a second kernel adds them in a fixed order, so
//     results are bitwise reproducible.
// Operands are read through the read-only path; a block of G is reused M
// times from L1 (once per a), the self-energy row stays L2-resident.

#include <algorithm>
#include <cmath>

#include "row_kernels.cuh"

namespace kbe {
namespace {

using rk::PartialArgs;

constexpr int kHistBlock = 128;  // threads per block of the contraction

__global__ void __launch_bounds__(256) history_prep(int MM, int n, const double* __restrict__ Sl,
                                                    const double* __restrict__ Sg, WeightsView w,
                                                    double* __restrict__ A1, double* __restrict__ Bl,
                                                    double* __restrict__ Bg) {
  const int64_t total = (int64_t)(n + 1) * MM;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    rk::history_prep_entry(MM, n, e, Sl, Sg, w, A1, Bl, Bg);
}

// Output entries lin in [lin0, lin_end) (whole columns: lin = c M^2 + a M + b).
// Blocks take the columns from the last one down: within a chunk of the
// history index, the columns past the chunk carry both terms of Eq. (KBE2)
// and the ones before it term 1 only, so the launch order (x fastest) puts
// the heavier blocks of each chunk first and the last wave holds light ones.
__global__ void __launch_bounds__(256) history_partial(PartialArgs p, int64_t lin0, int64_t lin_end) {
  const int64_t lin = lin0 + (int64_t)(gridDim.x - 1 - blockIdx.x) * blockDim.x + threadIdx.x;
  if (lin >= lin_end) return;
  rk::history_partial_entry(p, lin, blockIdx.y);
}

// out = sum over chunks in order; flags non-finite results.
__global__ void __launch_bounds__(256) history_reduce(int64_t per_chunk, int nchunk, const double2* __restrict__ part,
                                                      double2* __restrict__ out, int* status) {
  bool ok = true;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < per_chunk;
       e += (int64_t)gridDim.x * blockDim.x)
    ok &= rk::history_reduce_entry(per_chunk, nchunk, e, part, out);
  if (!ok) atomicOr(status, kStatusNumeric);
}

__global__ void __launch_bounds__(256) finite_check(int64_t n, const double2* __restrict__ v, int* status) {
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 x = v[e];
    bad |= !(isfinite(x.x) && isfinite(x.y));
  }
  if (bad) atomicOr(status, kStatusNumeric);
}

inline unsigned grid_for(int64_t n, int64_t cap) {
  int64_t b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

// Split of the history index m of the FP64 slice of row n: at least enough
// threads for full occupancy (every SM x 2048 threads), and chunks short
// enough that one 128-thread block does about 2^16 complex multiply-adds
// (3M per point and output), which keeps the tail of the launch short; the
// partials must fit the workspace.  A band of stored rows below n
// contributes only history points m < band_hi: the chunks beyond them have
// no work.  False when even one chunk does not fit.
//
// Rows of at most kRunMaxRow entries are latency-bound: a phase lasts as
// long as its longest per-thread chain of dependent loads and FP64
// operations (the FP64 pipe measured 6% busy over the small-row run kernel).
// Measured on the dimer's rows: about 1.7 M us per history point of a chunk
// in the contraction and 0.075 us per chunk in the chunk sum, so the chunk
// length that minimises the two together, about sqrt((n+1) / (24M)) points,
// is taken (chunks of 1, 2 and 4 points at n = 63, M = 2: whole run 2.43,
// 2.50 and 2.65 ms), with up to
// kMaxSplitSmall chunks while the items stay within one per thread of one
// 256-thread block per SM (kbe_step and the cooperative run kernel of
// kbe_run_steps take the same split).
bool history_f64_split(int M, int n, size_t part_bytes, int band_hi, int* nchunk_out, int* chunk_len_out) {
  const int64_t row = (int64_t)(n + 1) * M * M;
  int64_t want = ((int64_t)sm_count() * 2048 + row - 1) / row;
  const int64_t len_target = std::max<int64_t>(1, (1 << 16) / (kHistBlock * 3 * M));
  want = std::max<int64_t>(want, (n + 1 + len_target - 1) / len_target);
  int nchunk = (int)(want < 1 ? 1 : (want > kMaxSplit ? kMaxSplit : want));
  if (row <= kRunMaxRow) {
    const int len = std::max(1, (int)std::lround(std::sqrt((n + 1) / (24.0 * M))));
    const int64_t cap = std::max<int64_t>(kMaxSplit, (int64_t)sm_count() * 256 / row);
    nchunk = (int)std::min<int64_t>(std::min<int64_t>((n + 1 + len - 1) / len, cap), kMaxSplitSmall);
  }
  if (nchunk > n + 1) nchunk = n + 1;
  const size_t prep_bytes = (size_t)3 * row * 16;
  while (nchunk > 1 && prep_bytes + (size_t)nchunk * 2 * row * 16 > part_bytes) --nchunk;
  if (prep_bytes + (nchunk > 1 ? (size_t)nchunk * 2 * row * 16 : 0) > part_bytes) return false;
  const int chunk_len = (n + 1 + nchunk - 1) / nchunk;
  nchunk = (n + 1 + chunk_len - 1) / chunk_len;
  if (band_hi <= n) nchunk = std::max(1, std::min(nchunk, (band_hi + chunk_len - 1) / chunk_len));
  *nchunk_out = nchunk;
  *chunk_len_out = chunk_len;
  return true;
}

// Workspace layout (doubles): A1, Bl, Bg: 3 x (n+1) MM complex; then the
// split partials nchunk x 2 x (n+1) MM complex.  The output columns may be
// contracted in several launches (column ranges, each after an optional
// event, e.g. the arrival of the history rows it reads); every entry is
// computed by the same thread arithmetic whatever the ranges, so the
// results are bitwise those of one launch.
cudaError_t launch_history_f64_ranges(const HistoryArgs& a, int nranges, const int* c_lo, const int* c_hi,
                                      const cudaEvent_t* wait, cudaStream_t s, int* launches) {
  const int M = a.M, MM = M * M, n = a.n;
  const int64_t row = (int64_t)(n + 1) * MM;       // complex entries per s
  int nchunk = 0, chunk_len = 0;
  if (!history_f64_split(M, n, a.part_bytes, a.band_hi, &nchunk, &chunk_len)) return cudaErrorInvalidValue;

  double* A1 = a.part;
  double* Bl = A1 + 2 * row;
  double* Bg = Bl + 2 * row;
  double* partials = Bg + 2 * row;
  int nl = 0;
  history_prep<<<grid_for(row, sm_count() * 8), 256, 0, s>>>(MM, n, a.Sl, a.Sg, a.w, A1, Bl, Bg);
  ++nl;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { *launches = nl; return e; }
  PartialArgs p{M, MM, n, chunk_len, a.L, a.R, a.Sl, a.Sg, A1, Bl, Bg, a.w,
                nchunk == 1 ? a.out : partials};
  p.band_lo = a.band_lo;
  p.band_hi = a.band_hi;
  if (a.ev_begin) cudaEventRecord(a.ev_begin, s);
  for (int k = 0; k < nranges; ++k) {
    const int lo = std::max(0, c_lo[k]), hi = std::min(n + 1, c_hi[k]);
    if (wait && wait[k] && (e = cudaStreamWaitEvent(s, wait[k], 0)) != cudaSuccess) break;
    if (hi <= lo) continue;
    const int64_t lin0 = (int64_t)lo * MM, lin_end = (int64_t)hi * MM;
    dim3 grid((unsigned)((lin_end - lin0 + kHistBlock - 1) / kHistBlock), (unsigned)nchunk);
    history_partial<<<grid, kHistBlock, 0, s>>>(p, lin0, lin_end);
    ++nl;
    if ((e = cudaGetLastError()) != cudaSuccess) break;
  }
  if (a.ev_end) cudaEventRecord(a.ev_end, s);
  if (e != cudaSuccess) { *launches = nl; return e; }
  if (nchunk > 1) {
    history_reduce<<<grid_for(2 * row, sm_count() * 8), 256, 0, s>>>(2 * row, nchunk, (const double2*)partials,
                                                              (double2*)a.out, a.status);
  } else {
    finite_check<<<grid_for(2 * row, sm_count() * 8), 256, 0, s>>>(2 * row, (const double2*)a.out, a.status);
  }
  ++nl;
  *launches = nl;
  return cudaGetLastError();
}

// The last kernel of a split slice: partials [nchunk][2][row] summed in
// chunk order into out (or, for one chunk, out checked for finite values).
cudaError_t launch_history_finish(int nchunk, int64_t row, const double* partials, double* out, int* status,
                                  cudaStream_t s, int* launches) {
  if (nchunk > 1) {
    history_reduce<<<grid_for(2 * row, sm_count() * 8), 256, 0, s>>>(2 * row, nchunk, (const double2*)partials,
                                                              (double2*)out, status);
  } else {
    finite_check<<<grid_for(2 * row, sm_count() * 8), 256, 0, s>>>(2 * row, (const double2*)out, status);
  }
  *launches = 1;
  return cudaGetLastError();
}

cudaError_t launch_history_f64(const HistoryArgs& a, cudaStream_t s, int* launches) {
  const int lo = 0, hi = a.n + 1;
  return launch_history_f64_ranges(a, 1, &lo, &hi, nullptr, s, launches);
}

}  // namespace kbe
