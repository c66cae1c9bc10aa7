// run_small.cu -- consecutive KBE steps of a small system in one cooperative
// launch (Sec. 3.1 with the grid's steps and orders, Eq. (SE), Eq. (KBE2)).
//
// A step of a small system (the dimer: M = 2, a few dozen rows) is a dozen
// kernels of a few microseconds of work each, and the device spends about as
// long between two dependent kernels as inside one.  This kernel runs the
// same work -- predictor, then P sweeps of {self-energy row, weight fold,
// history contraction, chunk sum, Fock matrix, right-hand side, corrector}
// -- for up to kRunMaxSteps consecutive rows, with device-wide barriers
// instead of kernel boundaries, seven per step of two sweeps: work that reads
// only what the same thread, or the same CTA before a block barrier, wrote
// shares a phase (see the kernel).  Measured on the 63-step dimer run:
// 2.55 ms against 5.46 ms for one kbe_step call per step; a barrier costs
// about 1.2 us, and each phase is a short per-thread chain of dependent
// loads and FP64 operations.  Every entry is computed by the per-entry
// functions of the single-step kernels (row_kernels.cuh) with
// the same arguments and the same split of the history index, so the rows,
// slices and ring are bitwise those of kbe_step.
//
// The barrier is a counter in global memory: each block's first thread adds
// one and waits, a bounded number of polls, until every block of the grid
// has arrived; a wait that runs out sets the timeout bit of the status word
// and the block leaves the kernel (the others then run out too).  All blocks
// are resident at once (cooperative launch, one block per SM).
// Data that other blocks rewrite during the launch is read with plain loads
// (ordered after the barrier's acquire), never through the read-only cache.

#include <algorithm>

#include "row_kernels.cuh"

namespace kbe {
namespace {

// The per-row data of one step (the rest is common to the run).
struct RunStep {
  int n, kn;             // row and its interval's order
  int chunk_len, nchunk; // split of the history index of the contraction
  double field;          // E(t_n)
};

struct RunSmallArgs {
  StepArgs base;         // the step arguments common to the rows (n, kn, field, corr, pred per row)
  const double* Sl;      // self-energy row buffers [n_max][M][M]
  const double* Sg;
  double* Sl_w;
  double* Sg_w;
  double* I;             // history slice [2][n+1][M][M]
  WeightsView w;
  double* part;          // workspace: A1 | Bl | Bg | chunk partials
  const double* corr0;   // stepper weight tables of row 0 ([n_max][kMaxOrder][kWTab])
  const double* pred0;
  unsigned* bar;         // barrier counter, zero at launch
  long long spin;        // polls of a barrier wait before it gives up
  int withhold;          // barrier at which block 0 leaves without arriving (failure-path test), or -1
  int P, nsteps;
  RunStep step[kRunMaxSteps];
};

// Device-wide barrier number `k` (0, 1, ...) of the launch.  The block's
// first thread arrives with a release add (the block's writes of the phase,
// ordered before it by the block barrier, become visible with it) and polls
// with acquire loads until every block has arrived.  Returns false when the
// wait ran out (status bit set); the caller then leaves the kernel.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned k, int* status, long long limit,
                                             int withhold) {
  if ((int)k == withhold && blockIdx.x == 0) return false;  // the whole block leaves; the others' waits run out
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    const unsigned target = (k + 1) * gridDim.x;
    unsigned cur;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(cur) : "l"(bar) : "memory");
    ++cur;  // the count with this block's arrival
    long long it = 0;
    while (cur < target) {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(bar) : "memory");
      if (++it > limit) {
        atomicOr(status, kStatusTimeout);
        ok = 0;
        break;
      }
      if (it > 256) __nanosleep(64);
    }
  }
  return __syncthreads_and(ok) != 0;
}

__device__ __forceinline__ StepArgs row_args(const RunSmallArgs& a, int st) {
  const RunStep& r = a.step[st];
  StepArgs sa = a.base;
  sa.n = r.n;
  sa.kn = r.kn;
  sa.field = r.field;
  sa.corr = a.corr0 + (size_t)r.n * kMaxOrder * kWTab;
  sa.pred = a.pred0 + (size_t)r.n * kMaxOrder * kWTab;
  return sa;
}

// Phases of a step, separated by device-wide barriers (4 in the first sweep,
// 3 in each later one):
//   A  self-energy row n, its weight fold (a thread folds the entries it
//      has just written) and the Fock matrix (reads only the diagonal block
//      of row n); in the sweeps after the first, A shares a phase with the
//      previous sweep's corrector D, separated by a block barrier: a block's
//      span of row entries is a whole number of M x M blocks, so the entries
//      that the self-energy and the Fock matrix read (an entry, the
//      transposed entry of the diagonal block, the diagonal block itself)
//      were corrected by the same CTA;
//   B  history partials, chunk by chunk of the history index;
//   C  chunk sum of one component (I^< or I^>) of an entry, then that
//      component of the entry's right-hand side (which reads only that sum);
//   D  corrector; after the last sweep also the predictor of the next row of
//      the launch: entry (c, ab) of row n+1 reads the entry (c, ab) of row n
//      that the same thread has just corrected, and the new diagonal entry
//      (n+1, ab) is taken by the thread of (n, ab), whose corrected value it
//      reads.
// The first step of a launch starts with its own predictor phase.
// Work items [0, total) of a phase: block b takes the contiguous span
// [b per, (b+1) per), per = ceil(total / blocks), its threads consecutive
// items of it, so a small row's items are spread over every SM and packed
// into as few warps of each as they fill.  (A phase is bound by its longest
// per-thread chain of dependent loads and FP64 operations; spreading a
// block's items over all eight of its warps was measured 1.3x slower in the
// contraction phase.)
struct Span {
  int64_t lo, hi;  // this thread's first item, the end of the block's span
  int64_t base;    // the block's first item
};
__device__ __forceinline__ Span span(int64_t total) {
  const int64_t per = rk::div_idx(total + gridDim.x - 1, (int)gridDim.x);
  const int64_t lo = (int64_t)blockIdx.x * per;
  return Span{lo + threadIdx.x, min(total, lo + per), lo};
}
// ... with per rounded up to a multiple of `unit` (row entries: whole M x M blocks)
__device__ __forceinline__ Span span_units(int64_t total, int unit) {
  const int64_t per = (int64_t)rk::div_idx(rk::div_idx(total + gridDim.x - 1, (int)gridDim.x) + unit - 1, unit) * unit;
  const int64_t lo = (int64_t)blockIdx.x * per;
  return Span{lo + threadIdx.x, min(total, lo + per), lo};
}

__global__ void __launch_bounds__(kRunThreads, 2) run_small_kernel(const __grid_constant__ RunSmallArgs a) {
  const int M = a.base.M, MM = M * M;
  const int64_t bs = blockDim.x;
  int* status = a.base.status;
  unsigned k = 0;  // barriers passed
  bool ok = true;  // no non-finite value met by this thread
  for (int st = 0; st < a.nsteps; ++st) {
    const RunStep& r = a.step[st];
    const int n = r.n;
    const int64_t row = (int64_t)(n + 1) * MM;  // complex entries of row n per component
    if (st == 0) {
      const StepArgs sa = row_args(a, st);
      const Span sp = span_units(row, MM);
      for (int64_t lin = sp.lo; lin < sp.hi; lin += bs) rk::adams_entry(sa, lin, false);
      if (!grid_barrier(a.bar, k++, status, a.spin, a.withhold)) return;
    }
    const int64_t off = (int64_t)tri(n, 0) * MM;
    const double2* Lr = reinterpret_cast<const double2*>(a.base.L) + off;
    const double2* Rr = reinterpret_cast<const double2*>(a.base.R) + off;
    double* A1 = a.part;
    double* Bl = A1 + 2 * row;
    double* Bg = Bl + 2 * row;
    double* partials = Bg + 2 * row;
    rk::PartialArgs p{M, MM, n, r.chunk_len, a.base.L, a.base.R, a.Sl, a.Sg, A1, Bl, Bg, a.w,
                      r.nchunk == 1 ? a.I : partials};
    const bool next = st + 1 < a.nsteps;
    const Span sr = span_units(row, MM);
    // A: self-energy row n (Eq. SE; the diagonal block is block n of the
    // row), weight fold of the same entries, Fock matrix (by the block whose
    // span holds the diagonal block)
    auto phase_a = [&]() {
      for (int64_t e = sr.lo; e < sr.hi; e += bs) {
        const int blk = rk::div_idx(e, MM), ab = (int)(e - (int64_t)blk * MM);
        ok &= rk::sigma_entry(M, e, ab, blk == n, rk::sigma_uu(M, ab, a.base.U), Lr, Rr,
                              reinterpret_cast<double2*>(a.Sl_w), reinterpret_cast<double2*>(a.Sg_w));
        rk::history_prep_entry(MM, n, e, a.Sl, a.Sg, a.w, A1, Bl, Bg);
      }
      if (sr.base <= row - MM && row - MM < sr.hi) {
        // threads from the top of the block: those past the span's entries
        // run it alongside the self-energy instead of after it
        const StepArgs sa = row_args(a, st);
        for (int ab = (int)blockDim.x - 1 - (int)threadIdx.x; ab < MM; ab += blockDim.x) rk::fock_entry(sa, ab);
      }
    };
    for (int it = 0; it < a.P; ++it) {
      if (it == 0) {
        phase_a();
        if (!grid_barrier(a.bar, k++, status, a.spin, a.withhold)) return;
      }
      // B: history slice of row n (Eq. KBE2), chunk by chunk of the history index
      const Span sq = span(row * r.nchunk);
      for (int64_t q = sq.lo; q < sq.hi; q += bs) {
        const int chunk = rk::div_idx(q, (int)row);
        rk::history_partial_entry<false>(p, q - (int64_t)chunk * row, chunk);
      }
      if (!grid_barrier(a.bar, k++, status, a.spin, a.withhold)) return;
      // C: chunk sum of one component of an entry, then that component's F
      const Span sc = span(2 * row);
      for (int64_t u = sc.lo; u < sc.hi; u += bs) {
        const StepArgs sa = row_args(a, st);
        if (r.nchunk > 1) {
          ok &= rk::history_reduce_entry(2 * row, r.nchunk, u, reinterpret_cast<const double2*>(partials),
                                         reinterpret_cast<double2*>(a.I));
        } else {
          const double2 x = reinterpret_cast<const double2*>(a.I)[u];
          ok &= isfinite(x.x) && isfinite(x.y);
        }
        const int comp = u >= row ? 1 : 0;
        ok &= rk::rhs_entry_s(sa, u - comp * row, comp);
      }
      if (!grid_barrier(a.bar, k++, status, a.spin, a.withhold)) return;
      // D: corrector, then the next sweep's A after a block barrier, or after
      // the last sweep the next row's predictor
      const bool pred_next = next && it == a.P - 1;
      for (int64_t lin = sr.lo; lin < sr.hi; lin += bs) {
        rk::adams_entry(row_args(a, st), lin, true);
        if (pred_next) {
          const StepArgs sn = row_args(a, st + 1);
          rk::adams_entry(sn, lin, false);
          if (lin >= row - MM) rk::adams_entry(sn, lin + MM, false);
        }
      }
      if (it + 1 < a.P) {
        __syncthreads();  // the CTA's corrected entries are visible to all of its threads
        phase_a();
      }
      if (!grid_barrier(a.bar, k++, status, a.spin, a.withhold)) return;
    }
  }
  if (!ok) atomicOr(status, kStatusNumeric);
}

}  // namespace

// Host side: one cooperative launch for the steps args.step[0..nsteps).
cudaError_t launch_run_small(const RunSmallHost& h, cudaStream_t s, int* launches) {
  *launches = 0;
  static int blocks_per_sm = 0;  // the kernel's occupancy (the same on every device of a build)
  if (blocks_per_sm == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, run_small_kernel, kRunThreads, 0);
    if (e != cudaSuccess || blocks_per_sm < 1) return e != cudaSuccess ? e : cudaErrorInvalidConfiguration;
  }
  RunSmallArgs a{};
  a.base = h.base;
  a.Sl = h.Sl;
  a.Sg = h.Sg;
  a.Sl_w = h.Sl;
  a.Sg_w = h.Sg;
  a.I = h.I;
  a.w = h.w;
  a.part = h.part;
  a.corr0 = h.corr0;
  a.pred0 = h.pred0;
  a.bar = h.bar;
  a.spin = h.spin;
  a.withhold = h.withhold;
  a.P = h.P;
  a.nsteps = h.nsteps;
  for (int i = 0; i < h.nsteps; ++i)
    a.step[i] = RunStep{h.n[i], h.kn[i], h.chunk_len[i], h.nchunk[i], h.field[i]};
  // one block per SM (the phases' spans spread the FP64 work over all of them)
  const int grid = std::min(blocks_per_sm, 1) * sm_count();
  cudaError_t e = cudaMemsetAsync(h.bar, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  void* params[] = {&a};
  e = cudaLaunchCooperativeKernel((const void*)run_small_kernel, dim3((unsigned)grid), dim3(kRunThreads), params, 0, s);
  if (e == cudaSuccess) *launches = 1;
  return e;
}

}  // namespace kbe
