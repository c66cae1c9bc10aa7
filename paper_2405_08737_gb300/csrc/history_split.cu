// history_split.cu -- split-precision history slice of Eq. (KBE2) on tcgen05.
//
// The same contraction as history_f64.cu,
//   I^s(n,c) = sum_m w_{n,m} Sigma^R(n,m) G^s(m,c) + sum_{m<=c} w_{c,m} Sigma^s(n,m) G^A(m,c),
// evaluated on the fp16 tensor cores with error-free fixed-point slicing
// (split_common.cuh): every operand becomes four 8-bit digits, each
// tensor-core sum is exact in FP32, and the per-chunk scales are applied in
// double-float arithmetic on the FP32 pipe.  No FP64 instruction touches the
// O(n^2 M^3) part; the result matches FP64 to about 1e-9 relative.
//
// Real-GEMM form.  Write term 1 with the full-plane values of G (both
// triangles through G(m,c) = -G(c,m)^+) and term 2 with
// G^A(m,c) = R(c,m)^+ = -Q(m,c) for m <= c, where the plane Q(m,c) = R(m,c)
// below and on the diagonal and -R(c,m)^+ above it (R(c,c) = -i*1 makes both
// readings agree on the diagonal).  With A1[m] = w_{n,m}(S^> - S^<)[m],
// NB^<[m] = -wbar_m S^<[m] and NBD[m] = -wbar_m (S^> - S^<)[m] (settled
// weights), the tensor cores form
//   I^<[c]          = sum_m A1[m] PL(m,c) + sum_{m<=c} NB^<[m] Q(m,c)
//   D[c] = (I^> - I^<)[c] = sum_m A1[m] Q(m,c) + sum_{m<=c} NBD[m] Q(m,c)
// (G^> - G^< = G^R gives the difference without a second PL product), and
// the reduction adds I^> = I^< + D.
// For one output tile (128 rows j = (c,b)) and one chunk of 16 complex K
// entries (m,x), the big operands are the plane tiles PL, Q and the masked
// QU = Q [m <= c]; the small operands A1, NB^<, NBD (prepared once per
// slice) are the "B" matrices of the MMA.  Term 2 for the band m > c - K,
// where w_{c,m} still differs from wbar_m, is left out of QU and added with
// the exact weights in double-float by the reduction kernel.
//
// Two forms of the contraction share the prep and reduction kernels.  The
// planes path (one system, with a buffer that keeps every unit's digit
// planes between slices) streams the encoded units into the tensor-core
// kernel; the fused path (batches, or no buffer) converts the FP64 history
// inside the tensor-core kernel.  Both are persistent (one CTA per SM) over
// contiguous ranges of (column tile, chunk) units, with the roles and
// buffers described at each kernel.  All mbarrier waits are bounded; a wait
// that runs out sets the status word and every role leaves its loop.

#include <atomic>
#include <cstdio>

#include "dfloat.cuh"
#include "kbe_internal.h"
#include "split_common.cuh"

namespace kbe {
namespace {

using namespace split;

constexpr int kConvThreads = 256;        // threads that convert FP64 history rows into digit planes
constexpr int kKC = 16;                     // complex K entries per chunk (32 real)
constexpr int kNS = 16;                     // small-operand columns per slice: 8 a x (re, im)
constexpr int kNA = 8;                      // a values per part
constexpr int kBigSlice = 128 * 2 * kKC * 2;          // bytes of one digit plane: 128 rows x 32 fp16
constexpr int kBigTile = kSlices * kBigSlice;         // 32 KB
constexpr int kSmallVar = 4 * kSlices * 2 * 128;      // 4 kgroups x 4 slices x 2 colgroups x 128 B = 4 KB
constexpr int kSmallBytes = 3 * kSmallVar;            // 12 KB
constexpr int kStages = 2;
constexpr int kGroupCols = kLevels * kNS;   // 5 levels x 16 columns
constexpr int kAccCols = 2 * kGroupCols;    // groups I^< and I^>: 160 columns
constexpr int kTmemCols = 512;              // two accumulator buffers (320 used)
constexpr long long kSpinLimit = 1ll << 26; // bounded waits
constexpr int kMaxSplitCtas = 160;          // persistent CTAs of a contraction, at most
constexpr int kSlotComplex = 2 * 128 * 8;   // one partial slot: [group][c_l][a_l < 8][b], CT M <= 128

struct SplitGeom {
  int M, MM, n;
  int CT;          // columns per tile
  int parts;       // a-ranges of 8
  int cpt;         // chunks per tile
  int tiles;       // column tiles x parts
  long long U;     // total units
  int G;           // CTAs
  int S;           // partial slots per CTA
  int band_w;      // composite-weight band width (K+1)
};

// ---------------------------------------------------------------- prep ---
// Small operands of chunk kc, part p: A1, NB^<, NBD as fp16 digit planes in
// the shared-memory layout [variant][kgroup 4][slice 4][colgroup 2][8][8],
// entries B[(a, q_out)][(kappa, q_in)] of the real form of P z:
//   (re,re) = P.re, (re,im) = -P.im, (im,re) = P.im, (im,im) = P.re.
__device__ __forceinline__ void prep_chunk(int M, int n, int parts, const double* __restrict__ Sl,
                                           const double* __restrict__ Sg, const WeightsView& w,
                                           uint8_t* __restrict__ small, int* __restrict__ e_small, int kc, int p,
                                           int* s_ef) {
  const int MM = M * M;
  if (threadIdx.x == 0) *s_ef = 0;
  __syncthreads();
  // 3 variants x 16 kappa x 8 a: 384 complex values, 2 per thread (256 threads -> 512 slots)
  double vr[2], vi[2];
  int my_ef = 0;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int idx = threadIdx.x + 256 * r;  // (v, kl, al)
    vr[r] = 0.0; vi[r] = 0.0;
    if (idx < 3 * kKC * kNA) {
      const int v = idx / (kKC * kNA), kl = (idx / kNA) % kKC, al = idx % kNA;
      const int kappa = kc * kKC + kl;
      const int m = kappa / M, x = kappa - m * M;
      const int a = p * kNA + al;
      if (m <= n && a < M) {
        const double2 l = reinterpret_cast<const double2*>(Sl)[(size_t)m * MM + a * M + x];
        const double2 g = reinterpret_cast<const double2*>(Sg)[(size_t)m * MM + a * M + x];
        if (v == 0) {
          const double wn = w.at(n, m);
          vr[r] = wn * (g.x - l.x); vi[r] = wn * (g.y - l.y);
        } else if (v == 1) {
          const double wb = -w.wbar[m];
          vr[r] = wb * l.x; vi[r] = wb * l.y;
        } else {
          const double wb = -w.wbar[m];
          vr[r] = wb * (g.x - l.x); vi[r] = wb * (g.y - l.y);
        }
      }
      my_ef = max(my_ef, max(exp_field(vr[r]), exp_field(vi[r])));
    }
  }
  my_ef = __reduce_max_sync(0xffffffffu, my_ef);
  if ((threadIdx.x & 31) == 0) atomicMax(s_ef, my_ef);
  __syncthreads();
  const int e = scale_from_field(*s_ef);
  uint8_t* out = small + ((size_t)kc * parts + p) * kSmallBytes;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int idx = threadIdx.x + 256 * r;
    if (idx >= 3 * kKC * kNA) continue;
    const int v = idx / (kKC * kNA), kl = (idx / kNA) % kKC, al = idx % kNA;
    int dr[kSlices], di[kSlices];
    digits(vr[r], e, dr);
    digits(vi[r], e, di);
    const int k = 2 * kl;            // even real K index (re), k+1 (im)
    const int kg = k >> 3, kin = k & 7;
#pragma unroll
    for (int sl = 0; sl < kSlices; ++sl) {
      const uint32_t pr = f16_of_int(dr[sl]), pi = f16_of_int(di[sl]), npi = f16_of_int(-di[sl]);
      // column (al, re): (P.re, -P.im); column (al, im): (P.im, P.re)
      const int col_re = 2 * al, col_im = 2 * al + 1;
      uint8_t* base = out + v * kSmallVar + ((kg * kSlices + sl) * 2) * 128;
      uint32_t* pre = reinterpret_cast<uint32_t*>(base + (col_re >> 3) * 128 + (col_re & 7) * 16 + kin * 2);
      uint32_t* pim = reinterpret_cast<uint32_t*>(base + (col_im >> 3) * 128 + (col_im & 7) * 16 + kin * 2);
      *pre = pack2(pr, npi);
      *pim = pack2(pi, pr);
    }
  }
  if (threadIdx.x == 0) e_small[kc * parts + p] = e;
}

__global__ void __launch_bounds__(256) split_prep(int M, int n, int parts, const double* __restrict__ Sl,
                                                  const double* __restrict__ Sg, WeightsView w,
                                                  uint8_t* __restrict__ small, int* __restrict__ e_small) {
  __shared__ int s_ef;
  prep_chunk(M, n, parts, Sl, Sg, w, small, e_small, blockIdx.x, blockIdx.y, &s_ef);
}

// ---------------------------------------------------------------- main ---
__device__ __forceinline__ long long unit_begin(const SplitGeom& g, int cta) { return g.U * cta / g.G; }

// AND of a predicate over the converter warps (named barrier 1); every
// converter thread must call it at the same point.
template <int NT = kConvThreads>
__device__ __forceinline__ bool conv_all(bool ok) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.and.pred q, 1, %2, p;\nselp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)ok), "r"(NT)
      : "memory");
  return r != 0;
}

// ecol[col] = max(ecol[col], ef) for every lane of the warp, with one shared
// atomic per distinct column of the warp (lanes of one column reduce first;
// a per-lane atomic serializes on the lanes that share an address).  Every
// lane of the warp must call it; lanes with live == false contribute nothing.
__device__ __forceinline__ void column_max(int* ecol, int col, int ef, bool live) {
  const unsigned grp = __match_any_sync(0xffffffffu, live ? col : -1);
  const int m = __reduce_max_sync(grp, live ? ef : 0);
  if (live && m > 0 && (threadIdx.x & 31) == __ffs(grp) - 1) atomicMax(&ecol[col], m);
}

// Chunk class relative to the tile's column range [c0, c1]: term 2 of the
// tensor-core part covers m <= c - band_w (QU = Q there, 0 elsewhere).
// 0: QU = 0 for every (m, c) of the chunk; 1: QU = Q for all; 2: mixed.
__device__ __forceinline__ int chunk_class(int m_lo, int m_hi, int c0, int c1, int band_w) {
  if (m_lo > c1 - band_w) return 0;
  if (m_hi <= c0 - band_w) return 1;
  return 2;
}

// ============================================================ planes path ==
// The same contraction with the conversion taken off the main kernel: an
// encoder kernel at full occupancy writes, per (column tile, chunk), the
// digit planes of PL and Q and the column exponents in exactly the
// shared-memory image the MMAs read (and QU for the chunks straddling the
// band), and the main kernel streams them in with bulk copies issued by one
// producer thread.  Eight epilogue warps drain the accumulators, four per
// accumulator group (I^< and I^>).

constexpr int kUnitBytes = 2 * kBigTile + 1024;                 // PL | Q | column exponents (padded)
constexpr int kStage2Bytes = kUnitBytes + kBigTile + kSmallBytes;  // + QU | small operand
constexpr int kEpi2 = 16;                                       // 4 lane quadrants x 2 groups x 2 column halves
constexpr int kThreads2 = (kEpi2 + 3) * 32;                     // + MMA warp, producer warp, second MMA warp

// Slot of a straddling chunk kc in the QU buffer of the tile starting at
// column c0 (the first straddling chunk is the first whose last point
// m_hi exceeds c0 - band_w).
__host__ __device__ __forceinline__ int qu_slot(int kc, int c0, int M, int band_w) {
  const int t = (c0 - band_w + 1) * M - 15;
  const int first = t <= 0 ? 0 : (t + 15) / 16;
  return kc - first;
}

struct EncodeArgs {
  SplitGeom g;
  const double* L;
  const double* R;
  uint8_t* planes;     // [column tile][cpt_stride][kUnitBytes]
  uint8_t* qu;         // [column tile][qu_slots][kBigTile]
  int cpt_stride, qu_slots;
  int ct_base, kc_base, kc_count;  // units: ct_base + i / kc_count, kc_base + i % kc_count
  int c_min;                       // only the columns c >= c_min are encoded
  int* status;
  // rows [row_lo, row_lo + rows) of each unit, upc units per CTA, units in
  // all (whole units: 0, 128, 1)
  int row_lo, rows, upc;
  unsigned units;
};
constexpr int kEncMaxUpc = 16;  // units per CTA of the encoder, at most

// Thread (arr, k, jrow) encodes row jrow of plane arr (0: G^< from L, 1: Q
// from R) for the 16 K entries of the CTA's k-th unit (column tile, chunk).
// Whole units take one CTA each (256 threads: rows 0..127 of both planes);
// a KBE step's new column takes its few rows of 16 units per CTA.  Every
// column has its own exponent, so the rows of the columns below c_min are
// left as they are.  Threads past the mapped ones (the block is a whole
// number of warps) only join the collective steps.  kNarrow: the general
// mapping (several units per CTA, a band of rows), at one CTA per SM's
// worth of registers; otherwise whole units at three CTAs per SM.
template <bool kNarrow>
__global__ void __launch_bounds__(256, kNarrow ? 1 : 3) split_encode(EncodeArgs a) {
  const SplitGeom& g = a.g;
  const int M = g.M, MM = g.MM, n = g.n, CT = g.CT;
  constexpr int kUpcMax = kNarrow ? kEncMaxUpc : 1;
  __shared__ int ecol[kUpcMax * 128];
  const int upc = kNarrow ? a.upc : 1, rows = kNarrow ? a.rows : 128;
  const int t = threadIdx.x, per = upc * rows;
  const int arr = kNarrow ? t / per : t >> 7;
  const int rem = t - arr * per, k = kNarrow ? rem / rows : 0;
  const int jrow = kNarrow ? a.row_lo + (rem - k * rows) : (t & 127);
  const unsigned ui = blockIdx.x * (unsigned)upc + (unsigned)k;
  const bool mapped = kNarrow ? (arr < 2 && ui < a.units) : true;
  const int ctile = a.ct_base + (int)(mapped ? ui / (unsigned)a.kc_count : 0u);
  const int kc = a.kc_base + (int)(mapped ? ui % (unsigned)a.kc_count : 0u);
  const bool row_live = mapped && jrow < CT * M;
  const int cl = row_live ? jrow / M : 0, bb = jrow - cl * M;
  const int c0 = ctile * CT;
  const int kap0 = kc * kKC;
  const int cls = chunk_class(kap0 / M, (kap0 + kKC - 1) / M, c0, c0 + CT - 1, g.band_w);
  for (int e = t; e < upc * 128; e += blockDim.x) ecol[e] = 0;
  __syncthreads();
  const double2* base = reinterpret_cast<const double2*>(arr == 0 ? a.L : a.R);
  const int c = c0 + cl;
  const bool enc = row_live && c >= a.c_min;
  const bool col_live = enc && c <= n;
  double er[kKC], ei[kKC];
  unsigned keep = 0;
  int ef = 0;
  {
    int m = kap0 / M, x = kap0 - m * M;
#pragma unroll
    for (int k = 0; k < kKC; ++k) {
      double2 z = make_double2(0.0, 0.0);
      if (col_live && m <= n) {
        if (m >= c) {
          z = __ldcs(base + tri(m, c) * MM + x * M + bb);
        } else {
          z = __ldcs(base + tri(c, m) * MM + bb * M + x);
          z.x = -z.x;  // -conj
        }
      }
      er[k] = z.x;
      ei[k] = z.y;
      keep |= (unsigned)(m <= c - g.band_w) << k;
      if (++x == M) { x = 0; ++m; }
    }
#pragma unroll
    for (int k = 0; k < kKC; ++k) ef = max(ef, max(exp_field(er[k]), exp_field(ei[k])));
  }
  column_max(ecol, k * 128 + cl, ef, enc);
  __syncthreads();
  uint8_t* unit = a.planes + ((size_t)ctile * a.cpt_stride + kc) * kUnitBytes;
  uint8_t* dst = unit + (arr & 1) * kBigTile;
  uint8_t* QU = nullptr;
  if (mapped && arr == 1 && cls == 2) {
    const int slot = qu_slot(kc, c0, M, g.band_w);
    if (slot >= 0 && slot < a.qu_slots) QU = a.qu + ((size_t)ctile * a.qu_slots + slot) * kBigTile;
    else if (jrow == a.row_lo) atomicOr(a.status, kStatusInternal);  // geometry error: reported, never written
  }
  const int e = scale_from_field(ecol[k * 128 + cl]);
#pragma unroll
  for (int kg = 0; kg < 4 && enc; ++kg) {
    uint32_t w[kSlices][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int Vr = fixed31_fast(er[4 * kg + q], e), Vi = fixed31_fast(ei[4 * kg + q], e);
      w[0][q] = digit_pair_f16<0>(Vr, Vi);
      w[1][q] = digit_pair_f16<1>(Vr, Vi);
      w[2][q] = digit_pair_f16<2>(Vr, Vi);
      w[3][q] = digit_pair_f16<3>(Vr, Vi);
    }
    const int off = (kg * 16 + (jrow >> 3)) * 128 + (jrow & 7) * 16;
#pragma unroll
    for (int sl = 0; sl < kSlices; ++sl) {
      *reinterpret_cast<uint4*>(dst + sl * kBigSlice + off) = make_uint4(w[sl][0], w[sl][1], w[sl][2], w[sl][3]);
      if (QU) {
        const unsigned kb = keep >> (4 * kg);
        *reinterpret_cast<uint4*>(QU + sl * kBigSlice + off) =
            make_uint4(kb & 1u ? w[sl][0] : 0u, kb & 2u ? w[sl][1] : 0u, kb & 4u ? w[sl][2] : 0u,
                       kb & 8u ? w[sl][3] : 0u);
      }
    }
  }
  // exponents of the encoded columns (and the padding beyond the tile's CT)
  for (int e2 = t; e2 < upc * 128; e2 += blockDim.x) {
    const int k2 = e2 >> 7, col = e2 & 127;
    const unsigned u2 = blockIdx.x * (unsigned)upc + (unsigned)k2;
    if (u2 >= a.units) break;
    const int ct2 = a.ct_base + (int)(u2 / (unsigned)a.kc_count), kc2 = a.kc_base + (int)(u2 % (unsigned)a.kc_count);
    if (ct2 * CT + col >= a.c_min)
      reinterpret_cast<int*>(a.planes + ((size_t)ct2 * a.cpt_stride + kc2) * kUnitBytes + 2 * kBigTile)[col] =
          ecol[e2];
  }
}

struct Smem2 {
  uint8_t stage[kStages][kStage2Bytes];
  uint64_t full[kStages], empty[kStages], accfull[2], accempty[2];
  uint64_t mmadone[2];  // one per MMA-issuing thread: all of its MMAs have completed
  uint32_t tmem;
  int abort;
};

struct Split2Args {
  SplitGeom g;
  const uint8_t* planes;
  const uint8_t* qu;
  int cpt_stride, qu_slots;
  const uint8_t* small;
  const int* e_small;
  double* part;
  int* status;
  // failure-path test: the producer issues nothing for unit `withhold` (or
  // later) and every work wait gives up after `spin` polls; the final waits
  // for copies and MMAs already issued keep the full limit
  long long withhold;
  long long spin;
};

__device__ __forceinline__ bool wait_bar2(Smem2& sm, void* bar, uint32_t parity, int* status, long long limit) {
  long long it = 0;
  while (!mbar_try(bar, parity)) {
    if (++it > limit || *(volatile int*)&sm.abort) {
      if (it > limit) { atomicOr(status, kStatusTimeout); sm.abort = 1; }
      return false;
    }
    if (it > 64) __nanosleep(64);
  }
  return true;
}

// Where unit u = tile * cpt + kc sits (tile = column tile * parts + part),
// advanced one unit at a time so that no role divides per unit: the chunk's
// first and last history points m_lo = 16 kc / M, m_hi = (16 kc + 15) / M
// with their remainders, and the first QU slot of the column tile.
struct UnitCur {
  int kc, ctile, part, c0, qfirst;
  int m_lo, r_lo, m_hi, r_hi;
};
__device__ __forceinline__ int qu_first(int c0, int M, int band_w) { return -qu_slot(0, c0, M, band_w); }
__device__ __forceinline__ UnitCur unit_cur(const SplitGeom& g, long long u) {
  UnitCur c;
  const int tile = (int)(u / g.cpt);
  c.kc = (int)(u - (long long)tile * g.cpt);
  c.ctile = tile / g.parts;
  c.part = tile - c.ctile * g.parts;
  c.c0 = c.ctile * g.CT;
  c.qfirst = qu_first(c.c0, g.M, g.band_w);
  const int k0 = c.kc * kKC, k1 = k0 + kKC - 1;
  c.m_lo = k0 / g.M;
  c.r_lo = k0 - c.m_lo * g.M;
  c.m_hi = k1 / g.M;
  c.r_hi = k1 - c.m_hi * g.M;
  return c;
}
// q16 = 16 / M and r16 = 16 % M of the launch
__device__ __forceinline__ void unit_next(const SplitGeom& g, UnitCur& c, int q16, int r16) {
  if (++c.kc == g.cpt) {
    c.kc = 0;
    c.m_lo = 0;
    c.r_lo = 0;
    c.m_hi = (kKC - 1) / g.M;
    c.r_hi = (kKC - 1) - c.m_hi * g.M;
    if (++c.part == g.parts) {
      c.part = 0;
      ++c.ctile;
      c.c0 += g.CT;
      c.qfirst = qu_first(c.c0, g.M, g.band_w);
    }
    return;
  }
  c.m_lo += q16;
  c.r_lo += r16;
  if (c.r_lo >= g.M) { c.r_lo -= g.M; ++c.m_lo; }
  c.m_hi += q16;
  c.r_hi += r16;
  if (c.r_hi >= g.M) { c.r_hi -= g.M; ++c.m_hi; }
}

__global__ void __launch_bounds__(kThreads2, 1) split_main2(Split2Args a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  Smem2& sm = *reinterpret_cast<Smem2*>(smem_raw);
  const SplitGeom& g = a.g;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int M = g.M, n = g.n, CT = g.CT;
  const int q16 = kKC / M, r16 = kKC - q16 * M;
  const long long u0 = unit_begin(g, blockIdx.x), u1 = unit_begin(g, blockIdx.x + 1);

  if (tid == 0) {
    // full: the producer's transaction count; empty and accfull: one commit
    // from each of the two MMA threads; accempty: every epilogue thread
    for (int s = 0; s < kStages; ++s) { mbar_init(&sm.full[s], 1); mbar_init(&sm.empty[s], 2); }
    for (int b = 0; b < 2; ++b) { mbar_init(&sm.accfull[b], 2); mbar_init(&sm.accempty[b], kEpi2 * 32); }
    mbar_init(&sm.mmadone[0], 1);
    mbar_init(&sm.mmadone[1], 1);
    sm.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kEpi2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem;

  if (warp == kEpi2 + 1) {
    // -------------------------------------------------------- producer --
    if (lane == 0) {
      long long issued = u0;
      UnitCur cu = unit_cur(g, u0);
      for (long long u = u0; u < u1; ++u, unit_next(g, cu, q16, r16)) {
        const int it = (int)(u - u0);
        const int s = it % kStages;
        if (!wait_bar2(sm, &sm.empty[s], ((it / kStages) & 1) ^ 1, a.status, a.spin)) break;
        if (u == a.withhold) break;  // test of the failure path: nothing issued for this stage
        const int cls = chunk_class(cu.m_lo, cu.m_hi, cu.c0, cu.c0 + CT - 1, g.band_w);
        const int slot = cls == 2 ? cu.kc - cu.qfirst : 0;
        const bool with_qu = cls == 2 && slot >= 0 && slot < a.qu_slots;
        uint8_t* st = sm.stage[s];
        mbar_arrive_expect_tx(&sm.full[s], kUnitBytes + kSmallBytes + (with_qu ? kBigTile : 0));
        bulk_g2s(st, a.planes + ((size_t)cu.ctile * a.cpt_stride + cu.kc) * kUnitBytes, kUnitBytes, &sm.full[s]);
        bulk_g2s(st + kUnitBytes + kBigTile, a.small + ((size_t)cu.kc * g.parts + cu.part) * kSmallBytes,
                 kSmallBytes, &sm.full[s]);
        if (with_qu)
          bulk_g2s(st + kUnitBytes, a.qu + ((size_t)cu.ctile * a.qu_slots + slot) * kBigTile, kBigTile,
                   &sm.full[s]);
        issued = u + 1;
      }
      // before the CTA can exit, the copies of the last units must have landed
      // (after an abort the MMA warp may not have waited for them)
      for (long long u = issued - 1; u >= u0 && u >= issued - kStages; --u) {
        const int it = (int)(u - u0);
        long long spins = 0;
        while (!mbar_try(&sm.full[it % kStages], (it / kStages) & 1) && ++spins < kSpinLimit) __nanosleep(64);
        if (spins >= kSpinLimit) atomicOr(a.status, kStatusTimeout);  // copies or MMAs may still be in flight
      }
    }
    __syncwarp();
  } else if (warp == kEpi2 || warp == kEpi2 + 2) {
    // -------------------------------------------------------- MMA warps --
    // Two threads issue the MMAs, one per accumulator group (warp kEpi2:
    // I^<, from PL and QU x NB^<; warp kEpi2 + 2: D, from Q and QU x NBD),
    // so that issuing overlaps; each commits to the stage and accumulator
    // barriers, which count both.  Descriptors are a per-stage base plus
    // compile-time offsets (a descriptor's start address is in 16-byte units).
    const int mgrp = warp == kEpi2 ? 0 : 1;
    if (lane == 0) {
      const uint64_t big0 = umma_desc(smem_u32(sm.stage[0]), 2048, 128);
      const uint64_t small0 = umma_desc(smem_u32(sm.stage[0] + kUnitBytes + kBigTile), 1024, 128);
      long long last = -1;
      UnitCur cu = unit_cur(g, u0);
      for (long long u = u0; u < u1; ++u, unit_next(g, cu, q16, r16)) {
        const int it = (int)(u - u0);
        const int s = it % kStages, b = it & 1;
        // the unit's class before the waits (it depends on the position only)
        int cls = chunk_class(cu.m_lo, cu.m_hi, cu.c0, cu.c0 + CT - 1, g.band_w);
        if (cls == 2) {
          const int slot = cu.kc - cu.qfirst;
          if (slot < 0 || slot >= a.qu_slots) cls = 0;  // reported by the encoder (status word)
        }
        if (!wait_bar2(sm, &sm.full[s], (it / kStages) & 1, a.status, a.spin)) break;
        if (!wait_bar2(sm, &sm.accempty[b], (it >> 1) & 1, a.status, a.spin)) break;
        tc_fence_after();
        const uint64_t so = (uint64_t)(s * kStage2Bytes) >> 4;
        const uint64_t dPL0 = big0 + so, dQ0 = dPL0 + (kBigTile >> 4);
        const uint64_t dQU0 = cls == 1 ? dQ0 : dPL0 + (kUnitBytes >> 4);
        const uint64_t dS0 = small0 + so;
        // group 0: I^< += PL A1 + QU NB^<;  group 1: D += Q A1 + QU NBD
        const uint32_t dacc = tmem + b * kAccCols + mgrp * kGroupCols;
        const uint64_t dA = mgrp == 0 ? dPL0 : dQ0;
        const uint64_t dSU = dS0 + (uint64_t)(((1 + mgrp) * kSmallVar) >> 4);
#pragma unroll
        for (int i = 0; i < kSlices; ++i) {
          const uint32_t idesc = umma_idesc_f16(kNS * (kLevels - i < kSlices ? kLevels - i : kSlices));
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            const uint64_t oa = (uint64_t)((i * kBigSlice + kk * 2 * 2048) >> 4);
            const uint64_t ob = (uint64_t)((kk * 2 * 1024) >> 4);
            umma_f16(dacc + i * kNS, dA + oa, dS0 + ob, idesc, 1);
            if (cls != 0) umma_f16(dacc + i * kNS, dQU0 + oa, dSU + ob, idesc, 1);
          }
        }
        umma_commit(&sm.accfull[b]);
        umma_commit(&sm.empty[s]);
        last = u;
      }
      // before the accumulators are freed, every MMA this thread issued must
      // have completed (its own barrier: after an abort the other thread may
      // not have committed the same units)
      if (last >= 0) {
        umma_commit(&sm.mmadone[mgrp]);
        long long spins = 0;
        while (!mbar_try(&sm.mmadone[mgrp], 0) && ++spins < kSpinLimit) __nanosleep(64);
        if (spins >= kSpinLimit) atomicOr(a.status, kStatusTimeout);  // MMAs may still be in flight
      }
    }
    __syncwarp();
  } else {
    // --------------------------------------------------------- epilogue --
    // warp = 8 half + 4 grp + quadrant: accumulator group grp (0: I^<,
    // 1: D = I^> - I^<), small-operand columns [8 half, 8 half + 8), for the 32 TMEM
    // lanes (= output rows) of its quadrant.
    constexpr int kQ = kNS / 2;
    const int quad = warp & 3, grp = (warp >> 2) & 1, half = warp >> 3;
    const int j = quad * 32 + lane;
    const int cl = j / M, bb = j - cl * M;
    const bool live_row = cl < CT;
    const uint32_t lane_addr = tmem + ((uint32_t)(quad * 32) << 16);
    const uint32_t my_cols = grp * kGroupCols + half * kQ;  // + level * kNS + q
    for (int bsel = 0; bsel < 2; ++bsel)
      for (int d = 0; d < kLevels; ++d) tmem_zero8(lane_addr + bsel * kAccCols + my_cols + d * kNS);
    tmem_wait_st();
    tc_fence_before();
    mbar_arrive(&sm.accempty[0]);
    mbar_arrive(&sm.accempty[1]);
    float run[kQ][2];
#pragma unroll
    for (int q = 0; q < kQ; ++q) { run[q][0] = 0.f; run[q][1] = 0.f; }
    int local_seg = 0;
    UnitCur cu = unit_cur(g, u0);
    for (long long u = u0; u < u1; ++u, unit_next(g, cu, q16, r16)) {
      const int it = (int)(u - u0);
      const int b = it & 1;
      // the unit's column exponent (stored with its planes) and small-operand
      // exponent, fetched before waiting for the accumulators
      const int ec = live_row ? __ldg(reinterpret_cast<const int*>(
                                      a.planes + ((size_t)cu.ctile * a.cpt_stride + cu.kc) * kUnitBytes +
                                      2 * kBigTile) + cl)
                              : 0;
      const int es = __ldg(a.e_small + cu.kc * g.parts + cu.part);
      if (!__all_sync(0xffffffffu, wait_bar2(sm, &sm.accfull[b], (it >> 1) & 1, a.status, a.spin))) break;
      tc_fence_after();
      const float sc = pow2f(scale_from_field(ec) + es - 14);
      const uint32_t buf = lane_addr + b * kAccCols + my_cols;
#pragma unroll
      for (int q4 = 0; q4 < kQ; q4 += 4) {
        float v[kLevels][4];
        tmem_ld4xL(buf + q4, kNS, v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float lv[kLevels] = {v[0][q], v[1][q], v[2][q], v[3][q], v[4][q]};
          float hi, lo;
          combine_levels(lv, hi, lo);
          float& rh = run[q4 + q][0];
          float& rl = run[q4 + q][1];
          df_add(rh, rl, hi * sc);
          rl += lo * sc;
        }
      }
#pragma unroll
      for (int d = 0; d < kLevels; ++d) tmem_zero8(buf + d * kNS);
      tmem_wait_st();
      tc_fence_before();
      mbar_arrive(&sm.accempty[b]);
      if (u + 1 == u1 || cu.kc + 1 == g.cpt) {
        const int c = cu.c0 + cl;
        if (live_row && c <= n) {
          double2* out = reinterpret_cast<double2*>(a.part) + ((size_t)blockIdx.x * g.S + local_seg) * (2 * 128 * kNA);
#pragma unroll
          for (int k = 0; k < kQ / 2; ++k) {
            const int al = half * (kQ / 2) + k;  // small-operand column = 2 al + (re, im)
            const double re = (double)run[2 * k][0] + (double)run[2 * k][1];
            const double im = (double)run[2 * k + 1][0] + (double)run[2 * k + 1][1];
            out[((size_t)grp * CT + cl) * kNA * M + al * M + bb] = make_double2(re, im);
          }
        }
#pragma unroll
        for (int q = 0; q < kQ; ++q) { run[q][0] = 0.f; run[q][1] = 0.f; }
        ++local_seg;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kEpi2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// ============================================================ fused path ==
// The same contraction with the conversion inside the contraction kernel,
// over the units of one or many systems: no digit-plane buffer (a batch of
// systems cannot hold one next to its histories).  A unit here is half a
// chunk: one column tile (128 output rows) times 8 complex history entries,
// one MMA K-step per digit slice.  Work list: the units of every system in
// order, split into contiguous ranges of about equal cost, one range per
// persistent CTA.
//
// Roles in one CTA (one per SM):
//  * 16 converter warps stream the FP64 history entries of the units three
//    ahead into a ring of five shared-memory stages with per-thread
//    asynchronous copies (cp.async, zero-filled outside the triangle), so
//    HBM latency hides behind the conversion of the units before.  For the
//    current unit each thread reads its own 4 entries back, the column
//    exponents are reduced in shared memory, and the digit planes PL and Q
//    overwrite the FP64 data of the same stage (after a barrier: the two take
//    the same 32 KB); the rare units that straddle the weight band also
//    write the masked QU plane into one separate buffer.
//  * one producer thread copies the small operands of each (unit, 8-orbital
//    part) into a ring of three 6 KB slots (the unit's half of the chunk's
//    12 KB of digit planes);
//  * two MMA-issuing threads, one per accumulator group (I^< and
//    D = I^> - I^<), run the unit's MMAs once per part into two TMEM
//    accumulator buffers;
//  * eight epilogue warps (4 lane quadrants x 2 groups) fold each part's
//    levels and scales into double-float running sums kept in tensor
//    memory, one per part, written out as FP64 partials when the range
//    leaves a column tile.
// Tensor memory: two accumulator buffers of 160 columns and up to three
// parts' running sums of 64 columns (512 columns), so an entry has at most
// three parts; larger systems run as entries of part ranges.
constexpr int kFEpiWarps = 8;
constexpr int kFConvWarps = 16;                                 // 512 threads: 4 entries of one row and array each
constexpr int kFConvThreads = kFConvWarps * 32;
constexpr int kFThreads = (kFEpiWarps + kFConvWarps + 3) * 32;  // + producer, two MMA warps: 864
constexpr int kHK = kKC / 2;                                    // complex history entries per unit
constexpr int kHSlice = 128 * 2 * kHK * 2;                      // one digit slice of one plane: 4 KB
constexpr int kHPlane = kSlices * kHSlice;                      // 16 KB
constexpr int kFStageBytes = 2 * kHPlane + 512;                 // PL | Q (FP64 staging in place) | exponents
constexpr int kFStages = 5;
constexpr int kFAhead = 3;                                      // units whose copies are in flight
constexpr int kFSmallHalf = kSmallVar / 2;                      // one variant's half of a chunk: 2 KB
constexpr int kFSmallSlot = 3 * kFSmallHalf;                    // 6 KB
constexpr int kFSlots = 3;
constexpr int kFMaxParts = 3;
constexpr int kFConvWeight = 7;                                 // a unit's conversion, in MMA-and-epilogue passes
constexpr int kFRunCol = 2 * kAccCols;                          // running sums from column 320
constexpr int kFRunPart = 2 * 2 * kNS;                          // per part: 2 groups x (16 hi, 16 lo)

struct FusedSys {
  const double* L;
  const double* R;
  const double* Sl;
  const double* Sg;
  WeightsView w;
  double* out;
  const uint8_t* small;   // [cpt][parts_total][kSmallBytes], written by fused_prep
  int* e_small;           // [cpt][parts_total]
  int M, n, CT, cpt, col_tiles;
  uint32_t magic;              // ceil(2^32 / M) (0 for M = 1): x / M without a division (fused_div)
  int upt;                     // units per column tile: 2 cpt
  int parts;                   // 8-orbital parts this entry contracts (<= 3): part0 .. part0 + parts - 1
  int part0, parts_total;      // first part, and all parts of the system (small-operand layout)
  long long unit_base, units;  // global units [unit_base, unit_base + units)
  long long tile_base;         // global index of the first column tile
  long long chunk_base;        // global index of the first chunk (prep grid)
  long long col_base;          // global index of the first output column (reduce grid)
};

// x / M for 0 <= x < 2^32 / M: floor(x ceil(2^32/M) / 2^32) equals floor(x / M)
// there (the product's excess over x 2^32 / M is below x / 2^32 < 1 / M).
__device__ __forceinline__ int fused_div(int x, int M, uint32_t magic) {
  return M == 1 ? x : (int)__umulhi((uint32_t)x, magic);
}

struct FusedArgs {
  const FusedSys* sys;
  int n_sys, G;
  const long long* cta_lo;     // [G + 1]: CTA i takes the units [cta_lo[i], cta_lo[i+1])
  const long long* cta_tile0;  // [G]: global column tile of CTA i's first unit
  const long long* seg_base;   // [G]: CTA i's first segment (one per column tile it touches)
  const long long* seg_slot;   // [segments]: first partial slot of the segment (one slot per part)
  double* part;                // [slots][kSlotComplex] complex
  int* status;
  long long withhold;          // failure-path test: no small operand is issued from this unit on
  long long spin;              // polls of a work wait before it gives up
};

struct SmemF {
  uint8_t stage[kFStages][kFStageBytes];
  uint8_t qu[kHPlane];
  uint8_t small[kFSlots][kFSmallSlot];
  uint64_t full[kFStages], empty[kFStages], qufull, quempty, sfull[kFSlots], sempty[kFSlots];
  uint64_t accfull[2], accempty[2], mmadone[2];
  int accmeta[2][128];   // column exponents of the unit whose part is in accumulator buffer b
  uint32_t tmem;
  int abort;
};

__device__ __forceinline__ bool wait_f(SmemF& sm, void* bar, uint32_t parity, int* status, long long limit) {
  long long it = 0;
  while (!mbar_try(bar, parity)) {
    if (++it > limit || *(volatile int*)&sm.abort) {
      if (it > limit) { atomicOr(status, kStatusTimeout); sm.abort = 1; }
      return false;
    }
    if (it > 64) __nanosleep(64);
  }
  return true;
}

__device__ __forceinline__ int first_sys(const FusedArgs& a, long long u) {
  int lo = 0, hi = a.n_sys;  // sys[lo].unit_base <= u
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a.sys[mid].unit_base <= u) lo = mid; else hi = mid;
  }
  return lo;
}

// 16 consecutive FP32 columns of this thread's TMEM lane from registers.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float v[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}

// 16-byte asynchronous copy global -> shared of this thread (zero-filled
// when `bytes` is 0), tracked by the thread's commit groups.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Where the units of a CTA's range sit, advanced one unit at a time (no
// division per unit): entry si, column tile, half-chunk hk of the tile.
struct UnitPos {
  int ctile, kc, half, kap0;
};
struct Cursor {
  int si, ctile, hk;
};
__device__ __forceinline__ Cursor cursor_at(const FusedArgs& a, long long u) {
  Cursor c;
  c.si = first_sys(a, u);
  const FusedSys& S = a.sys[c.si];
  const long long lu = u - S.unit_base;
  c.ctile = (int)(lu / S.upt);
  c.hk = (int)(lu - (long long)c.ctile * S.upt);
  return c;
}
__device__ __forceinline__ void cursor_next(const FusedArgs& a, Cursor& c) {
  const FusedSys& S = a.sys[c.si];
  if (++c.hk == S.upt) {
    c.hk = 0;
    if (++c.ctile == S.col_tiles) {
      c.ctile = 0;
      ++c.si;
    }
  }
}
__device__ __forceinline__ UnitPos unit_pos(const Cursor& c) {
  UnitPos p;
  p.ctile = c.ctile;
  p.kc = c.hk >> 1;
  p.half = c.hk & 1;
  p.kap0 = c.hk * kHK;
  return p;
}

// Small operands of every system's chunks (grid: global chunk x part).
__global__ void __launch_bounds__(256) fused_prep(const FusedSys* __restrict__ sys, int n_sys) {
  __shared__ int s_ef;
  const long long g = blockIdx.x;
  int lo = 0, hi = n_sys;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (sys[mid].chunk_base <= g) lo = mid; else hi = mid;
  }
  const FusedSys& S = sys[lo];
  if ((int)blockIdx.y >= S.parts) return;
  prep_chunk(S.M, S.n, S.parts_total, S.Sl, S.Sg, S.w, const_cast<uint8_t*>(S.small), S.e_small,
             (int)(g - S.chunk_base), S.part0 + (int)blockIdx.y, &s_ef);
}

__global__ void __launch_bounds__(kFThreads, 1) split_fused(FusedArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  SmemF& sm = *reinterpret_cast<SmemF*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long ua = a.cta_lo[blockIdx.x], ub = a.cta_lo[blockIdx.x + 1];
  constexpr int kProdWarp = kFEpiWarps + kFConvWarps, kMmaWarp = kProdWarp + 1;

  // rows beyond a unit's CT M are never written by the converters: zero the stages once
  for (int i = tid; i < (kFStages * kFStageBytes + kHPlane) / 16; i += kFThreads)
    reinterpret_cast<uint4*>(sm.stage)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    // full, qufull: every converter thread; empty, quempty, sempty: one commit
    // from each MMA thread; sfull: the producer's transaction count;
    // accfull: the first MMA thread's arrival (exponents copied) and both
    // commits; accempty: every epilogue thread
    for (int s = 0; s < kFStages; ++s) { mbar_init(&sm.full[s], kFConvThreads); mbar_init(&sm.empty[s], 2); }
    mbar_init(&sm.qufull, kFConvThreads);
    mbar_init(&sm.quempty, 2);
    for (int s = 0; s < kFSlots; ++s) { mbar_init(&sm.sfull[s], 1); mbar_init(&sm.sempty[s], 2); }
    for (int b = 0; b < 2; ++b) { mbar_init(&sm.accfull[b], 3); mbar_init(&sm.accempty[b], kFEpiWarps * 32); }
    mbar_init(&sm.mmadone[0], 1);
    mbar_init(&sm.mmadone[1], 1);
    sm.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kProdWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem;

  if (warp >= kFEpiWarps && warp < kProdWarp) {
    // ------------------------------------------------------ converters --
    // Thread ct: array arr (0: L -> the G^< plane PL, 1: R -> the Q plane),
    // output row jrow = (c_l, b), K entries 4 q .. 4 q + 3 of the unit (K-group
    // q of the plane).  Its staged entry k sits at (k * 512 + ct) * 16 bytes
    // of the stage (each warp reads 32 consecutive 16-byte words).
    const int ct = tid - kFEpiWarps * 32;
    const int arr = ct >> 8, jrow = (ct >> 1) & 127, q = ct & 1;
    Cursor ci = cursor_at(a, ua);  // issue cursor (runs kFAhead units ahead)
    auto issue = [&](long long v) {  // asynchronous copies of unit v (at cursor ci) into its stage
      const FusedSys& S = a.sys[ci.si];
      const int M = S.M, MM = M * M, n = S.n, CT = S.CT;
      const uint32_t mg = S.magic;
      const UnitPos P = unit_pos(ci);
      const bool row_live = jrow < CT * M;
      const int cl = row_live ? fused_div(jrow, M, mg) : 0, bb = jrow - cl * M;
      const int c = P.ctile * CT + cl;
      const bool col_live = row_live && c <= n;
      uint8_t* st = sm.stage[(int)((v - ua) % kFStages)];
      if (ct < 128) reinterpret_cast<int*>(st + 2 * kHPlane)[ct] = 0;
      const double2* base = reinterpret_cast<const double2*>(arr == 0 ? S.L : S.R);
      const int kap = P.kap0 + 4 * q;
      int m = fused_div(kap, M, mg), x = kap - m * M;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool ok = col_live && m <= n;
        const double2* src = base;
        if (ok) src = m >= c ? base + tri(m, c) * MM + x * M + bb : base + tri(c, m) * MM + bb * M + x;
        cp_async16(st + ((size_t)k * kFConvThreads + ct) * 16, src, ok ? 16u : 0u);
        if (++x == M) { x = 0; ++m; }
      }
    };
    // the first kFAhead units' copies
    for (int d = 0; d < kFAhead; ++d) {
      const long long v = ua + d;
      if (v < ub && conv_all<kFConvThreads>(wait_f(sm, &sm.empty[d % kFStages], 1, a.status, a.spin))) {
        issue(v);
        cursor_next(a, ci);
      }
      cp_async_commit();
    }
    long long ncls2 = 0;
    Cursor cu = cursor_at(a, ua);
    for (long long u = ua; u < ub; ++u, cursor_next(a, cu)) {
      const int it = (int)(u - ua);
      const int s = it % kFStages;
      const FusedSys& S = a.sys[cu.si];
      const int M = S.M, CT = S.CT, bw = S.w.band_w;
      const uint32_t mg = S.magic;
      const UnitPos P = unit_pos(cu);
      const bool row_live = jrow < CT * M;
      const int cl = row_live ? fused_div(jrow, M, mg) : 0;
      const int c0 = P.ctile * CT, c = c0 + cl;
      const int cls = chunk_class(fused_div(P.kap0, M, mg), fused_div(P.kap0 + kHK - 1, M, mg), c0, c0 + CT - 1, bw);
      uint8_t* st = sm.stage[s];
      int* ecol = reinterpret_cast<int*>(st + 2 * kHPlane);
      cp_async_wait<kFAhead - 1>();  // this thread's copies of unit u have landed
      double er[4], ei[4];
      unsigned keep = 0;  // bit k: entry k lies in the tensor-core part of term 2 (m <= c - band_w)
      int ef = 0;
      {
        const int kap = P.kap0 + 4 * q;
        int m = fused_div(kap, M, mg), x = kap - m * M;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          double2 z = *reinterpret_cast<const double2*>(st + ((size_t)k * kFConvThreads + ct) * 16);
          if (m < c) z.x = __hiloint2double(__double2hiint(z.x) ^ (int)0x80000000, __double2loint(z.x));  // -conj
          er[k] = z.x;
          ei[k] = z.y;
          ef = max(ef, max(exp_field(z.x), exp_field(z.y)));
          keep |= (unsigned)(m <= c - bw) << k;
          if (++x == M) { x = 0; ++m; }
        }
      }
      column_max(ecol, cl, ef, row_live);
      // every exponent is in and every staged entry of the stage has been read
      asm volatile("bar.sync 1, %0;" ::"r"(kFConvThreads) : "memory");
      const bool qu = cls == 2;
      if (qu) {  // the masked plane's buffer must be free (its last unit's MMAs done)
        if (!conv_all<kFConvThreads>(wait_f(sm, &sm.quempty, (uint32_t)((ncls2 & 1) ^ 1), a.status, a.spin))) break;
      }
      if (row_live) {
        const int e = scale_from_field(ecol[cl]);
        uint32_t w[kSlices][4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int Vr = fixed31_fast(er[k], e), Vi = fixed31_fast(ei[k], e);
          w[0][k] = digit_pair_f16<0>(Vr, Vi);
          w[1][k] = digit_pair_f16<1>(Vr, Vi);
          w[2][k] = digit_pair_f16<2>(Vr, Vi);
          w[3][k] = digit_pair_f16<3>(Vr, Vi);
        }
        const int off = (q * 16 + (jrow >> 3)) * 128 + (jrow & 7) * 16;
        uint8_t* dst = st + arr * kHPlane;
#pragma unroll
        for (int sl = 0; sl < kSlices; ++sl) {
          *reinterpret_cast<uint4*>(dst + sl * kHSlice + off) = make_uint4(w[sl][0], w[sl][1], w[sl][2], w[sl][3]);
          if (qu && arr == 1)
            *reinterpret_cast<uint4*>(sm.qu + sl * kHSlice + off) =
                make_uint4(keep & 1u ? w[sl][0] : 0u, keep & 2u ? w[sl][1] : 0u, keep & 4u ? w[sl][2] : 0u,
                           keep & 8u ? w[sl][3] : 0u);
        }
      }
      fence_async_smem();
      mbar_arrive(&sm.full[s]);
      if (qu) {
        mbar_arrive(&sm.qufull);
        ++ncls2;
      }
      // the copies of unit u + kFAhead, once its stage is free
      const long long v = u + kFAhead;
      if (v < ub) {
        const int sv = (int)((v - ua) % kFStages);
        if (!conv_all<kFConvThreads>(
                wait_f(sm, &sm.empty[sv], (uint32_t)((((v - ua) / kFStages) & 1) ^ 1), a.status, a.spin))) {
          cp_async_wait<0>();
          break;
        }
        issue(v);
        cursor_next(a, ci);
      }
      cp_async_commit();
    }
    cp_async_wait<0>();  // no copy may be in flight when the CTA exits
  } else if (warp == kProdWarp) {
    // -------------------------------------------------------- producer --
    // Small operands of each (unit, part), in the order the MMAs use them:
    // the unit's half of each variant (2 KB) of the chunk's digit planes.
    if (lane == 0) {
      long long it2 = 0, issued = 0;
      bool stop = false;
      Cursor cu = cursor_at(a, ua);
      for (long long u = ua; u < ub && !stop; ++u, cursor_next(a, cu)) {
        const FusedSys& S = a.sys[cu.si];
        const UnitPos P = unit_pos(cu);
        for (int p = 0; p < S.parts; ++p, ++it2) {
          const int ss = (int)(it2 % kFSlots);
          if (!wait_f(sm, &sm.sempty[ss], (uint32_t)(((it2 / kFSlots) & 1) ^ 1), a.status, a.spin) ||
              u == a.withhold) {
            stop = true;  // (withhold: test of the failure path, nothing issued from this unit on)
            break;
          }
          const uint8_t* src = S.small + ((size_t)P.kc * S.parts_total + S.part0 + p) * kSmallBytes + P.half * kFSmallHalf;
          mbar_arrive_expect_tx(&sm.sfull[ss], kFSmallSlot);
#pragma unroll
          for (int var = 0; var < 3; ++var)
            bulk_g2s(sm.small[ss] + var * kFSmallHalf, src + var * kSmallVar, kFSmallHalf, &sm.sfull[ss]);
          issued = it2 + 1;
        }
      }
      // the copies already issued must land before the CTA can exit
      for (long long k = issued - 1; k >= 0 && k >= issued - kFSlots; --k) {
        long long spins = 0;
        while (!mbar_try(&sm.sfull[k % kFSlots], (uint32_t)((k / kFSlots) & 1)) && ++spins < kSpinLimit)
          __nanosleep(64);
        if (spins >= kSpinLimit) atomicOr(a.status, kStatusTimeout);
      }
    }
    __syncwarp();
  } else if (warp > kProdWarp) {
    // -------------------------------------------------------- MMA warps --
    // group 0: I^< += PL A1 + QU NB^<;  group 1: D += Q A1 + QU NBD
    const int mgrp = warp - kMmaWarp;
    if (lane == 0) {
      // A: [slice 4][K-group 2][row group 16][8 rows][16 B]; B: [K-group 2][slice 4][col group 2][8][16 B]
      const uint64_t big0 = umma_desc(smem_u32(sm.stage[0]), 2048, 128);
      const uint64_t qu0 = umma_desc(smem_u32(sm.qu), 2048, 128);
      const uint64_t small0 = umma_desc(smem_u32(sm.small[0]), 1024, 128);
      long long it2 = 0, ncls2 = 0;
      bool any = false, stop = false;
      Cursor cu = cursor_at(a, ua);
      for (long long u = ua; u < ub && !stop; ++u, cursor_next(a, cu)) {
        const int it = (int)(u - ua);
        const int s = it % kFStages;
        const FusedSys& S = a.sys[cu.si];
        const int M = S.M, CT = S.CT, bw = S.w.band_w;
        const UnitPos P = unit_pos(cu);
        const int c0 = P.ctile * CT;
        const int cls =
            chunk_class(fused_div(P.kap0, M, S.magic), fused_div(P.kap0 + kHK - 1, M, S.magic), c0, c0 + CT - 1, bw);
        if (!wait_f(sm, &sm.full[s], (uint32_t)((it / kFStages) & 1), a.status, a.spin)) break;
        if (cls == 2 && !wait_f(sm, &sm.qufull, (uint32_t)(ncls2 & 1), a.status, a.spin)) break;
        const uint64_t so = (uint64_t)(s * kFStageBytes) >> 4;
        const uint64_t dPL0 = big0 + so, dQ0 = dPL0 + (kHPlane >> 4);
        const uint64_t dQU0 = cls == 1 ? dQ0 : qu0;
        const uint64_t dA = mgrp == 0 ? dPL0 : dQ0;
        for (int p = 0; p < S.parts; ++p, ++it2) {
          const int b = (int)(it2 & 1), ss = (int)(it2 % kFSlots);
          if (!wait_f(sm, &sm.sfull[ss], (uint32_t)((it2 / kFSlots) & 1), a.status, a.spin) ||
              !wait_f(sm, &sm.accempty[b], (uint32_t)((it2 >> 1) & 1), a.status, a.spin)) {
            stop = true;
            break;
          }
          tc_fence_after();
          if (mgrp == 0) {
            const int* ecol = reinterpret_cast<const int*>(sm.stage[s] + 2 * kHPlane);
            for (int k = 0; k < CT; ++k) sm.accmeta[b][k] = ecol[k];
            mbar_arrive(&sm.accfull[b]);
          }
          const uint64_t dS0 = small0 + ((uint64_t)(ss * kFSmallSlot) >> 4);
          const uint64_t dSU = dS0 + (uint64_t)(((1 + mgrp) * kFSmallHalf) >> 4);
          const uint32_t dacc = tmem + b * kAccCols + mgrp * kGroupCols;
#pragma unroll
          for (int i = 0; i < kSlices; ++i) {
            const uint32_t idesc = umma_idesc_f16(kNS * (kLevels - i < kSlices ? kLevels - i : kSlices));
            const uint64_t oa = (uint64_t)((i * kHSlice) >> 4);
            umma_f16(dacc + i * kNS, dA + oa, dS0, idesc, 1);
            if (cls != 0) umma_f16(dacc + i * kNS, dQU0 + oa, dSU, idesc, 1);
          }
          umma_commit(&sm.accfull[b]);
          umma_commit(&sm.sempty[ss]);
          any = true;
        }
        if (stop) break;
        umma_commit(&sm.empty[s]);
        if (cls == 2) {
          umma_commit(&sm.quempty);
          ++ncls2;
        }
      }
      // every MMA this thread issued must complete before tensor memory is freed
      if (any) {
        umma_commit(&sm.mmadone[mgrp]);
        long long spins = 0;
        while (!mbar_try(&sm.mmadone[mgrp], 0) && ++spins < kSpinLimit) __nanosleep(64);
        if (spins >= kSpinLimit) atomicOr(a.status, kStatusTimeout);
      }
    }
    __syncwarp();
  } else {
    // --------------------------------------------------------- epilogue --
    // warp = 4 grp + quadrant: accumulator group grp (0: I^<, 1: D = I^> -
    // I^<), all 16 small-operand columns, the 32 TMEM lanes (output rows) of
    // its quadrant.
    const int quad = warp & 3, grp = warp >> 2;
    const int j = quad * 32 + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(quad * 32) << 16);
    for (int b = 0; b < 2; ++b)
      for (int d = 0; d < kLevels; ++d) tmem_zero16(lane_addr + b * kAccCols + grp * kGroupCols + d * kNS);
    for (int p = 0; p < kFMaxParts; ++p) {
      tmem_zero16(lane_addr + kFRunCol + p * kFRunPart + grp * 2 * kNS);
      tmem_zero16(lane_addr + kFRunCol + p * kFRunPart + grp * 2 * kNS + kNS);
    }
    tmem_wait_st();
    tc_fence_before();
    mbar_arrive(&sm.accempty[0]);
    mbar_arrive(&sm.accempty[1]);
    long long it2 = 0, seg = a.seg_base[blockIdx.x];
    bool stop = false;
    Cursor cu = cursor_at(a, ua);
    for (long long u = ua; u < ub && !stop; ++u, cursor_next(a, cu)) {
      const FusedSys& S = a.sys[cu.si];
      const int M = S.M, n = S.n, CT = S.CT, parts = S.parts;
      const UnitPos P = unit_pos(cu);
      const int cl = fused_div(j, M, S.magic), bb = j - cl * M;
      const bool live_row = cl < CT;
      for (int p = 0; p < parts; ++p, ++it2) {
        const int b = (int)(it2 & 1);
        const int es = __ldg(S.e_small + P.kc * S.parts_total + S.part0 + p);
        if (!__all_sync(0xffffffffu, wait_f(sm, &sm.accfull[b], (uint32_t)((it2 >> 1) & 1), a.status, a.spin))) {
          stop = true;
          break;
        }
        tc_fence_after();
        const int ec = live_row ? sm.accmeta[b][cl] : 0;
        const float sc = pow2f(scale_from_field(ec) + es - 14);
        const uint32_t buf = lane_addr + b * kAccCols + grp * kGroupCols;
        const uint32_t run = lane_addr + kFRunCol + p * kFRunPart + grp * 2 * kNS;
        float rh[kNS], rl[kNS];
        tmem_ld16(run, rh);
        tmem_ld16(run + kNS, rl);
#pragma unroll
        for (int q4 = 0; q4 < kNS; q4 += 4) {
          float v[kLevels][4];
          tmem_ld4xL(buf + q4, kNS, v);
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            const float lv[kLevels] = {v[0][qq], v[1][qq], v[2][qq], v[3][qq], v[4][qq]};
            float hi, lo;
            combine_levels(lv, hi, lo);
            df_add(rh[q4 + qq], rl[q4 + qq], hi * sc);
            rl[q4 + qq] += lo * sc;
          }
        }
        tmem_st16(run, rh);
        tmem_st16(run + kNS, rl);
#pragma unroll
        for (int d = 0; d < kLevels; ++d) tmem_zero16(buf + d * kNS);
        tmem_wait_st();
        tc_fence_before();
        mbar_arrive(&sm.accempty[b]);
      }
      if (stop) break;
      // segment end: the next unit is in another column tile or system, or the range ends
      const bool last = u + 1 == ub || cu.hk + 1 == S.upt;
      if (last) {
        const int c = P.ctile * CT + cl;
        const long long slot0 = a.seg_slot[seg];
        for (int p = 0; p < parts; ++p) {
          const uint32_t run = lane_addr + kFRunCol + p * kFRunPart + grp * 2 * kNS;
          float rh[kNS], rl[kNS];
          tmem_ld16(run, rh);
          tmem_ld16(run + kNS, rl);
          if (live_row && c <= n) {
            double2* out = reinterpret_cast<double2*>(a.part) + (slot0 + p) * kSlotComplex;
#pragma unroll
            for (int al = 0; al < kNA; ++al) {
              const double re = (double)rh[2 * al] + (double)rl[2 * al];
              const double im = (double)rh[2 * al + 1] + (double)rl[2 * al + 1];
              out[((size_t)grp * CT + cl) * kNA * M + al * M + bb] = make_double2(re, im);
            }
          }
          tmem_zero16(run);
          tmem_zero16(run + kNS);
        }
        tmem_wait_st();
        ++seg;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kProdWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// ---------------------------------------------------------------- reduce -
// Reduction of one output column c and one 8-orbital part: the per-CTA
// partials of the column's tile (FP64, in CTA order; I^< from group 0,
// I^> from groups 0 and 1), plus the band of term 2,
//   sum_{m in (c - band_w, c]} w_{c,m} Sigma^s(n,m) G^A(m,c),
// with the exact composite weights.  The band runs in double-float on the
// FP32 pipe: the band points' R(c,m) (transposed, [x][b]) and
// w_{c,m} Sigma^s(n,m) for the part's rows a are staged as double-float
// pairs in shared memory, and each thread accumulates its outputs' products
// with Ogita-Rump-Oishi's compensated dot product (TwoSum of the leading
// products, the product errors and the TwoSum errors in a float tail),
// about 2^-47 of the products' sizes, far below the slice's 1e-8 bound.  In
// FP64 the band's band_w M^3 complex products per column and sign set this
// kernel's time (the FP64 pipe issues 1/64 of the FP32 rate on this part).
constexpr int kRedThreads = 128;
constexpr int kRedOut = 2 * kNA * 32 / kRedThreads;  // outputs per thread at M = 32
constexpr int kRedStage = 1792;  // float4 of staged operands: one point at M = 32 (1024 + 512)
constexpr int kRedGroup = 16;    // band points staged together at most (band_w <= 13)

struct DotAcc {
  float s, c;
};
// a += p q (p, q double-float)
__device__ __forceinline__ void dot_acc(DotAcc& a, float ph, float pl, float qh, float ql) {
  const float h = ph * qh;
  float e = fmaf(ph, qh, -h);
  e = fmaf(ph, ql, e);
  e = fmaf(pl, qh, e);
  const float s = a.s + h;
  const float v = s - a.s;
  a.c += ((a.s - (s - v)) + (h - v)) + e;
  a.s = s;
}
__device__ __forceinline__ float4 c2_of(double2 v) {
  const df::F2 re = df::from_double_fast(v.x), im = df::from_double_fast(v.y);
  return make_float4(re.hi, re.lo, im.hi, im.lo);
}

struct RedShared {
  int cnt, mnext, nslot;
  float4 stage[kRedStage];   // the group's R(c,m) (transposed, [x][b]), then its w_{c,m} Sigma^s(n,m) ([s][al][x])
  int m[kRedGroup];
  double dw[kRedGroup], wt[kRedGroup];
  long long slot[kMaxSplitCtas];  // partial slots of the column's tile, in CTA order
};

// Called by every thread of the block after slot[0..nslot) is set (and a
// __syncthreads).  As many band points as the shared arrays hold are
// staged together (all of them at M <= 8), so that their loads are in
// flight at once; the sums take the points in the same order either way.
__device__ __forceinline__ void reduce_column(RedShared& sh, int M, int n, int CT, int c, int pt,
                                              const double* __restrict__ part, const double* __restrict__ Sl,
                                              const double* __restrict__ Sg, const double* __restrict__ R,
                                              const WeightsView& w, double* __restrict__ out, int* status) {
  const int MM = M * M;
  const int cl = c % CT;
  const int na = min(kNA, M - pt * kNA);
  const int nout = 2 * na * M;
  DotAcc acc[kRedOut][2];
#pragma unroll
  for (int q = 0; q < kRedOut; ++q) acc[q][0] = acc[q][1] = DotAcc{0.f, 0.f};
  const int per = min(kRedGroup, kRedStage / (MM + nout));
  float4* s_r = sh.stage;
  float4* s_s = sh.stage + per * MM;
  for (int m_next = max(0, c - w.band_w + 1); m_next <= c;) {
    __syncthreads();  // the previous group's operands are consumed
    if (threadIdx.x < kRedGroup) {  // the next candidates' weights, loaded in parallel
      const int m = m_next + (int)threadIdx.x;
      sh.wt[threadIdx.x] = m <= c ? w.at(c, m) : 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int cnt = 0, k = 0;
      for (; k < kRedGroup && m_next + k <= c && cnt < per; ++k) {
        const double dw = sh.wt[k];
        if (dw != 0.0) { sh.m[cnt] = m_next + k; sh.dw[cnt] = dw; ++cnt; }
      }
      sh.cnt = cnt;
      sh.mnext = m_next + k;
    }
    __syncthreads();
    const int cnt = sh.cnt;
    m_next = sh.mnext;
#pragma unroll 4
    for (int f = threadIdx.x; f < cnt * MM; f += kRedThreads) {
      const int j = f / MM, i = f - j * MM;
      const int b = i / M, x = i - b * M;
      s_r[j * MM + x * M + b] = c2_of(reinterpret_cast<const double2*>(R)[tri(c, sh.m[j]) * MM + i]);
    }
#pragma unroll 4
    for (int f = threadIdx.x; f < cnt * nout; f += kRedThreads) {
      const int j = f / nout, i = f - j * nout;
      const int s = i / (na * M), r = i - s * (na * M);
      const double2 v = reinterpret_cast<const double2*>(s ? Sg : Sl)[(size_t)sh.m[j] * MM + pt * kNA * M + r];
      const double dw = sh.dw[j];
      s_s[f] = c2_of(make_double2(dw * v.x, dw * v.y));
    }
    __syncthreads();
    for (int j = 0; j < cnt; ++j) {
      const float4* sr = s_r + j * MM;
#pragma unroll
      for (int q = 0; q < kRedOut; ++q) {
        const int o = threadIdx.x + q * kRedThreads;
        if (o >= nout) break;
        const int row = o / M, bb = o - row * M;  // row = s * na + al
        const float4* sp = s_s + j * nout + row * M;
        for (int x = 0; x < M; ++x) {  // p conj(r): (p.re r.re + p.im r.im) + i (p.im r.re - p.re r.im)
          const float4 p = sp[x], r = sr[x * M + bb];
          dot_acc(acc[q][0], p.x, p.y, r.x, r.y);
          dot_acc(acc[q][0], p.z, p.w, r.z, r.w);
          dot_acc(acc[q][1], p.z, p.w, r.x, r.y);
          dot_acc(acc[q][1], -p.x, -p.y, r.z, r.w);
        }
      }
    }
  }
  __syncthreads();
  const int nslot = sh.nslot;
  bool bad = false;
#pragma unroll
  for (int q = 0; q < kRedOut; ++q) {
    const int o = threadIdx.x + q * kRedThreads;
    if (o >= nout || c > n) break;
    const int s = o / (na * M), r = o - s * (na * M);
    const int al = r / M, bb = r - al * M;
    // a non-finite float word is reported (to_double needs finite words)
    bad |= !(df::finite_bits(acc[q][0].s) && df::finite_bits(acc[q][0].c) && df::finite_bits(acc[q][1].s) &&
             df::finite_bits(acc[q][1].c));
    double re = df::to_double(df::F2{acc[q][0].s, acc[q][0].c});
    double im = df::to_double(df::F2{acc[q][1].s, acc[q][1].c});
    // group 0 holds I^<, group 1 holds D = I^> - I^<
    for (int grp = 0; grp <= s; ++grp)
      for (int k = 0; k < nslot; ++k) {
        const double2 v = reinterpret_cast<const double2*>(part)[sh.slot[k] * kSlotComplex +
                                                                  ((size_t)grp * CT + cl) * kNA * M + al * M + bb];
        re += v.x;
        im += v.y;
      }
    bad |= !(isfinite(re) && isfinite(im));
    reinterpret_cast<double2*>(out)[((size_t)s * (n + 1) + c) * MM + (pt * kNA + al) * M + bb] = make_double2(re, im);
  }
  if (bad) atomicOr(status, kStatusNumeric);
}

// Planes path: the CTAs of the uniform partition of the units that cover the
// column's tile, with their segment of that tile.  Seven CTAs per SM (at
// most 73 registers, 29 KB of shared memory each): one wave for the 1024
// (c, part) blocks of an 8-orbital slice of row 1023.
__global__ void __launch_bounds__(kRedThreads, 7) split_reduce2(SplitGeom g, const double* __restrict__ part,
                                                             const double* __restrict__ Sl,
                                                             const double* __restrict__ Sg,
                                                             const double* __restrict__ R, WeightsView w,
                                                             double* __restrict__ out, int* status) {
  __shared__ RedShared sh;
  const int c = blockIdx.x, pt = blockIdx.y;
  const int tile = (c / g.CT) * g.parts + pt;
  if (threadIdx.x == 0) {
    const long long ulo = (long long)tile * g.cpt, uhi = ulo + g.cpt;
    int i = (int)((ulo * g.G) / g.U);
    while (i > 0 && g.U * i / g.G > ulo) --i;
    while (i + 1 < g.G && g.U * (i + 1) / g.G <= ulo) ++i;
    int k = 0;
    for (; i < g.G && k < kMaxSplitCtas; ++i) {
      const long long b0 = g.U * i / g.G, b1 = g.U * (i + 1) / g.G;
      if (b0 >= uhi) break;
      if (b1 > b0) sh.slot[k++] = (long long)i * g.S + (tile - b0 / g.cpt);
    }
    sh.nslot = k;
  }
  reduce_column(sh, g.M, g.n, g.CT, c, pt, part, Sl, Sg, R, w, out, status);
}

// Fused path: the CTAs of the work list whose unit ranges meet the column's
// tile, each with the segment it wrote for that tile (grid: global column x
// part of the entry).
__global__ void __launch_bounds__(kRedThreads, 7) fused_reduce(FusedArgs a) {
  __shared__ RedShared sh;
  const long long gcol = blockIdx.x;
  int lo = 0, hi = a.n_sys;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a.sys[mid].col_base <= gcol) lo = mid; else hi = mid;
  }
  // entries of one system with different part ranges share its columns: take the one holding this part
  while (lo > 0 && a.sys[lo - 1].col_base == a.sys[lo].col_base) --lo;
  int pt = blockIdx.y;
  while (lo + 1 < a.n_sys && a.sys[lo + 1].col_base == a.sys[lo].col_base && pt >= a.sys[lo].parts) {
    pt -= a.sys[lo].parts;
    ++lo;
  }
  const FusedSys& S = a.sys[lo];
  if (pt >= S.parts) return;
  const int c = (int)(gcol - S.col_base);
  if (threadIdx.x == 0) {
    const int ct = c / S.CT;
    const long long T = S.tile_base + ct;
    const long long ulo = S.unit_base + (long long)ct * S.upt, uhi = ulo + S.upt;
    int l = 0, h = a.G - 1;  // first CTA whose range ends beyond ulo
    while (l < h) {
      const int mid = (l + h) >> 1;
      if (a.cta_lo[mid + 1] > ulo) h = mid; else l = mid + 1;
    }
    int k = 0;
    for (int i = l; i < a.G && a.cta_lo[i] < uhi && k < kMaxSplitCtas; ++i) {
      if (a.cta_lo[i + 1] <= a.cta_lo[i]) continue;
      sh.slot[k++] = a.seg_slot[a.seg_base[i] + (T - a.cta_tile0[i])] + pt;
    }
    sh.nslot = k;
  }
  reduce_column(sh, S.M, S.n, S.CT, c, S.part0 + pt, a.part, S.Sl, S.Sg, S.R, S.w, S.out, a.status);
}

inline dim3 reduce2_grid(const SplitGeomHost& h) { return dim3((unsigned)(h.n + 1), (unsigned)h.parts); }

}  // namespace

// Geometry of a split slice; returns false when the orbital count is not supported.
bool split_geometry(int M, int n, SplitGeomHost* h) {
  if (M < 1 || M > 32) return false;
  h->M = M;
  h->n = n;
  h->CT = 128 / M;
  h->parts = (M + kNA - 1) / kNA;
  h->cpt = (int)(((long long)(n + 1) * M + kKC - 1) / kKC);
  const int col_tiles = (n + 1 + h->CT - 1) / h->CT;
  h->tiles = col_tiles * h->parts;
  h->U = (long long)h->tiles * h->cpt;
  const int ctas = std::min(sm_count(), kMaxSplitCtas);
  h->G = (int)(h->U < ctas ? h->U : ctas);
  // tiles touched by one CTA range: at most ceil(range / cpt) + 1
  const long long range = (h->U + h->G - 1) / h->G;
  h->S = (int)((range + h->cpt - 1) / h->cpt + 1);
  return true;
}

// Upper bounds of a fused launch over one system of n_max rows (its slice of
// row n_max - 1 is the largest): partial slots and the plan image.
static size_t fused_single_part_bytes(const SplitGeomHost& h) {
  const int ctas = std::min(sm_count(), kMaxSplitCtas);
  const long long col_tiles = (h.n + 1 + h.CT - 1) / h.CT;
  return (size_t)(col_tiles + 2 * ctas) * h.parts * kSlotComplex * 16;
}
static size_t fused_single_plan_bytes(const SplitGeomHost& h) {
  const int ctas = std::min(sm_count(), kMaxSplitCtas);
  const long long col_tiles = (h.n + 1 + h.CT - 1) / h.CT;
  return 4 * sizeof(FusedSys) + 8 * (size_t)(3 * ctas + 1) + 8 * (size_t)(2 * (col_tiles + ctas)) + 5 * 256;
}

size_t split_workspace_bytes(int M, int n_max) {
  SplitGeomHost h;
  if (!split_geometry(M, n_max - 1, &h)) return 0;
  const size_t small = (size_t)h.cpt * h.parts * kSmallBytes + (size_t)h.cpt * h.parts * sizeof(int) + 256;
  const size_t part = std::max((size_t)h.G * h.S * 2 * 128 * kNA * 16, fused_single_part_bytes(h));
  return small + part + fused_single_plan_bytes(h) + 1024;
}

// The main kernel's dynamic shared memory exceeds the default limit; the
// attribute is set once per device (outside any stream capture when the
// first call is made before capturing).
cudaError_t split_prepare() {
  static std::atomic<unsigned long long> done_mask{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done_mask.load() & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(split_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SmemF));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(split_main2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem2));
  if (e == cudaSuccess) done_mask.fetch_or(bit);
  return e;
}

// Digit-plane buffers of the planes path for slices up to n_max - 1:
// [column tile][chunk] units of kUnitBytes at a fixed chunk stride (the
// chunk count of slice n_max - 1), then the QU slots.  Units of earlier
// slices stay valid at their places as the history grows.
static int qu_slots_of(const SplitGeomHost& h) { return (h.CT * h.M + 15) / 16 + 2; }

bool split_planes_layout(int M, int n_max, SplitPlanes* p) {
  SplitGeomHost h;
  if (!split_geometry(M, n_max - 1, &h)) return false;
  p->cpt_stride = h.cpt;
  p->col_tiles = (n_max + h.CT - 1) / h.CT;
  p->qu_slots = qu_slots_of(h);
  p->bytes = (size_t)p->col_tiles * h.cpt * kUnitBytes + (size_t)p->col_tiles * p->qu_slots * kBigTile + 256;
  return true;
}

cudaError_t launch_history_split2(const SplitLaunch& l, const SplitPlanes& pl_layout, void* planes, int r0,
                                  cudaStream_t s, int* launches) {
  SplitGeomHost h;
  *launches = 0;
  if (!split_geometry(l.M, l.n, &h)) return cudaErrorInvalidValue;
  SplitGeom g{h.M, h.M * h.M, h.n, h.CT, h.parts, h.cpt, h.tiles, h.U, h.G, h.S, l.w.band_w};
  uint8_t* ws = reinterpret_cast<uint8_t*>(l.work);
  uint8_t* small = ws;
  int* e_small = reinterpret_cast<int*>(small + (size_t)h.cpt * h.parts * kSmallBytes);
  size_t off = ((size_t)h.cpt * h.parts * kSmallBytes + (size_t)h.cpt * h.parts * sizeof(int) + 255) / 256 * 256;
  double* part = reinterpret_cast<double*>(ws + off);
  if (off + (size_t)h.G * h.S * 2 * 128 * kNA * 16 > l.work_bytes) return cudaErrorInvalidValue;
  const int col_tiles = (h.n + 1 + h.CT - 1) / h.CT;
  const int qs = qu_slots_of(h);
  if (col_tiles > pl_layout.col_tiles || h.cpt > pl_layout.cpt_stride || qs != pl_layout.qu_slots)
    return cudaErrorInvalidValue;
  uint8_t* pl = reinterpret_cast<uint8_t*>(planes);
  uint8_t* qu = pl + (size_t)pl_layout.col_tiles * pl_layout.cpt_stride * kUnitBytes;

  cudaError_t e = split_prepare();
  if (e != cudaSuccess) return e;
  split_prep<<<dim3(h.cpt, h.parts), 256, 0, s>>>(l.M, l.n, h.parts, l.Sl, l.Sg, l.w, small, e_small);
  ++*launches;
  // entries involving rows >= r0: every chunk of the columns c >= r0 (the
  // column tiles from the one holding column r0, those columns only), and
  // the chunks from the one holding row r0 onwards in the tiles up to that
  // one (all their columns; the columns >= r0 of the tile holding r0 get
  // the same values twice)
  if (r0 < 0) r0 = 0;
  const int ct_lo = r0 > h.n ? col_tiles : r0 / h.CT;
  const int kc_lo = (int)(((long long)r0 * h.M) / kKC);
  if (ct_lo < col_tiles) {
    EncodeArgs ea{g, l.L, l.R, pl, qu, pl_layout.cpt_stride, qs, ct_lo, 0, h.cpt, r0, l.status};
    ea.units = (unsigned)(col_tiles - ct_lo) * (unsigned)h.cpt;
    ea.row_lo = 0;
    ea.rows = 128;
    ea.upc = 1;
    unsigned threads = 256;
    if (col_tiles - ct_lo == 1) {  // one tile: only its rows from column r0 on, several chunks per CTA
      ea.row_lo = (r0 - ct_lo * h.CT) * h.M;
      ea.rows = h.CT * h.M - ea.row_lo;
      ea.upc = std::max(1, std::min(kEncMaxUpc, 128 / ea.rows));
      threads = (unsigned)((2 * ea.upc * ea.rows + 31) / 32 * 32);
    }
    if (ea.upc > 1 || ea.row_lo > 0)
      split_encode<true><<<(ea.units + ea.upc - 1) / ea.upc, threads, 0, s>>>(ea);
    else
      split_encode<false><<<ea.units, 256, 0, s>>>(ea);
    ++*launches;
  }
  const int ct_hi = std::min(col_tiles, ct_lo + 1);
  if (r0 > 0 && kc_lo < h.cpt) {
    EncodeArgs ea{g, l.L, l.R, pl, qu, pl_layout.cpt_stride, qs, 0, kc_lo, h.cpt - kc_lo, 0, l.status};
    ea.units = (unsigned)ct_hi * (unsigned)(h.cpt - kc_lo);
    ea.row_lo = 0;
    ea.rows = 128;
    ea.upc = 1;
    split_encode<false><<<ea.units, 256, 0, s>>>(ea);
    ++*launches;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  Split2Args args{g, pl, qu, pl_layout.cpt_stride, qs, small, e_small, part, l.status,
                  l.withhold, l.spin_limit > 0 ? l.spin_limit : kSpinLimit};
  if (l.ev_begin) cudaEventRecord(l.ev_begin, s);
  split_main2<<<h.G, kThreads2, sizeof(Smem2), s>>>(args);
  if (l.ev_end) cudaEventRecord(l.ev_end, s);
  ++*launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  split_reduce2<<<reduce2_grid(h), kRedThreads, 0, s>>>(g, part, l.Sl, l.Sg, l.R, l.w, l.out, l.status);
  ++*launches;
  return cudaGetLastError();
}

// ------------------------------------------------------------ fused host --
bool fused_build(const FusedSystem* in, int n_sys, FusedPlanHost* p) {
  p->image.clear();
  p->max_parts = 0;
  p->total_chunks = p->total_cols = 0;
  p->G = std::min(sm_count(), kMaxSplitCtas);
  if (n_sys < 1) return false;
  std::vector<FusedSys> ent;
  long long units = 0, tiles = 0, chunks = 0, cols = 0;
  for (int i = 0; i < n_sys; ++i) {
    SplitGeomHost h;
    if (!split_geometry(in[i].M, in[i].n, &h)) return false;
    const int col_tiles = (h.n + 1 + h.CT - 1) / h.CT;
    // systems of more than three 8-orbital parts run as entries of at most three parts each
    const int n_ent = (h.parts + kFMaxParts - 1) / kFMaxParts;
    const int per = (h.parts + n_ent - 1) / n_ent;
    for (int q = 0, part0 = 0; q < n_ent; ++q, part0 += per) {
      FusedSys f{};
      f.L = in[i].L; f.R = in[i].R; f.Sl = in[i].Sl; f.Sg = in[i].Sg; f.w = in[i].w; f.out = in[i].out;
      f.small = reinterpret_cast<const uint8_t*>(in[i].small);
      f.e_small = reinterpret_cast<int*>(reinterpret_cast<uint8_t*>(in[i].small) +
                                         (size_t)h.cpt * h.parts * kSmallBytes);
      f.M = h.M; f.n = h.n; f.CT = h.CT; f.cpt = h.cpt; f.col_tiles = col_tiles;
      f.magic = h.M == 1 ? 0u : (uint32_t)((0x100000000ull + (unsigned long long)h.M - 1) / (unsigned long long)h.M);
      f.upt = 2 * h.cpt;
      f.part0 = part0;
      f.parts = std::min(per, h.parts - part0);
      f.parts_total = h.parts;
      f.unit_base = units;
      f.units = (long long)col_tiles * f.upt;
      f.tile_base = tiles;
      f.chunk_base = chunks;
      f.col_base = cols;
      units += f.units;
      tiles += col_tiles;
      chunks += h.cpt;
      ent.push_back(f);
    }
    cols += h.n + 1;
    p->max_parts = std::max(p->max_parts, h.parts);
  }
  // contiguous unit ranges of about equal cost: a unit costs its conversion
  // plus one MMA-and-epilogue pass per part, weights kFConvWeight + parts
  // (measured per-system times at M = 4..24 put a unit's conversion at
  // about seven passes)
  const int G = p->G;
  long long W = 0;
  for (const FusedSys& f : ent) W += f.units * (kFConvWeight + f.parts);
  std::vector<long long> lo(G + 1), tile0(G, -1), segb(G);
  size_t e = 0;
  long long cw = 0;  // weight of the units before entry e
  for (int i = 0; i <= G; ++i) {
    const long long target = (long long)((__int128)W * i / G);
    while (e + 1 < ent.size() && cw + ent[e].units * (kFConvWeight + ent[e].parts) <= target) {
      cw += ent[e].units * (kFConvWeight + ent[e].parts);
      ++e;
    }
    const long long w = kFConvWeight + ent[e].parts;
    long long k = (target - cw + w - 1) / w;
    if (k > ent[e].units) k = ent[e].units;
    lo[i] = i == G ? units : ent[e].unit_base + k;
  }
  for (int i = 1; i <= G; ++i) lo[i] = std::max(lo[i], lo[i - 1]);
  std::vector<long long> slot;
  long long seg = 0, slots = 0;
  size_t k = 0;
  for (int i = 0; i < G; ++i) {
    segb[i] = seg;
    if (lo[i + 1] <= lo[i]) continue;
    while (k + 1 < ent.size() && lo[i] >= ent[k].unit_base + ent[k].units) ++k;
    size_t kk = k;
    long long prev_tile = -1;
    for (long long u = lo[i]; u < lo[i + 1];) {
      while (u >= ent[kk].unit_base + ent[kk].units) ++kk;
      const FusedSys& f = ent[kk];
      const long long t = f.tile_base + (u - f.unit_base) / f.upt;
      if (prev_tile < 0) tile0[i] = t;
      prev_tile = t;
      slot.push_back(slots);
      slots += f.parts;
      ++seg;
      // next unit of another tile: the end of this tile in the entry
      u = f.unit_base + ((u - f.unit_base) / f.upt + 1) * f.upt;
    }
  }
  p->n_ent = (int)ent.size();
  p->total_chunks = chunks;
  p->total_cols = cols;
  p->slots = slots;
  p->segments = seg;
  // device image: entries | cta_lo | cta_tile0 | seg_base | seg_slot
  auto align = [](size_t x) { return (x + 255) / 256 * 256; };
  p->off_sys = 0;
  p->off_lo = align(ent.size() * sizeof(FusedSys));
  p->off_tile0 = align(p->off_lo + (G + 1) * 8);
  p->off_segb = align(p->off_tile0 + G * 8);
  p->off_slot = align(p->off_segb + G * 8);
  p->image.assign(align(p->off_slot + std::max<size_t>(1, slot.size()) * 8), 0);
  memcpy(p->image.data() + p->off_sys, ent.data(), ent.size() * sizeof(FusedSys));
  memcpy(p->image.data() + p->off_lo, lo.data(), (G + 1) * 8);
  memcpy(p->image.data() + p->off_tile0, tile0.data(), G * 8);
  memcpy(p->image.data() + p->off_segb, segb.data(), G * 8);
  if (!slot.empty()) memcpy(p->image.data() + p->off_slot, slot.data(), slot.size() * 8);
  return true;
}

size_t fused_part_bytes(const FusedPlanHost& p) { return (size_t)std::max<long long>(1, p.slots) * kSlotComplex * 16; }

cudaError_t launch_history_fused(const FusedPlanHost& p, const void* plan_dev, double* part, int* status,
                                 cudaStream_t s, int* launches, cudaEvent_t ev_begin, cudaEvent_t ev_end,
                                 long long withhold, long long spin) {
  *launches = 0;
  cudaError_t e = split_prepare();
  if (e != cudaSuccess) return e;
  const uint8_t* b = reinterpret_cast<const uint8_t*>(plan_dev);
  FusedArgs a{};
  a.sys = reinterpret_cast<const FusedSys*>(b + p.off_sys);
  a.n_sys = p.n_ent;
  a.G = p.G;
  a.cta_lo = reinterpret_cast<const long long*>(b + p.off_lo);
  a.cta_tile0 = reinterpret_cast<const long long*>(b + p.off_tile0);
  a.seg_base = reinterpret_cast<const long long*>(b + p.off_segb);
  a.seg_slot = reinterpret_cast<const long long*>(b + p.off_slot);
  a.part = part;
  a.status = status;
  a.withhold = withhold < 0 ? (1ll << 62) : withhold;
  a.spin = spin > 0 ? spin : kSpinLimit;
  fused_prep<<<dim3((unsigned)p.total_chunks, (unsigned)kFMaxParts), 256, 0, s>>>(a.sys, a.n_sys);
  ++*launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev_begin) cudaEventRecord(ev_begin, s);
  split_fused<<<p.G, kFThreads, sizeof(SmemF), s>>>(a);
  if (ev_end) cudaEventRecord(ev_end, s);
  ++*launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  fused_reduce<<<dim3((unsigned)p.total_cols, (unsigned)p.max_parts), kRedThreads, 0, s>>>(a);
  ++*launches;
  return cudaGetLastError();
}

// Single system without a plane buffer: the fused contraction, its plan
// image uploaded from host memory into the tail of the workspace.
cudaError_t launch_history_split(const SplitLaunch& l, cudaStream_t s, int* launches) {
  SplitGeomHost h;
  *launches = 0;
  if (!split_geometry(l.M, l.n, &h)) return cudaErrorInvalidValue;
  FusedSystem in{l.M, l.n, l.L, l.R, l.Sl, l.Sg, l.w, l.out, l.work};
  FusedPlanHost p;
  if (!fused_build(&in, 1, &p)) return cudaErrorInvalidValue;
  uint8_t* ws = reinterpret_cast<uint8_t*>(l.work);
  const size_t off = ((size_t)h.cpt * h.parts * kSmallBytes + (size_t)h.cpt * h.parts * sizeof(int) + 255) / 256 * 256;
  const size_t pb = (fused_part_bytes(p) + 255) / 256 * 256;
  if (off + pb + p.image.size() > l.work_bytes) return cudaErrorInvalidValue;
  double* part = reinterpret_cast<double*>(ws + off);
  void* plan = ws + off + pb;
  // pageable source: staged before the call returns, so the host image may go
  cudaError_t e = cudaMemcpyAsync(plan, p.image.data(), p.image.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return launch_history_fused(p, plan, part, l.status, s, launches, l.ev_begin, l.ev_end, l.withhold, l.spin_limit);
}

}  // namespace kbe
