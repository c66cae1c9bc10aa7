// history_split.cu -- split-precision history slice of Eq. (KBE2) on tcgen05.
//
// The same contraction as history_f64.cu,
//   I^s(n,c) = sum_m w_{n,m} Sigma^R(n,m) G^s(m,c) + sum_{m<=c} w_{c,m} Sigma^s(n,m) G^A(m,c),
// evaluated on the bf16 tensor cores with error-free fixed-point slicing
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
// Roles in one CTA (1 CTA per SM, persistent over a contiguous range of
// (tile, chunk) units): 8 converter warps load the FP64 blocks, find the
// chunk exponent of each column, and write the bf16 digit planes into shared
// memory (two stages); one MMA warp issues tcgen05.mma into two TMEM buffers;
// 4 epilogue warps drain TMEM into double-float running sums and write one
// FP64 partial per (CTA, tile).  All mbarrier waits are bounded; a wait that
// runs out sets the status word and every role leaves its loop.

#include <atomic>
#include <cstdio>

#include "dfloat.cuh"
#include "kbe_internal.h"
#include "split_common.cuh"

namespace kbe {
namespace {

using namespace split;

constexpr int kConvWarps = 8;
constexpr int kEpiWarps = 4;
constexpr int kThreads = (kEpiWarps + 1 + kConvWarps) * 32;  // 416
constexpr int kConvThreads = kConvWarps * 32;
constexpr int kKC = 16;                     // complex K entries per chunk (32 real)
constexpr int kNS = 16;                     // small-operand columns per slice: 8 a x (re, im)
constexpr int kNA = 8;                      // a values per part
constexpr int kBigSlice = 128 * 2 * kKC * 2;          // bytes of one digit plane: 128 rows x 32 bf16
constexpr int kBigTile = kSlices * kBigSlice;         // 32 KB
constexpr int kSmallVar = 4 * kSlices * 2 * 128;      // 4 kgroups x 4 slices x 2 colgroups x 128 B = 4 KB
constexpr int kSmallBytes = 3 * kSmallVar;            // 12 KB
constexpr int kStageBytes = 3 * kBigTile + kSmallBytes + 512;  // + column exponents
constexpr int kStages = 2;
constexpr int kGroupCols = kLevels * kNS;   // 5 levels x 16 columns
constexpr int kAccCols = 2 * kGroupCols;    // groups I^< and I^>: 160 columns
constexpr int kTmemCols = 512;              // two accumulator buffers (320 used)
constexpr long long kSpinLimit = 1ll << 26; // bounded waits
constexpr int kMaxSplitCtas = 160;          // persistent CTAs of a contraction, at most

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

struct SplitArgs {
  SplitGeom g;
  const double* L;
  const double* R;
  const uint8_t* small;   // [cpt][parts][12288 B]
  const int* e_small;     // [cpt][parts]
  double* part;           // [G][S][2][CT][8][M] complex
  int* status;
};

// ---------------------------------------------------------------- prep ---
// Small operands of chunk kc, part p: A1, NB^<, NBD as bf16 digit planes in
// the shared-memory layout [variant][kgroup 4][slice 4][colgroup 2][8][8],
// entries B[(a, q_out)][(kappa, q_in)] of the real form of P z:
//   (re,re) = P.re, (re,im) = -P.im, (im,re) = P.im, (im,im) = P.re.
__global__ void __launch_bounds__(256) split_prep(int M, int n, int parts, const double* __restrict__ Sl,
                                                  const double* __restrict__ Sg, WeightsView w,
                                                  uint8_t* __restrict__ small, int* __restrict__ e_small) {
  const int kc = blockIdx.x, p = blockIdx.y;
  const int MM = M * M;
  __shared__ int s_ef;
  if (threadIdx.x == 0) s_ef = 0;
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
  if ((threadIdx.x & 31) == 0) atomicMax(&s_ef, my_ef);
  __syncthreads();
  const int e = scale_from_field(s_ef);
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
      const uint32_t pr = bf16_of_int(dr[sl]), pi = bf16_of_int(di[sl]), npi = bf16_of_int(-di[sl]);
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

// ---------------------------------------------------------------- main ---
struct Smem {
  uint8_t stage[kStages][kStageBytes];
  uint64_t full[kStages], empty[kStages], accfull[2], accempty[2];
  int accmeta[2][128];
  uint32_t tmem;
  int abort;
};

__device__ __forceinline__ long long unit_begin(const SplitGeom& g, int cta) { return g.U * cta / g.G; }

// AND of a predicate over the converter warps (named barrier 1); every
// converter thread must call it at the same point.
__device__ __forceinline__ bool conv_all(bool ok) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.and.pred q, 1, %2, p;\nselp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)ok), "r"(kConvThreads)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ bool wait_bar(Smem& sm, void* bar, uint32_t parity, int* status) {
  long long it = 0;
  while (!mbar_try(bar, parity)) {
    if (++it > kSpinLimit || *(volatile int*)&sm.abort) {
      if (it > kSpinLimit) { atomicOr(status, kStatusTimeout); sm.abort = 1; }
      return false;
    }
    if (it > 64) __nanosleep(64);
  }
  return true;
}

// Chunk class relative to the tile's column range [c0, c1]: term 2 of the
// tensor-core part covers m <= c - band_w (QU = Q there, 0 elsewhere).
// 0: QU = 0 for every (m, c) of the chunk; 1: QU = Q for all; 2: mixed.
__device__ __forceinline__ int chunk_class(int m_lo, int m_hi, int c0, int c1, int band_w) {
  if (m_lo > c1 - band_w) return 0;
  if (m_hi <= c0 - band_w) return 1;
  return 2;
}

__global__ void __launch_bounds__(kThreads, 1) split_main(SplitArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
  const SplitGeom& g = a.g;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int M = g.M, MM = g.MM, n = g.n, CT = g.CT;
  const long long u0 = unit_begin(g, blockIdx.x), u1 = unit_begin(g, blockIdx.x + 1);

  // zero the digit planes once (rows beyond CT*M are never written later)
  for (int i = tid; i < kStages * kStageBytes / 16; i += kThreads)
    reinterpret_cast<uint4*>(smem_raw)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) { mbar_init(&sm.full[s], kConvThreads); mbar_init(&sm.empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&sm.accfull[b], 2); mbar_init(&sm.accempty[b], kEpiWarps * 32); }
    sm.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kEpiWarps) {
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

  if (warp > kEpiWarps) {
    // ------------------------------------------------------ converters --
    // Thread ct owns one row j = (c_l, b) of one big operand (arr 0: the
    // G^< plane from L, arr 1: the Q plane from R) and all 16 K entries of
    // a chunk: 16 loads in flight, then one 16-byte store per K-group.
    const int ct = tid - (kEpiWarps + 1) * 32;  // 0..255
    const int arr = ct >> 7, jrow = ct & 127;
    const bool row_live = jrow < CT * M;
    const int cl = row_live ? jrow / M : 0, bb = jrow - cl * M;
    const double2* base = reinterpret_cast<const double2*>(arr == 0 ? a.L : a.R);
    for (long long u = u0; u < u1; ++u) {
      const int it = (int)(u - u0);
      const int s = it % kStages;
      if (!conv_all(wait_bar(sm, &sm.empty[s], ((it / kStages) & 1) ^ 1, a.status))) break;
      uint8_t* st = sm.stage[s];
      int* ecol = reinterpret_cast<int*>(st + 3 * kBigTile + kSmallBytes);
      const int tile = (int)(u / g.cpt), kc = (int)(u % g.cpt);
      const int ctile = tile / g.parts, part = tile % g.parts;
      const int c0 = ctile * CT;
      const int kap0 = kc * kKC;
      const int cls = chunk_class(kap0 / M, (kap0 + kKC - 1) / M, c0, c0 + CT - 1, g.band_w);
      {  // small operand of (kc, part): 12 KB
        const uint4* src = reinterpret_cast<const uint4*>(a.small + ((size_t)kc * g.parts + part) * kSmallBytes);
        uint4* dst = reinterpret_cast<uint4*>(st + 3 * kBigTile);
        for (int i = ct; i < kSmallBytes / 16; i += kConvThreads) dst[i] = src[i];
      }
      if (ct < CT) ecol[ct] = 0;
      asm volatile("bar.sync 1, %0;" ::"r"(kConvThreads) : "memory");
      const int c = c0 + cl;
      const bool col_live = row_live && c <= n;
      double er[kKC], ei[kKC];
      unsigned keep = 0;  // bit k: K entry k lies in the tensor-core part of term 2 (m <= c - band_w)
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
      if (row_live && ef > 0) atomicMax(&ecol[cl], ef);
      asm volatile("bar.sync 1, %0;" ::"r"(kConvThreads) : "memory");
      if (row_live) {
        const int e = scale_from_field(ecol[cl]);
        uint8_t* dst = st + arr * kBigTile;  // PL or Q
        uint8_t* QU = st + 2 * kBigTile;
        const bool qu = arr == 1 && cls == 2;
#pragma unroll
        for (int kg = 0; kg < 4; ++kg) {
          uint32_t w[kSlices][4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            uint32_t dr[kSlices], di[kSlices];
            digits_bf16(fixed31(er[4 * kg + q], e), dr);
            digits_bf16(fixed31(ei[4 * kg + q], e), di);
#pragma unroll
            for (int sl = 0; sl < kSlices; ++sl) w[sl][q] = __byte_perm(dr[sl], di[sl], 0x5410);
          }
          const int off = (kg * 16 + (jrow >> 3)) * 128 + (jrow & 7) * 16;
#pragma unroll
          for (int sl = 0; sl < kSlices; ++sl) {
            *reinterpret_cast<uint4*>(dst + sl * kBigSlice + off) = make_uint4(w[sl][0], w[sl][1], w[sl][2], w[sl][3]);
            if (qu) {
              const unsigned kb = keep >> (4 * kg);
              *reinterpret_cast<uint4*>(QU + sl * kBigSlice + off) =
                  make_uint4(kb & 1u ? w[sl][0] : 0u, kb & 2u ? w[sl][1] : 0u, kb & 4u ? w[sl][2] : 0u,
                             kb & 8u ? w[sl][3] : 0u);
            }
          }
        }
      }
      fence_async_smem();
      mbar_arrive(&sm.full[s]);
    }
  } else if (warp == kEpiWarps) {
    // --------------------------------------------------------- MMA warp --
    if (lane == 0) {
      long long last = -1;
      for (long long u = u0; u < u1; ++u) {
        const int it = (int)(u - u0);
        const int s = it % kStages, b = it & 1;
        if (!wait_bar(sm, &sm.full[s], (it / kStages) & 1, a.status)) break;
        if (!wait_bar(sm, &sm.accempty[b], (it >> 1) & 1, a.status)) break;
        tc_fence_after();
        uint8_t* st = sm.stage[s];
        const int* ecol = reinterpret_cast<const int*>(st + 3 * kBigTile + kSmallBytes);
        for (int c = 0; c < CT; ++c) sm.accmeta[b][c] = ecol[c];
        mbar_arrive(&sm.accfull[b]);  // releases accmeta; the commit below is the second arrival
        const int tile = (int)(u / g.cpt), kc = (int)(u % g.cpt);
        const int c0 = (tile / g.parts) * CT;
        const int kap0 = kc * kKC;
        const int cls = chunk_class(kap0 / M, (kap0 + kKC - 1) / M, c0, c0 + CT - 1, g.band_w);
        const uint32_t aPL = smem_u32(st), aQ = smem_u32(st + kBigTile);
        const uint32_t aQU = cls == 1 ? aQ : smem_u32(st + 2 * kBigTile);
        const uint32_t bS = smem_u32(st + 3 * kBigTile);
        const uint32_t dl = tmem + b * kAccCols, dg = dl + kGroupCols;
        for (int i = 0; i < kSlices; ++i) {
          // small digits j with i + j <= 4: N = 16 * min(4, 5 - i)
          const uint32_t idesc = umma_idesc_bf16(kNS * min(kSlices, kLevels - i));
          for (int kk = 0; kk < 2; ++kk) {
            const uint32_t ka = (uint32_t)(i * kBigSlice + kk * 2 * 2048);
            const uint64_t dPL = umma_desc(aPL + ka, 2048, 128);
            const uint64_t dQ = umma_desc(aQ + ka, 2048, 128);
            const uint64_t dQU = umma_desc(aQU + ka, 2048, 128);
            const uint32_t kb = (uint32_t)(kk * 2 * 1024);
            const uint64_t dA1 = umma_desc(bS + 0 * kSmallVar + kb, 1024, 128);
            const uint64_t dNl = umma_desc(bS + 1 * kSmallVar + kb, 1024, 128);
            const uint64_t dNg = umma_desc(bS + 2 * kSmallVar + kb, 1024, 128);
            umma_bf16(dl + i * kNS, dPL, dA1, idesc, 1);
            umma_bf16(dg + i * kNS, dQ, dA1, idesc, 1);
            if (cls != 0) {
              umma_bf16(dl + i * kNS, dQU, dNl, idesc, 1);
              umma_bf16(dg + i * kNS, dQU, dNg, idesc, 1);
            }
          }
        }
        umma_commit(&sm.accfull[b]);
        umma_commit(&sm.empty[s]);
        last = u;
      }
      // wait for the MMAs still in flight before the accumulators are freed
      if (last >= 0) {
        const int it = (int)(last - u0);
        long long spins = 0;
        while (!mbar_try(&sm.empty[it % kStages], (it / kStages) & 1) && ++spins < kSpinLimit) __nanosleep(64);
        if (spins >= kSpinLimit) atomicOr(a.status, kStatusTimeout);  // copies or MMAs may still be in flight
      }
    }
    __syncwarp();
  } else {
    // --------------------------------------------------------- epilogue --
    const int j = tid;  // TMEM lane = output row (c_l, b)
    const int cl = j / M, bb = j - cl * M;
    const bool live_row = cl < CT;
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    // both accumulator buffers start at zero; every drain zeroes its buffer again
    for (int col = 0; col < 2 * kAccCols; col += 16) tmem_zero16(lane_addr + col);
    tmem_wait_st();
    tc_fence_before();
    mbar_arrive(&sm.accempty[0]);
    mbar_arrive(&sm.accempty[1]);
    float run[2][kNS][2];
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
      for (int q = 0; q < kNS; ++q) { run[s2][q][0] = 0.f; run[s2][q][1] = 0.f; }
    int local_seg = 0;
    for (long long u = u0; u < u1; ++u) {
      const int it = (int)(u - u0);
      const int b = it & 1;
      if (!__all_sync(0xffffffffu, wait_bar(sm, &sm.accfull[b], (it >> 1) & 1, a.status))) break;
      tc_fence_after();
      const int tile = (int)(u / g.cpt), kc = (int)(u % g.cpt);
      const int part = tile % g.parts;
      const int ec = live_row ? sm.accmeta[b][cl] : 0;
      const float sc = pow2f(scale_from_field(ec) + a.e_small[kc * g.parts + part] - 14);
      const uint32_t buf = lane_addr + b * kAccCols;
#pragma unroll
      for (int grp = 0; grp < 2; ++grp) {
#pragma unroll
        for (int q4 = 0; q4 < kNS; q4 += 4) {
          float v[kLevels][4];
          tmem_ld4xL(buf + grp * kGroupCols + q4, kNS, v);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            // sum_d v_d 2^(-8d) in double-float; every v_d is an exact integer
            float hi = v[0][q], lo = 0.f, f = 1.f;
#pragma unroll
            for (int d = 1; d < kLevels; ++d) {
              f *= 0.00390625f;  // 2^-8
              df_add(hi, lo, v[d][q] * f);
            }
            float& rh = run[grp][q4 + q][0];
            float& rl = run[grp][q4 + q][1];
            df_add(rh, rl, hi * sc);
            rl += lo * sc;
          }
        }
      }
      for (int col = 0; col < kAccCols; col += 16) tmem_zero16(buf + col);
      tmem_wait_st();
      tc_fence_before();
      mbar_arrive(&sm.accempty[b]);
      // segment end: the next unit is in another tile, or the range ends
      if ((u + 1 == u1) || ((u + 1) / g.cpt != tile)) {
        const int c = (tile / g.parts) * CT + cl;
        if (live_row && c <= n) {
          double2* out = reinterpret_cast<double2*>(a.part) + ((size_t)blockIdx.x * g.S + local_seg) * (2 * 128 * kNA);
          // slot layout [s][c_l][a_l][b], a_l < 8; small-operand column = 2 a_l + (re, im)
#pragma unroll
          for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
            for (int al = 0; al < kNA; ++al) {
              const double re = (double)run[s2][2 * al][0] + (double)run[s2][2 * al][1];
              const double im = (double)run[s2][2 * al + 1][0] + (double)run[s2][2 * al + 1][1];
              out[((size_t)s2 * CT + cl) * kNA * M + al * M + bb] = make_double2(re, im);
            }
        }
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
          for (int q = 0; q < kNS; ++q) { run[s2][q][0] = 0.f; run[s2][q][1] = 0.f; }
        ++local_seg;
      }
    }
  }
  // ------------------------------------------------------------ teardown --
  tc_fence_before();
  __syncthreads();
  if (warp == kEpiWarps) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
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
};

// One CTA per (column tile, chunk): thread (arr, jrow) encodes row jrow of
// plane arr (0: G^< from L, 1: Q from R) for the chunk's 16 K entries.
// Every column has its own exponent, so the rows of the columns below c_min
// are left as they are.
__global__ void __launch_bounds__(256, 3) split_encode(EncodeArgs a) {
  const SplitGeom& g = a.g;
  const int M = g.M, MM = g.MM, n = g.n, CT = g.CT;
  const int ctile = a.ct_base + (int)(blockIdx.x / (unsigned)a.kc_count);
  const int kc = a.kc_base + (int)(blockIdx.x % (unsigned)a.kc_count);
  __shared__ int ecol[128];
  const int ct = threadIdx.x, arr = ct >> 7, jrow = ct & 127;
  const bool row_live = jrow < CT * M;
  const int cl = row_live ? jrow / M : 0, bb = jrow - cl * M;
  const int c0 = ctile * CT;
  const int kap0 = kc * kKC;
  const int cls = chunk_class(kap0 / M, (kap0 + kKC - 1) / M, c0, c0 + CT - 1, g.band_w);
  if (ct < 128) ecol[ct] = 0;
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
  if (enc && ef > 0) atomicMax(&ecol[cl], ef);
  __syncthreads();
  uint8_t* unit = a.planes + ((size_t)ctile * a.cpt_stride + kc) * kUnitBytes;
  uint8_t* dst = unit + arr * kBigTile;
  uint8_t* QU = nullptr;
  if (arr == 1 && cls == 2) {
    const int slot = qu_slot(kc, c0, M, g.band_w);
    if (slot >= 0 && slot < a.qu_slots) QU = a.qu + ((size_t)ctile * a.qu_slots + slot) * kBigTile;
    else if (ct == 128) atomicOr(a.status, kStatusInternal);  // geometry error: reported, never written
  }
  const int e = scale_from_field(ecol[cl]);
#pragma unroll
  for (int kg = 0; kg < 4 && enc; ++kg) {
    uint32_t w[kSlices][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t dr[kSlices], di[kSlices];
      digits_bf16(fixed31(er[4 * kg + q], e), dr);
      digits_bf16(fixed31(ei[4 * kg + q], e), di);
#pragma unroll
      for (int sl = 0; sl < kSlices; ++sl) w[sl][q] = __byte_perm(dr[sl], di[sl], 0x5410);
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
  if (ct < 128 && c0 + ct >= a.c_min) reinterpret_cast<int*>(unit + 2 * kBigTile)[ct] = ecol[ct];
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

__global__ void __launch_bounds__(kThreads2, 1) split_main2(Split2Args a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  Smem2& sm = *reinterpret_cast<Smem2*>(smem_raw);
  const SplitGeom& g = a.g;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int M = g.M, n = g.n, CT = g.CT;
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
      for (long long u = u0; u < u1; ++u) {
        const int it = (int)(u - u0);
        const int s = it % kStages;
        if (!wait_bar2(sm, &sm.empty[s], ((it / kStages) & 1) ^ 1, a.status, a.spin)) break;
        if (u == a.withhold) break;  // test of the failure path: nothing issued for this stage
        const int tile = (int)(u / g.cpt), kc = (int)(u % g.cpt);
        const int ctile = tile / g.parts, part = tile % g.parts;
        const int c0 = ctile * CT;
        const int kap0 = kc * kKC;
        const int cls = chunk_class(kap0 / M, (kap0 + kKC - 1) / M, c0, c0 + CT - 1, g.band_w);
        const int slot = cls == 2 ? qu_slot(kc, c0, M, g.band_w) : 0;
        const bool with_qu = cls == 2 && slot >= 0 && slot < a.qu_slots;
        uint8_t* st = sm.stage[s];
        mbar_arrive_expect_tx(&sm.full[s], kUnitBytes + kSmallBytes + (with_qu ? kBigTile : 0));
        bulk_g2s(st, a.planes + ((size_t)ctile * a.cpt_stride + kc) * kUnitBytes, kUnitBytes, &sm.full[s]);
        bulk_g2s(st + kUnitBytes + kBigTile, a.small + ((size_t)kc * g.parts + part) * kSmallBytes, kSmallBytes,
                 &sm.full[s]);
        if (with_qu)
          bulk_g2s(st + kUnitBytes, a.qu + ((size_t)ctile * a.qu_slots + slot) * kBigTile, kBigTile, &sm.full[s]);
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
      for (long long u = u0; u < u1; ++u) {
        const int it = (int)(u - u0);
        const int s = it % kStages, b = it & 1;
        if (!wait_bar2(sm, &sm.full[s], (it / kStages) & 1, a.status, a.spin)) break;
        if (!wait_bar2(sm, &sm.accempty[b], (it >> 1) & 1, a.status, a.spin)) break;
        tc_fence_after();
        const int tile = (int)(u / g.cpt), kc = (int)(u % g.cpt);
        const int c0 = (tile / g.parts) * CT;
        const int kap0 = kc * kKC;
        int cls = chunk_class(kap0 / M, (kap0 + kKC - 1) / M, c0, c0 + CT - 1, g.band_w);
        if (cls == 2) {
          const int slot = qu_slot(kc, c0, M, g.band_w);
          if (slot < 0 || slot >= a.qu_slots) cls = 0;  // reported by the encoder (status word)
        }
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
          const uint32_t idesc = umma_idesc_bf16(kNS * (kLevels - i < kSlices ? kLevels - i : kSlices));
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            const uint64_t oa = (uint64_t)((i * kBigSlice + kk * 2 * 2048) >> 4);
            const uint64_t ob = (uint64_t)((kk * 2 * 1024) >> 4);
            umma_bf16(dacc + i * kNS, dA + oa, dS0 + ob, idesc, 1);
            if (cls != 0) umma_bf16(dacc + i * kNS, dQU0 + oa, dSU + ob, idesc, 1);
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
    for (long long u = u0; u < u1; ++u) {
      const int it = (int)(u - u0);
      const int b = it & 1;
      const int tile = (int)(u / g.cpt), kc = (int)(u % g.cpt);
      // the unit's column exponent (stored with its planes) and small-operand
      // exponent, fetched before waiting for the accumulators
      const int ec = live_row ? __ldg(reinterpret_cast<const int*>(
                                      a.planes + ((size_t)(tile / g.parts) * a.cpt_stride + kc) * kUnitBytes +
                                      2 * kBigTile) + cl)
                              : 0;
      const int es = __ldg(a.e_small + kc * g.parts + tile % g.parts);
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
      if ((u + 1 == u1) || ((u + 1) / g.cpt != tile)) {
        const int c = (tile / g.parts) * CT + cl;
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

// ---------------------------------------------------------------- reduce -
// I_out[s][c][a][b] = sum of the partials of every CTA that covered the
// tile of (c, a), in CTA order (I^< from group 0; I^> from groups 0 and 1),
// plus the band of term 2 with the exact composite weights,
//   sum_{m = c-K..c} w_{c,m} S^s(n,m)_ax conj(R(c,m)_bx).
// Reduction of one output column c and one 8-orbital part (block (c, part)):
// the per-CTA partials of the column's tile in CTA order (FP64), plus the
// band of term 2, sum_{m in (c - band_w, c]} w_{c,m} Sigma^s(n,m) G^A(m,c),
// with the exact weights.  The band runs in double-float on the FP32 pipe:
// per band point m the block stages R(c,m) (transposed, [x][b]) and
// w_{c,m} Sigma^s(n,m) for its rows a as double-float pairs in shared memory,
// and each thread accumulates its outputs' products with Ogita-Rump-Oishi's
// compensated dot product (TwoSum of the leading products, the product
// errors and the TwoSum errors in a float tail), about 2^-47 of the
// products' sizes, far below the slice's 1e-8 bound.  In FP64 the band's
// band_w M^3 complex products per column and sign set this kernel's time
// (the FP64 pipe issues 1/64 of the FP32 rate on this part).
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

// Seven CTAs per SM (at most 73 registers, 29 KB of shared memory each):
// one wave for the 1024 (c, part) blocks of an 8-orbital slice of row 1023.
__global__ void __launch_bounds__(kRedThreads, 7) split_reduce2(SplitGeom g, const double* __restrict__ part,
                                                             const double* __restrict__ Sl,
                                                             const double* __restrict__ Sg,
                                                             const double* __restrict__ R, WeightsView w,
                                                             double* __restrict__ out, int* status) {
  const int M = g.M, MM = g.MM, n = g.n, CT = g.CT;
  const int c = blockIdx.x, pt = blockIdx.y;
  const int ctile = c / CT, cl = c - ctile * CT;
  const int tile = ctile * g.parts + pt;
  const int na = min(kNA, M - pt * kNA);
  const int nout = 2 * na * M;
  __shared__ int s_i0, s_k, s_cnt, s_mnext;
  __shared__ int s_seg[kMaxSplitCtas];
  __shared__ float4 s_stage[kRedStage];        // the group's R(c,m) (transposed, [x][b]), then its
                                               // w_{c,m} Sigma^s(n,m) ([s][al][x]), per point
  __shared__ int s_m[kRedGroup];
  __shared__ double s_dw[kRedGroup], s_wt[kRedGroup];
  if (threadIdx.x == 0) {
    const long long ulo = (long long)tile * g.cpt, uhi = ulo + g.cpt;
    int i = (int)((ulo * g.G) / g.U);
    while (i > 0 && g.U * i / g.G > ulo) --i;
    while (i + 1 < g.G && g.U * (i + 1) / g.G <= ulo) ++i;
    const int i0 = i;
    int k = 0;
    for (; i < g.G && k < kMaxSplitCtas; ++i) {
      const long long b0 = g.U * i / g.G, b1 = g.U * (i + 1) / g.G;
      if (b0 >= uhi) break;
      s_seg[k++] = b1 <= b0 ? -1 : (int)(tile - b0 / g.cpt);
    }
    s_i0 = i0;
    s_k = k;
  }
  DotAcc acc[kRedOut][2];
#pragma unroll
  for (int q = 0; q < kRedOut; ++q) acc[q][0] = acc[q][1] = DotAcc{0.f, 0.f};
  // band of term 2: the points m = c - band_w + 1 .. c with w_{c,m} != 0,
  // in increasing m.  As many points as the shared arrays hold are staged
  // together (all of them at M <= 8), so that their loads are in flight at
  // once; the sums take the points in the same order either way.
  const int per = min(kRedGroup, kRedStage / (MM + nout));
  float4* s_r = s_stage;
  float4* s_s = s_stage + per * MM;
  for (int m_next = max(0, c - w.band_w + 1); m_next <= c;) {
    __syncthreads();  // the previous group's operands are consumed
    if (threadIdx.x < kRedGroup) {  // the next candidates' weights, loaded in parallel
      const int m = m_next + (int)threadIdx.x;
      s_wt[threadIdx.x] = m <= c ? w.at(c, m) : 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int cnt = 0, k = 0;
      for (; k < kRedGroup && m_next + k <= c && cnt < per; ++k) {
        const double dw = s_wt[k];
        if (dw != 0.0) { s_m[cnt] = m_next + k; s_dw[cnt] = dw; ++cnt; }
      }
      s_cnt = cnt;
      s_mnext = m_next + k;
    }
    __syncthreads();
    const int cnt = s_cnt;
    m_next = s_mnext;
#pragma unroll 4
    for (int f = threadIdx.x; f < cnt * MM; f += kRedThreads) {
      const int j = f / MM, i = f - j * MM;
      const int b = i / M, x = i - b * M;
      s_r[j * MM + x * M + b] = c2_of(reinterpret_cast<const double2*>(R)[tri(c, s_m[j]) * MM + i]);
    }
#pragma unroll 4
    for (int f = threadIdx.x; f < cnt * nout; f += kRedThreads) {
      const int j = f / nout, i = f - j * nout;
      const int s = i / (na * M), r = i - s * (na * M);
      const double2 v = reinterpret_cast<const double2*>(s ? Sg : Sl)[(size_t)s_m[j] * MM + pt * kNA * M + r];
      const double dw = s_dw[j];
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
  const int i0 = s_i0, nk = s_k;
  bool bad = false;
#pragma unroll
  for (int q = 0; q < kRedOut; ++q) {
    const int o = threadIdx.x + q * kRedThreads;
    if (o >= nout || c > n) break;
    const int s = o / (na * M), r = o - s * (na * M);
    const int al = r / M, bb = r - al * M;
    // group 0 holds I^<, group 1 holds D = I^> - I^<
    // a non-finite float word is reported (to_double needs finite words)
    bad |= !(df::finite_bits(acc[q][0].s) && df::finite_bits(acc[q][0].c) && df::finite_bits(acc[q][1].s) &&
             df::finite_bits(acc[q][1].c));
    double re = df::to_double(df::F2{acc[q][0].s, acc[q][0].c});
    double im = df::to_double(df::F2{acc[q][1].s, acc[q][1].c});
    for (int grp = 0; grp <= s; ++grp)
      for (int k = 0; k < nk; ++k) {
        const int seg = s_seg[k];
        if (seg < 0) continue;
        const double2 v = reinterpret_cast<const double2*>(part)[((size_t)(i0 + k) * g.S + seg) * (2 * 128 * kNA) +
                                                                  ((size_t)grp * CT + cl) * kNA * M + al * M + bb];
        re += v.x;
        im += v.y;
      }
    bad |= !(isfinite(re) && isfinite(im));
    reinterpret_cast<double2*>(out)[((size_t)s * (n + 1) + c) * MM + (pt * kNA + al) * M + bb] = make_double2(re, im);
  }
  if (bad) atomicOr(status, kStatusNumeric);
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

size_t split_workspace_bytes(int M, int n_max) {
  SplitGeomHost h;
  if (!split_geometry(M, n_max - 1, &h)) return 0;
  const size_t small = (size_t)h.cpt * h.parts * kSmallBytes + (size_t)h.cpt * h.parts * sizeof(int) + 256;
  const size_t part = (size_t)h.G * h.S * 2 * 128 * kNA * 16;
  return small + part + 1024;
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
  e = cudaFuncSetAttribute(split_main, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
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
    split_encode<<<(unsigned)((size_t)(col_tiles - ct_lo) * h.cpt), 256, 0, s>>>(ea);
    ++*launches;
  }
  const int ct_hi = std::min(col_tiles, ct_lo + 1);
  if (r0 > 0 && kc_lo < h.cpt) {
    EncodeArgs ea{g, l.L, l.R, pl, qu, pl_layout.cpt_stride, qs, 0, kc_lo, h.cpt - kc_lo, 0, l.status};
    split_encode<<<(unsigned)((size_t)ct_hi * (h.cpt - kc_lo)), 256, 0, s>>>(ea);
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

cudaError_t launch_history_split(const SplitLaunch& l, cudaStream_t s, int* launches) {
  SplitGeomHost h;
  *launches = 0;
  if (!split_geometry(l.M, l.n, &h)) return cudaErrorInvalidValue;
  SplitGeom g{h.M, h.M * h.M, h.n, h.CT, h.parts, h.cpt, h.tiles, h.U, h.G, h.S, l.w.band_w};
  uint8_t* ws = reinterpret_cast<uint8_t*>(l.work);
  uint8_t* small = ws;
  int* e_small = reinterpret_cast<int*>(small + (size_t)h.cpt * h.parts * kSmallBytes);
  size_t off = ((size_t)h.cpt * h.parts * kSmallBytes + (size_t)h.cpt * h.parts * sizeof(int) + 255) / 256 * 256;
  double* part = reinterpret_cast<double*>(ws + off);
  const size_t need = off + (size_t)h.G * h.S * 2 * 128 * kNA * 16;
  if (need > l.work_bytes) return cudaErrorInvalidValue;

  cudaError_t e = split_prepare();
  if (e != cudaSuccess) return e;
  split_prep<<<dim3(h.cpt, h.parts), 256, 0, s>>>(l.M, l.n, h.parts, l.Sl, l.Sg, l.w, small, e_small);
  ++*launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int smem = (int)sizeof(Smem);
  SplitArgs args{g, l.L, l.R, small, e_small, part, l.status};
  if (l.ev_begin) cudaEventRecord(l.ev_begin, s);
  split_main<<<h.G, kThreads, smem, s>>>(args);
  if (l.ev_end) cudaEventRecord(l.ev_end, s);
  ++*launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  split_reduce2<<<reduce2_grid(h), kRedThreads, 0, s>>>(g, part, l.Sl, l.Sg, l.R, l.w, l.out, l.status);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace kbe
