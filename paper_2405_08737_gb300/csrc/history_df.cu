// history_df.cu -- history slice of Eq. (KBE2) (Sec. 2) in double-float
// arithmetic on the FP32 pipe (precision KBE_DF64).
//
// The same sums as history_f64.cu,
//   I^<(n,c) = sum_m A1[m] G^<(m,c) + sum_{m<=c} B^<[m] G^A(m,c),
//   I^>(n,c) = sum_m A1[m] G^>(m,c) + sum_{m<=c} B^>[m] G^A(m,c),
// with A1[m] = w_{n,m} (S^> - S^<)[m], B^s[m] = wbar_m S^s[m] (w_{c,m} S^s[m]
// in the band m > c - K - 1), G^> = G^< + R below and on the diagonal, and
// the symmetries G^s(m,c) = -G^s(c,m)^+ (m < c), G^A(m,c) = R(c,m)^+.
//
// GB300 issues 64 FP32 operations per FP64 operation, so a complex
// multiply-add done as four double-float products (each hi*hi, its FMA
// error and the two cross terms, about 2^-47 relative) with Ogita-Rump-Oishi
// compensated accumulation (a TwoSum per term, the errors in a float tail)
// costs about 48 FP32 operations where FP64 needs 4 DFMA: at the two pipes'
// rates the slice runs about four times faster than on the FP64 pipe, with
// an error of order 1e-14 of the terms' sizes (Sec. 3.2's quadrature and
// the history are FP64 inputs, converted once per use to hi + lo floats).
//
// Layout.  A prep kernel forms A1, B^<, B^> in FP64 (as history_prep) and
// stores them as double-float (float4: re.hi, re.lo, im.hi, im.lo) rows.
// One thread owns one output column entry (c, b) for a group of 2 values of
// a and both s: each history entry it loads is converted once and used for
// its 2 values of a; the self-energy operands are shared by the warp
// (broadcast loads).  The history index m is split into chunks across
// grid.y; per-chunk partials go to the workspace as FP64 and the FP64
// reduction adds them in chunk order (deterministic).

#include <algorithm>

#include "dfloat.cuh"
#include "row_kernels.cuh"

namespace kbe {
namespace {

constexpr int kNA = 2;          // values of a per thread
constexpr int kDfBlock = 128;   // threads per block
// shared memory of a history_df_tiled block: 32 KB (two history points per
// tile at M = 8, seven blocks per SM) measured faster than 64 KB (four
// points, three blocks): 2.14 against 2.72 ms for the slice n = 767, M = 8
constexpr size_t kTileSmem = 32 * 1024;

struct DfArgs {
  int M, MM, n, AG;             // AG = ceil(M / kNA) groups of a
  int chunk_len;
  const double* L;
  const double* R;
  const double* Sl;             // raw row n (band points of term 2)
  const double* Sg;
  const float4* A1;             // double-float rows [n+1][M][M]
  const float4* Bl;
  const float4* Bg;
  WeightsView w;
  double* dst;                  // partials [chunk][2][n+1][MM] or the output
};

using df::Acc;
using df::c2f;
using df::cconj;
using df::cmac;
using df::cneg;
__device__ __forceinline__ float4 cadd(float4 a, float4 b) { return df::cadd4(a, b); }

__global__ void __launch_bounds__(256) history_df_prep(int MM, int n, const double* __restrict__ Sl,
                                                       const double* __restrict__ Sg, WeightsView w,
                                                       float4* __restrict__ A1, float4* __restrict__ Bl,
                                                       float4* __restrict__ Bg) {
  const int64_t total = (int64_t)(n + 1) * MM;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(e / MM);
    const double wn = w.at(n, m), wb = w.wbar[m];
    const double2 l = reinterpret_cast<const double2*>(Sl)[e];
    const double2 g = reinterpret_cast<const double2*>(Sg)[e];
    A1[e] = c2f(make_double2(wn * (g.x - l.x), wn * (g.y - l.y)));
    Bl[e] = c2f(make_double2(wb * l.x, wb * l.y));
    Bg[e] = c2f(make_double2(wb * g.x, wb * g.y));
  }
}

__global__ void __launch_bounds__(kDfBlock) history_df_partial(DfArgs p) {
  const int M = p.M, MM = p.MM, n = p.n, AG = p.AG;
  // column blocks from the last column down: the heavier blocks of each
  // chunk (columns past it carry both terms) start first
  const int64_t t = (int64_t)(gridDim.x - 1 - blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= (int64_t)(n + 1) * AG * M) return;
  const int c = (int)(t / ((int64_t)AG * M));
  const int r = (int)(t - (int64_t)c * AG * M);
  const int ag = r / M, b = r - ag * M;
  const int a0 = ag * kNA;
  const int na = min(kNA, M - a0);
  const int chunk = blockIdx.y;
  const int m0 = chunk * p.chunk_len;
  const int m1 = min(n + 1, m0 + p.chunk_len);
  const int band_lo = c - p.w.band_w + 1;  // m >= band_lo: w_{c,m} from the band

  Acc lr[kNA], li[kNA], gr[kNA], gi[kNA];  // I^< and I^> (re, im)
#pragma unroll
  for (int k = 0; k < kNA; ++k) lr[k] = li[k] = gr[k] = gi[k] = Acc{0.f, 0.f};
  const double2* L = reinterpret_cast<const double2*>(p.L);
  const double2* R = reinterpret_cast<const double2*>(p.R);

  for (int m = m0; m < m1; ++m) {
    const bool below = m > c, diag = m == c;
    const bool band = !below && m >= band_lo;
    const double wcm = band ? p.w.at(c, m) : 0.0;
    // this thread's column b of G(m,c): block (m,c) row x for m >= c; block
    // (c,m) row b, transposed and conjugated, for m < c
    const int64_t blk = below || diag ? tri(m, c) * MM : tri(c, m) * MM;
    for (int x = 0; x < M; ++x) {
      float4 gl, gs, ga;
      if (below || diag) {
        gl = c2f(L[blk + x * M + b]);
        const float4 rr = c2f(R[blk + x * M + b]);
        gs = cadd(gl, rr);                                 // G^>(m,c) = L + R
        ga = diag ? cconj(c2f(R[blk + b * M + x])) : rr;   // G^A(c,c)_xb = conj(R(c,c)_bx)
      } else {
        const float4 l = c2f(L[blk + b * M + x]), rr = c2f(R[blk + b * M + x]);
        gl = cneg(cconj(l));                               // G^<(m,c)_xb = -conj(L(c,m)_bx)
        gs = cneg(cconj(cadd(l, rr)));                     // G^>(m,c)_xb = -conj((L+R)(c,m)_bx)
        ga = cconj(rr);                                    // G^A(m,c)_xb = conj(R(c,m)_bx)
      }
      const float4* a1 = p.A1 + ((int64_t)m * M + a0) * M + x;
#pragma unroll
      for (int k = 0; k < kNA; ++k) {
        if (k < na) {
          const float4 s1 = a1[(int64_t)k * M];
          cmac(lr[k], li[k], s1, gl);
          cmac(gr[k], gi[k], s1, gs);
        }
      }
      if (below) continue;
      if (!band) {
        const float4* bl = p.Bl + ((int64_t)m * M + a0) * M + x;
        const float4* bg = p.Bg + ((int64_t)m * M + a0) * M + x;
#pragma unroll
        for (int k = 0; k < kNA; ++k) {
          if (k < na) {
            cmac(lr[k], li[k], bl[(int64_t)k * M], ga);
            cmac(gr[k], gi[k], bg[(int64_t)k * M], ga);
          }
        }
      } else {
        const double2* sl = reinterpret_cast<const double2*>(p.Sl) + ((int64_t)m * M + a0) * M + x;
        const double2* sg = reinterpret_cast<const double2*>(p.Sg) + ((int64_t)m * M + a0) * M + x;
#pragma unroll
        for (int k = 0; k < kNA; ++k) {
          if (k < na) {
            const double2 vl = sl[(int64_t)k * M], vg = sg[(int64_t)k * M];
            cmac(lr[k], li[k], c2f(make_double2(wcm * vl.x, wcm * vl.y)), ga);
            cmac(gr[k], gi[k], c2f(make_double2(wcm * vg.x, wcm * vg.y)), ga);
          }
        }
      }
    }
  }
  double2* d = reinterpret_cast<double2*>(p.dst);
  const int64_t stride_s = (int64_t)(n + 1) * MM;
  const int64_t base = (int64_t)chunk * 2 * stride_s + (int64_t)c * MM + b;
#pragma unroll
  for (int k = 0; k < kNA; ++k) {
    if (k < na) {
      const int64_t e = base + (int64_t)(a0 + k) * M;
      d[e] = make_double2((double)lr[k].s + (double)lr[k].c, (double)li[k].s + (double)li[k].c);
      d[e + stride_s] = make_double2((double)gr[k].s + (double)gr[k].c, (double)gi[k].s + (double)gi[k].c);
    }
  }
}

// Shared-memory form for M <= 32: a block owns CB output columns and AGB
// groups of a; per tile of TM history points it loads the G blocks its
// columns read and the operand rows of its values of a once, converts them
// once (instead of once per thread that reads them), and every thread then
// reads its operands from shared memory.  Same arithmetic in the same order
// per output as history_df_partial.
struct TileGeom {
  int CB, AGB, TM;    // columns, groups of a, history points per block tile
  int col_tiles, ag_tiles;
};

__global__ void __launch_bounds__(kDfBlock) history_df_tiled(DfArgs p, TileGeom tg) {
  extern __shared__ float4 sm[];
  const int M = p.M, MM = p.MM, n = p.n, AG = p.AG;
  const int CB = tg.CB, AGB = tg.AGB, TM = tg.TM, NAB = AGB * kNA;
  float4* sG = sm;                                  // [TM][CB][3][MM]: G^<, G^>, G^A as [x][b]
  float4* sS = sm + (size_t)TM * CB * 3 * MM;       // [TM][3][NAB][M]: A1, B^<, B^> rows
  // column tiles from the last one down (heavier tiles of each chunk first)
  const int bx = (int)(gridDim.x - 1 - blockIdx.x);
  const int ct = bx / tg.ag_tiles, at = bx - ct * tg.ag_tiles;
  const int c_base = ct * CB, ag_base = at * AGB;
  const int a_base = ag_base * kNA;
  const int tid = threadIdx.x;
  const int cl = tid / (AGB * M), rr0 = tid - cl * AGB * M;
  const int agl = rr0 / M, b = rr0 - agl * M;
  const int c = c_base + cl;
  const int a0 = (ag_base + agl) * kNA;
  const bool live = cl < CB && c <= n && ag_base + agl < AG;
  const int na = live ? min(kNA, M - a0) : 0;
  const int chunk = blockIdx.y;
  const int m0 = chunk * p.chunk_len;
  const int m1 = min(n + 1, m0 + p.chunk_len);
  const int band_lo = c - p.w.band_w + 1;
  const double2* L = reinterpret_cast<const double2*>(p.L);
  const double2* R = reinterpret_cast<const double2*>(p.R);
  const int nab = min(NAB, M - a_base);  // values of a of this block

  Acc lr[kNA], li[kNA], gr[kNA], gi[kNA];
#pragma unroll
  for (int k = 0; k < kNA; ++k) lr[k] = li[k] = gr[k] = gi[k] = Acc{0.f, 0.f};

  for (int mt = m0; mt < m1; mt += TM) {
    const int tm = min(TM, m1 - mt);
    __syncthreads();
    // G blocks of the block's columns: (m, c) read directly for m >= c,
    // (c, m) transposed for m < c
    const int g_items = tm * CB * MM;
    for (int i = tid; i < g_items; i += kDfBlock) {
      const int mi = i / (CB * MM), r = i - mi * CB * MM;
      const int cc = r / MM, e = r - cc * MM;
      const int m = mt + mi, col = c_base + cc;
      if (col > n) continue;
      float4* dst = sG + ((size_t)(mi * CB + cc) * 3) * MM;
      if (m >= col) {
        const int64_t blk = tri(m, col) * MM;
        const float4 l = c2f(L[blk + e]), rv = c2f(R[blk + e]);
        dst[e] = l;
        dst[MM + e] = cadd(l, rv);
        if (m == col) {  // G^A(c,c)_xb = conj(R(c,c)_bx)
          const int x = e / M, bb = e - x * M;
          dst[2 * MM + e] = cconj(c2f(R[blk + bb * M + x]));
        }
      } else {
        const int64_t blk = tri(col, m) * MM;   // stored entry (b, x) at e = b M + x
        const int bb = e / M, x = e - bb * M;
        const float4 l = c2f(L[blk + e]), rv = c2f(R[blk + e]);
        const int et = x * M + bb;
        dst[et] = cneg(cconj(l));
        dst[MM + et] = cneg(cconj(cadd(l, rv)));
        dst[2 * MM + et] = cconj(rv);
      }
    }
    // operand rows of the block's values of a
    const int s_items = tm * 3 * nab * M;
    for (int i = tid; i < s_items; i += kDfBlock) {
      const int mi = i / (3 * nab * M), r = i - mi * 3 * nab * M;
      const int v = r / (nab * M), e = r - v * nab * M;   // e = (a - a_base) M + x
      const float4* src = v == 0 ? p.A1 : (v == 1 ? p.Bl : p.Bg);
      sS[((size_t)(mi * 3 + v) * NAB) * M + e] = src[((int64_t)(mt + mi) * M + a_base) * M + e];
    }
    __syncthreads();
    if (!live) continue;
    for (int mi = 0; mi < tm; ++mi) {
      const int m = mt + mi;
      const bool below = m > c;
      const bool band = !below && m >= band_lo;
      const double wcm = band ? p.w.at(c, m) : 0.0;
      const float4* g = sG + ((size_t)(mi * CB + cl) * 3) * MM + b;
      const float4* s1p = sS + ((size_t)(mi * 3 + 0) * NAB + (a0 - a_base)) * M;
      const float4* blp = sS + ((size_t)(mi * 3 + 1) * NAB + (a0 - a_base)) * M;
      const float4* bgp = sS + ((size_t)(mi * 3 + 2) * NAB + (a0 - a_base)) * M;
      for (int x = 0; x < M; ++x) {
        const float4 gl = g[x * M], gs = g[MM + x * M];
#pragma unroll
        for (int k = 0; k < kNA; ++k) {
          if (k < na) {
            const float4 s1 = s1p[k * M + x];
            cmac(lr[k], li[k], s1, gl);
            cmac(gr[k], gi[k], s1, gs);
          }
        }
        if (below) continue;
        const float4 ga = g[2 * MM + x * M];
        if (!band) {
#pragma unroll
          for (int k = 0; k < kNA; ++k) {
            if (k < na) {
              cmac(lr[k], li[k], blp[k * M + x], ga);
              cmac(gr[k], gi[k], bgp[k * M + x], ga);
            }
          }
        } else {
          const double2* sl = reinterpret_cast<const double2*>(p.Sl) + ((int64_t)m * M + a0) * M + x;
          const double2* sg = reinterpret_cast<const double2*>(p.Sg) + ((int64_t)m * M + a0) * M + x;
#pragma unroll
          for (int k = 0; k < kNA; ++k) {
            if (k < na) {
              const double2 vl = sl[(int64_t)k * M], vg = sg[(int64_t)k * M];
              cmac(lr[k], li[k], c2f(make_double2(wcm * vl.x, wcm * vl.y)), ga);
              cmac(gr[k], gi[k], c2f(make_double2(wcm * vg.x, wcm * vg.y)), ga);
            }
          }
        }
      }
    }
  }
  if (!live) return;
  double2* d = reinterpret_cast<double2*>(p.dst);
  const int64_t stride_s = (int64_t)(n + 1) * MM;
  const int64_t base = (int64_t)chunk * 2 * stride_s + (int64_t)c * MM + b;
#pragma unroll
  for (int k = 0; k < kNA; ++k) {
    if (k < na) {
      const int64_t e = base + (int64_t)(a0 + k) * M;
      d[e] = make_double2((double)lr[k].s + (double)lr[k].c, (double)li[k].s + (double)li[k].c);
      d[e + stride_s] = make_double2((double)gr[k].s + (double)gr[k].c, (double)gi[k].s + (double)gi[k].c);
    }
  }
}

// Block tiling of history_df_tiled for M orbitals and n + 1 columns, within
// smem_max bytes of shared memory; false for orbital counts it does not take.
bool tile_geom(int M, int n, size_t smem_max, TileGeom* tg, size_t* smem) {
  if (M > 32) return false;
  const int AG = (M + kNA - 1) / kNA, TPC = AG * M;
  if (TPC <= kDfBlock) {
    tg->CB = kDfBlock / TPC;
    tg->AGB = AG;
  } else {
    tg->CB = 1;
    tg->AGB = kDfBlock / M;
  }
  const size_t per_m = ((size_t)tg->CB * 3 * M * M + (size_t)3 * tg->AGB * kNA * M) * sizeof(float4);
  tg->TM = (int)std::max<size_t>(1, std::min<size_t>(8, smem_max / per_m));
  if (per_m > smem_max) return false;
  *smem = per_m * tg->TM;
  tg->col_tiles = (n + 1 + tg->CB - 1) / tg->CB;
  tg->ag_tiles = (AG + tg->AGB - 1) / tg->AGB;
  return true;
}

inline unsigned grid_for(int64_t n, int64_t cap) {
  int64_t b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

// Workspace as launch_history_f64: the three double-float operand rows take
// the places of A1, Bl, Bg (16 bytes per complex either way), then the
// per-chunk partials.
cudaError_t launch_history_df(const HistoryArgs& a, cudaStream_t s, int* launches) {
  const int M = a.M, MM = M * M, n = a.n;
  const int AG = (M + kNA - 1) / kNA;
  const int64_t row = (int64_t)(n + 1) * MM;
  const int64_t threads = (int64_t)(n + 1) * AG * M;
  // enough threads for full occupancy, and chunks of at most ~32 history
  // points so that a block's work stays short
  int64_t want = std::max<int64_t>(((int64_t)sm_count() * 2048 + threads - 1) / threads, (n + 1 + 31) / 32);
  int nchunk = (int)std::min<int64_t>(std::max<int64_t>(want, 1), kMaxSplit);
  if (nchunk > n + 1) nchunk = n + 1;
  const size_t prep_bytes = (size_t)3 * row * 16;
  while (nchunk > 1 && prep_bytes + (size_t)nchunk * 2 * row * 16 > a.part_bytes) --nchunk;
  if (prep_bytes + (nchunk > 1 ? (size_t)nchunk * 2 * row * 16 : 0) > a.part_bytes) return cudaErrorInvalidValue;
  const int chunk_len = (n + 1 + nchunk - 1) / nchunk;
  nchunk = (n + 1 + chunk_len - 1) / chunk_len;

  float4* A1 = reinterpret_cast<float4*>(a.part);
  float4* Bl = A1 + row;
  float4* Bg = Bl + row;
  double* partials = a.part + 6 * row;
  int nl = 0;
  history_df_prep<<<grid_for(row, sm_count() * 8), 256, 0, s>>>(MM, n, a.Sl, a.Sg, a.w, A1, Bl, Bg);
  ++nl;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { *launches = nl; return e; }
  DfArgs p{M, MM, n, AG, chunk_len, a.L, a.R, a.Sl, a.Sg, A1, Bl, Bg, a.w, nchunk == 1 ? a.out : partials};
  TileGeom tg;
  size_t smem = 0;
  const bool tiled = tile_geom(M, n, kTileSmem, &tg, &smem);
  // (no attribute call at or below the default 48 KB, so that the launch can
  // be recorded in a graph capture)
  if (tiled && kTileSmem > 48 * 1024 &&
      (e = cudaFuncSetAttribute(history_df_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kTileSmem)) != cudaSuccess) {
    *launches = nl;
    return e;
  }
  if (a.ev_begin) cudaEventRecord(a.ev_begin, s);
  if (tiled) {
    dim3 grid((unsigned)((int64_t)tg.col_tiles * tg.ag_tiles), (unsigned)nchunk);
    history_df_tiled<<<grid, kDfBlock, smem, s>>>(p, tg);
  } else {
    dim3 grid((unsigned)((threads + kDfBlock - 1) / kDfBlock), (unsigned)nchunk);
    history_df_partial<<<grid, kDfBlock, 0, s>>>(p);
  }
  if (a.ev_end) cudaEventRecord(a.ev_end, s);
  ++nl;
  if ((e = cudaGetLastError()) != cudaSuccess) { *launches = nl; return e; }
  int nr = 0;
  e = launch_history_finish(nchunk, row, partials, a.out, a.status, s, &nr);
  *launches = nl + nr;
  return e;
}

}  // namespace kbe
