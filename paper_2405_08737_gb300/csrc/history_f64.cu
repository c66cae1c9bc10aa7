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

#include "kbe_internal.h"

namespace kbe {
namespace {

struct Cd {
  double re, im;
};
__device__ __forceinline__ Cd ld(const double* p) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return Cd{v.x, v.y};
}
// acc += a * b
__device__ __forceinline__ void mac(Cd& acc, Cd a, Cd b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc += a * conj(b)
__device__ __forceinline__ void mac_cj(Cd& acc, Cd a, Cd b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(-a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc -= a * conj(b)
__device__ __forceinline__ void msc_cj(Cd& acc, Cd a, Cd b) {
  acc.re = fma(-a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}

// prep: A1 = w_{n,m} (Sg - Sl), Bl = wbar_m Sl, Bg = wbar_m Sg  (complex, [n+1][M][M])
__global__ void __launch_bounds__(256) history_prep(int MM, int n, const double* __restrict__ Sl,
                                                    const double* __restrict__ Sg, WeightsView w,
                                                    double* __restrict__ A1, double* __restrict__ Bl,
                                                    double* __restrict__ Bg) {
  const int64_t total = (int64_t)(n + 1) * MM;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(e / MM);
    const double wn = w.at(n, m), wb = w.wbar[m];
    const double2 l = reinterpret_cast<const double2*>(Sl)[e];
    const double2 g = reinterpret_cast<const double2*>(Sg)[e];
    reinterpret_cast<double2*>(A1)[e] = make_double2(wn * (g.x - l.x), wn * (g.y - l.y));
    reinterpret_cast<double2*>(Bl)[e] = make_double2(wb * l.x, wb * l.y);
    reinterpret_cast<double2*>(Bg)[e] = make_double2(wb * g.x, wb * g.y);
  }
}

struct PartialArgs {
  int M, MM, n;
  int chunk_len;
  const double* L;
  const double* R;
  const double* Sl;   // raw row n (band points of term 2)
  const double* Sg;
  const double* A1;
  const double* Bl;
  const double* Bg;
  WeightsView w;
  double* dst;        // partials [chunk][2][n+1][MM] or the output when one chunk
};

__global__ void __launch_bounds__(256) history_partial(PartialArgs p) {
  const int M = p.M, MM = p.MM, n = p.n;
  const int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lin >= (int64_t)(n + 1) * MM) return;
  const int c = (int)(lin / MM);
  const int ab = (int)(lin - (int64_t)c * MM);
  const int a = ab / M, b = ab - a * M;
  const int m0 = blockIdx.y * p.chunk_len;
  const int m1 = min(n + 1, m0 + p.chunk_len);

  Cd P{0, 0}, Q{0, 0}, Tl{0, 0}, Tg{0, 0};  // A1 G^<, A1 G^R, term-2 <, term-2 >
  const int band_lo = c - p.w.band_w + 1;    // m >= band_lo: w_{c,m} from the band

  // region m < c: stored block (c, m), read transposed
  const int mA1 = min(m1, c);
  for (int m = m0; m < mA1; ++m) {
    const double* lc = p.L + (tri(c, m) * MM + b * M) * 2;
    const double* rc = p.R + (tri(c, m) * MM + b * M) * 2;
    const double* a1 = p.A1 + ((int64_t)m * MM + a * M) * 2;
    if (m < band_lo) {
      const double* bl = p.Bl + ((int64_t)m * MM + a * M) * 2;
      const double* bg = p.Bg + ((int64_t)m * MM + a * M) * 2;
#pragma unroll 4
      for (int x = 0; x < M; ++x) {
        const Cd l = ld(lc + 2 * x), r = ld(rc + 2 * x), s1 = ld(a1 + 2 * x);
        // G^<(m,c)_xb = -conj(L(c,m)_bx);  G^R part: -conj(R(c,m)_bx)
        msc_cj(P, s1, l);
        msc_cj(Q, s1, r);
        // G^A(m,c)_xb = conj(R(c,m)_bx)
        mac_cj(Tl, ld(bl + 2 * x), r);
        mac_cj(Tg, ld(bg + 2 * x), r);
      }
    } else {
      const double wcm = p.w.at(c, m);
      const double* sl = p.Sl + ((int64_t)m * MM + a * M) * 2;
      const double* sg = p.Sg + ((int64_t)m * MM + a * M) * 2;
      for (int x = 0; x < M; ++x) {
        const Cd l = ld(lc + 2 * x), r = ld(rc + 2 * x), s1 = ld(a1 + 2 * x);
        msc_cj(P, s1, l);
        msc_cj(Q, s1, r);
        Cd vl = ld(sl + 2 * x), vg = ld(sg + 2 * x);
        vl.re *= wcm; vl.im *= wcm; vg.re *= wcm; vg.im *= wcm;
        mac_cj(Tl, vl, r);
        mac_cj(Tg, vg, r);
      }
    }
  }
  // diagonal m == c
  if (c >= m0 && c < m1) {
    const int m = c;
    const double wcc = p.w.at(c, c);
    const double* lb = p.L + tri(c, c) * MM * 2;
    const double* rb = p.R + tri(c, c) * MM * 2;
    const double* a1 = p.A1 + ((int64_t)m * MM + a * M) * 2;
    const double* sl = p.Sl + ((int64_t)m * MM + a * M) * 2;
    const double* sg = p.Sg + ((int64_t)m * MM + a * M) * 2;
    for (int x = 0; x < M; ++x) {
      const Cd s1 = ld(a1 + 2 * x);
      mac(P, s1, ld(lb + 2 * (x * M + b)));
      mac(Q, s1, ld(rb + 2 * (x * M + b)));
      const Cd ra = ld(rb + 2 * (b * M + x));  // G^A(c,c)_xb = conj(R(c,c)_bx)
      Cd vl = ld(sl + 2 * x), vg = ld(sg + 2 * x);
      vl.re *= wcc; vl.im *= wcc; vg.re *= wcc; vg.im *= wcc;
      mac_cj(Tl, vl, ra);
      mac_cj(Tg, vg, ra);
    }
  }
  // region m > c: stored block (m, c), read directly
  for (int m = max(m0, c + 1); m < m1; ++m) {
    const double* lm = p.L + (tri(m, c) * MM + b) * 2;
    const double* rm = p.R + (tri(m, c) * MM + b) * 2;
    const double* a1 = p.A1 + ((int64_t)m * MM + a * M) * 2;
#pragma unroll 4
    for (int x = 0; x < M; ++x) {
      const Cd s1 = ld(a1 + 2 * x);
      mac(P, s1, ld(lm + 2 * x * M));
      mac(Q, s1, ld(rm + 2 * x * M));
    }
  }
  // I^< = P + Tl,  I^> = P + Q + Tg
  double2* d = reinterpret_cast<double2*>(p.dst);
  const int64_t stride_s = (int64_t)(n + 1) * MM;
  const int64_t base = (int64_t)blockIdx.y * 2 * stride_s + lin;
  d[base] = make_double2(P.re + Tl.re, P.im + Tl.im);
  d[base + stride_s] = make_double2(P.re + Q.re + Tg.re, P.im + Q.im + Tg.im);
}

// out = sum over chunks in order; flags non-finite results.
__global__ void __launch_bounds__(256) history_reduce(int64_t per_chunk, int nchunk, const double2* __restrict__ part,
                                                      double2* __restrict__ out, int* status) {
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < per_chunk;
       e += (int64_t)gridDim.x * blockDim.x) {
    double2 s = part[e];
    for (int k = 1; k < nchunk; ++k) {
      const double2 v = part[(int64_t)k * per_chunk + e];
      s.x += v.x;
      s.y += v.y;
    }
    bad |= !(isfinite(s.x) && isfinite(s.y));
    out[e] = s;
  }
  if (bad) atomicOr(status, kStatusNumeric);
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

// Workspace layout (doubles): A1, Bl, Bg: 3 x (n+1) MM complex; then the
// split partials nchunk x 2 x (n+1) MM complex.
cudaError_t launch_history_f64(const HistoryArgs& a, cudaStream_t s, int* launches) {
  const int M = a.M, MM = M * M, n = a.n;
  const int64_t row = (int64_t)(n + 1) * MM;       // complex entries per s
  const int64_t outputs = row;                     // threads of one chunk
  // Enough threads for full occupancy: 152 SMs x 2048 threads.
  int64_t want = (152LL * 2048 + outputs - 1) / outputs;
  int nchunk = (int)(want < 1 ? 1 : (want > kMaxSplit ? kMaxSplit : want));
  if (nchunk > n + 1) nchunk = n + 1;
  // the partials must fit the workspace
  const size_t prep_bytes = (size_t)3 * row * 16;
  while (nchunk > 1 && prep_bytes + (size_t)nchunk * 2 * row * 16 > a.part_bytes) --nchunk;
  if (prep_bytes + (nchunk > 1 ? (size_t)nchunk * 2 * row * 16 : 0) > a.part_bytes) return cudaErrorInvalidValue;
  const int chunk_len = (n + 1 + nchunk - 1) / nchunk;
  nchunk = (n + 1 + chunk_len - 1) / chunk_len;

  double* A1 = a.part;
  double* Bl = A1 + 2 * row;
  double* Bg = Bl + 2 * row;
  double* partials = Bg + 2 * row;
  int nl = 0;
  history_prep<<<grid_for(row, 152 * 8), 256, 0, s>>>(MM, n, a.Sl, a.Sg, a.w, A1, Bl, Bg);
  ++nl;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { *launches = nl; return e; }
  PartialArgs p{M, MM, n, chunk_len, a.L, a.R, a.Sl, a.Sg, A1, Bl, Bg, a.w,
                nchunk == 1 ? a.out : partials};
  dim3 grid((unsigned)((outputs + 255) / 256), (unsigned)nchunk);
  if (a.ev_begin) cudaEventRecord(a.ev_begin, s);
  history_partial<<<grid, 256, 0, s>>>(p);
  if (a.ev_end) cudaEventRecord(a.ev_end, s);
  ++nl;
  e = cudaGetLastError();
  if (e != cudaSuccess) { *launches = nl; return e; }
  if (nchunk > 1) {
    history_reduce<<<grid_for(2 * row, 152 * 8), 256, 0, s>>>(2 * row, nchunk, (const double2*)partials,
                                                              (double2*)a.out, a.status);
  } else {
    finite_check<<<grid_for(2 * row, 152 * 8), 256, 0, s>>>(2 * row, (const double2*)a.out, a.status);
  }
  ++nl;
  *launches = nl;
  return cudaGetLastError();
}

}  // namespace kbe
