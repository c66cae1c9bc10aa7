// row_kernels.cuh -- per-entry bodies of the row kernels (self-energy,
// history slice, predictor, Fock matrix, right-hand side, corrector), shared
// by the single-system launches and the batched persistent launches so that
// both run the same arithmetic in the same order.
#pragma once

#include "dfloat.cuh"
#include "kbe_internal.h"

namespace kbe {
namespace rk {

// floor(x / d) for 0 <= x, 0 < d: a 32-bit division where x fits (the
// 64-bit one is a long instruction sequence on the latency path of small
// rows); the same quotient either way.
__device__ __forceinline__ int div_idx(int64_t x, int d) {
  return x <= 0x7fffffff ? (int)((unsigned)x / (unsigned)d) : (int)(x / d);
}

struct Cd {
  double re, im;
};
// kReadOnly: through the read-only cache (data nobody writes during the
// launch); otherwise a plain load, which sees what other blocks of the same
// launch wrote before a device-wide barrier (release/acquire) that it follows.
template <bool kReadOnly = true>
__device__ __forceinline__ Cd ld(const double* p) {
  const double2 v = kReadOnly ? __ldg(reinterpret_cast<const double2*>(p)) : *reinterpret_cast<const double2*>(p);
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

__device__ __forceinline__ double2 ldd(const double* p) { return *reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ void std2(double* p, double2 v) { *reinterpret_cast<double2*>(p) = v; }

// ------------------------------------------------------------ self-energy --
// Eq. (SE) with a local interaction, entry e = (block, ab) of a run of
// blocks (see sigma.cu); `diag` says whether the entry's block is a diagonal
// block, and then the third factor is the stored transposed entry.  The
// products run in double-float on the FP32 pipe (dfloat.cuh; about 2^-47
// relative per operation), because ~40 FP64 instructions per 64-byte entry
// would hold the kernel far below memory bandwidth on this part.  Only
// G^> = R + L (where L and R may cancel), U_a U_b and the final hi + lo stay
// in FP64: 7 FP64 instructions per entry.  Off the diagonal, with
// q = -U_a U_b g conj(l):  S^> = g q,  S^< = l conj(q).
// Returns false on a non-finite result.
__device__ __forceinline__ df::C2 ld_c2(double2 v) {
  return df::C2{df::from_double_fast(v.x), df::from_double_fast(v.y)};
}
__device__ __forceinline__ double2 to_d2(df::C2 a) { return make_double2(df::to_double(a.re), df::to_double(a.im)); }

// uu = U_a U_b of entry ab = (a, b) in double-float (the caller may keep it
// while ab stays the same).
__device__ __forceinline__ df::F2 sigma_uu(int M, int ab, const double* __restrict__ U) {
  const int a = ab / M, b = ab - a * M;
  return df::from_double_fast(U[a] * U[b]);
}

// The same with the entry's L and R values already loaded (l64, r64), so
// that a caller can have the next entry's loads in flight meanwhile.
__device__ __forceinline__ bool sigma_entry_v(int M, int64_t e, int ab, bool diag, df::F2 uu, double2 l64,
                                              double2 r64, const double2* __restrict__ L,
                                              const double2* __restrict__ R, double2* __restrict__ Sl,
                                              double2* __restrict__ Sg) {
  const df::C2 l = ld_c2(l64);
  const df::C2 g = ld_c2(make_double2(r64.x + l64.x, r64.y + l64.y));
  df::C2 sg, sl;
  if (!diag) {
    const df::C2 q = df::cscale(df::neg(uu), df::cmul_cj(g, l));  // -uu g conj(l)
    sg = df::cmul(g, q);
    sl = df::cmul_cj(l, q);
  } else {
    const int a = ab / M, b = ab - a * M;
    const int64_t eb = e - ab + b * M + a;  // entry (b,a) of the same block
    const double2 lt64 = L[eb], rt64 = R[eb];
    const df::C2 lt = ld_c2(lt64);
    const df::C2 gt = ld_c2(make_double2(rt64.x + lt64.x, rt64.y + lt64.y));
    sg = df::cmul(df::cscale(uu, df::cmul(g, g)), lt);
    sl = df::cmul(df::cscale(uu, df::cmul(l, l)), gt);
  }
  Sg[e] = to_d2(sg);
  Sl[e] = to_d2(sl);
  // hi + lo is finite exactly when hi is: x - x is 0 for finite x, nan otherwise
  const float z = (sg.re.hi - sg.re.hi) + (sg.im.hi - sg.im.hi) + (sl.re.hi - sl.re.hi) + (sl.im.hi - sl.im.hi);
  return z == 0.0f;
}
__device__ __forceinline__ bool sigma_entry(int M, int64_t e, int ab, bool diag, df::F2 uu,
                                            const double2* __restrict__ L, const double2* __restrict__ R,
                                            double2* __restrict__ Sl, double2* __restrict__ Sg) {
  return sigma_entry_v(M, e, ab, diag, uu, L[e], R[e], L, R, Sl, Sg);
}

// ---------------------------------------------------------- history slice --
// prep entry e of row n: A1 = w_{n,m} (Sg - Sl), Bl = wbar_m Sl, Bg = wbar_m Sg
__device__ __forceinline__ void history_prep_entry(int MM, int n, int64_t e, const double* __restrict__ Sl,
                                                   const double* __restrict__ Sg, const WeightsView& w,
                                                   double* __restrict__ A1, double* __restrict__ Bl,
                                                   double* __restrict__ Bg) {
  const int m = div_idx(e, MM);
  const double wn = w.at(n, m), wb = w.wbar[m];
  const double2 l = reinterpret_cast<const double2*>(Sl)[e];
  const double2 g = reinterpret_cast<const double2*>(Sg)[e];
  reinterpret_cast<double2*>(A1)[e] = make_double2(wn * (g.x - l.x), wn * (g.y - l.y));
  reinterpret_cast<double2*>(Bl)[e] = make_double2(wb * l.x, wb * l.y);
  reinterpret_cast<double2*>(Bg)[e] = make_double2(wb * g.x, wb * g.y);
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
  // stored rows whose blocks contribute (a band of the triangle, one rank's
  // share of a slice split across devices); all rows by default
  int band_lo = 0;
  int band_hi = 0x7fffffff;
};

// Output entry lin = (c, a, b) of the history slice over history points
// m in chunk `chunk`; writes I^< and I^> partials of that chunk.  The
// operand loads take the path of ld<kReadOnly>; the arithmetic is the same.
template <bool kReadOnly = true>
__device__ __forceinline__ void history_partial_entry(const PartialArgs& p, int64_t lin, int chunk) {
  const auto ld = [](const double* q) { return rk::ld<kReadOnly>(q); };
  const int M = p.M, MM = p.MM, n = p.n;
  const int c = kReadOnly ? (int)(lin / MM) : div_idx(lin, MM);  // the bulk kernels keep their code
  const int ab = (int)(lin - (int64_t)c * MM);
  const int a = ab / M, b = ab - a * M;
  const int m0 = chunk * p.chunk_len;
  const int m1 = min(n + 1, m0 + p.chunk_len);

  Cd P{0, 0}, Q{0, 0}, Tl{0, 0}, Tg{0, 0};  // A1 G^<, A1 G^R, term-2 <, term-2 >
  const int band_lo = c - p.w.band_w + 1;    // m >= band_lo: w_{c,m} from the band
  // blocks of row c (m <= c) count when row c is in the stored-row band;
  // blocks of rows m > c when row m is
  const bool row_c = c >= p.band_lo && c < p.band_hi;

  // region m < c: stored block (c, m), read transposed
  const int mA1 = row_c ? min(m1, c) : m0;
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
  if (row_c && c >= m0 && c < m1) {
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
  for (int m = max(max(m0, c + 1), p.band_lo); m < min(m1, p.band_hi); ++m) {
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
  const int64_t base = (int64_t)chunk * 2 * stride_s + lin;
  d[base] = make_double2(P.re + Tl.re, P.im + Tl.im);
  d[base + stride_s] = make_double2(P.re + Q.re + Tg.re, P.im + Q.im + Tg.im);
}

// Ordered sum over the chunks of entry e; returns false if non-finite.
__device__ __forceinline__ bool history_reduce_entry(int64_t per_chunk, int nchunk, int64_t e,
                                                     const double2* __restrict__ part, double2* __restrict__ out) {
  double2 s = part[e];
  for (int k = 1; k < nchunk; ++k) {
    const double2 v = part[(int64_t)k * per_chunk + e];
    s.x += v.x;
    s.y += v.y;
  }
  out[e] = s;
  return isfinite(s.x) && isfinite(s.y);
}

// ----------------------------------------------------------------- stepper --
__device__ __forceinline__ const double* ring_at(const StepArgs& a, int j, int s, int c, int ab) {
  const int MM = a.M * a.M;
  const int64_t slot = (j - a.f_base) % a.f_rows;
  return a.F + (((slot * 2 + s) * a.n_max + c) * MM + ab) * 2;
}

// eps(t_n) = h0 + E(t_n) diag(v) + diag(U_a Im L(n,n)_aa), entry ab
__device__ __forceinline__ void fock_entry(const StepArgs& a, int ab) {
  const int M = a.M, MM = M * M;
  const double* Lnn = a.L + tri(a.n, a.n) * MM * 2;
  const int i = ab / M, j = ab - i * M;
  double2 e = ldd(a.h0 + 2 * ab);
  if (!a.HF) {
    if (i == j) e.x += a.field * a.v[i] + a.U[i] * Lnn[2 * ab + 1];
  } else {
    // Eq. (eps): eps_ij = h_ij(t) + i sum_ba (U_iabj - 2 U_ijba) G^<_ba(t,t)
    if (i == j) e.x += a.field * a.v[i];
    const double* hf = a.HF + (int64_t)ab * MM;
    double sr = 0.0, si = 0.0;
    for (int k = 0; k < MM; ++k) {
      sr = fma(hf[k], Lnn[2 * k], sr);
      si = fma(hf[k], Lnn[2 * k + 1], si);
    }
    e.x -= si;
    e.y += sr;
  }
  std2(a.eps + 2 * ab, e);
}

// predictor (corrector = false) or corrector (corrector = true) for entry
// lin = (c, a, b) of row n.
__device__ __forceinline__ void adams_entry(const StepArgs& a, int64_t lin, bool corrector) {
  const int M = a.M, MM = M * M, n = a.n;
  const int c = div_idx(lin, MM), ab = (int)(lin - (int64_t)c * MM);
  const int ia = ab / M, ib = ab - ia * M;
  const double* wt = corrector ? a.corr : a.pred;
  const int extra = corrector ? 1 : 0;  // the corrector also uses the node t_n
  double* Ln = a.L + (tri(n, c) * MM + ab) * 2;
  double* Rn = a.R + (tri(n, c) * MM + ab) * 2;
  if (c < n) {
    const int q = min(a.kn, n - c);
    const double* w = wt + (q - 1) * kWTab;
    const double2 l0 = ldd(a.L + (tri(n - 1, c) * MM + ab) * 2);
    const double2 r0 = ldd(a.R + (tri(n - 1, c) * MM + ab) * 2);
    double2 gl = l0, gg = make_double2(r0.x + l0.x, r0.y + l0.y);
    for (int p = 0; p < q + extra; ++p) {
      const int j = n - q + p;
      const double2 fl = ldd(ring_at(a, j, 0, c, ab)), fg = ldd(ring_at(a, j, 1, c, ab));
      gl.x = fma(w[p], fl.x, gl.x); gl.y = fma(w[p], fl.y, gl.y);
      gg.x = fma(w[p], fg.x, gg.x); gg.y = fma(w[p], fg.y, gg.y);
    }
    std2(Ln, gl);
    std2(Rn, make_double2(gg.x - gl.x, gg.y - gl.y));
  } else {
    const int q = min(a.kn, n);
    const double* w = wt + (q - 1) * kWTab;
    double2 gl = ldd(a.L + (tri(n - 1, n - 1) * MM + ab) * 2);
    const int ba = ib * M + ia;
    for (int p = 0; p < q + extra; ++p) {
      const int j = n - q + p;
      const double2 f = ldd(ring_at(a, j, 0, j, ab)), ft = ldd(ring_at(a, j, 0, j, ba));
      // D(j)_ab = F^<(j,j)_ab - conj(F^<(j,j)_ba)
      gl.x = fma(w[p], f.x - ft.x, gl.x);
      gl.y = fma(w[p], f.y + ft.y, gl.y);
    }
    std2(Ln, gl);
    std2(Rn, make_double2(0.0, ia == ib ? -1.0 : 0.0));
  }
}

// F^s(n,c)_ab = -i ( sum_x eps_ax G^s(n,c)_xb + I^s(n,c)_ab ),  G^> = R + L;
// returns false on a non-finite value.
__device__ __forceinline__ bool rhs_entry(const StepArgs& a, int64_t lin) {
  const int M = a.M, MM = M * M, n = a.n;
  const int c = div_idx(lin, MM), ab = (int)(lin - (int64_t)c * MM);
  const int ia = ab / M, ib = ab - ia * M;
  const double* Lb = a.L + tri(n, c) * MM * 2;
  const double* Rb = a.R + tri(n, c) * MM * 2;
  double2 sl = ldd(a.I + ((int64_t)c * MM + ab) * 2);
  double2 sg = ldd(a.I + (((int64_t)(n + 1) + c) * MM + ab) * 2);
  for (int x = 0; x < M; ++x) {
    const double2 e = ldd(a.eps + 2 * (ia * M + x));
    const double2 l = ldd(Lb + 2 * (x * M + ib));
    const double2 r = ldd(Rb + 2 * (x * M + ib));
    const double gr = r.x + l.x, gi = r.y + l.y;
    sl.x = fma(e.x, l.x, sl.x); sl.x = fma(-e.y, l.y, sl.x);
    sl.y = fma(e.x, l.y, sl.y); sl.y = fma(e.y, l.x, sl.y);
    sg.x = fma(e.x, gr, sg.x);  sg.x = fma(-e.y, gi, sg.x);
    sg.y = fma(e.x, gi, sg.y);  sg.y = fma(e.y, gr, sg.y);
  }
  // -i (x + i y) = y - i x
  const double2 fl = make_double2(sl.y, -sl.x), fg = make_double2(sg.y, -sg.x);
  std2(const_cast<double*>(ring_at(a, n, 0, c, ab)), fl);
  std2(const_cast<double*>(ring_at(a, n, 1, c, ab)), fg);
  return isfinite(fl.x) && isfinite(fl.y) && isfinite(fg.x) && isfinite(fg.y);
}

// The same for one component s (0: F^<, 1: F^>) of entry lin: the same
// operations in the same order as that component's in rhs_entry, so the
// value is bitwise rhs_entry's; returns false on a non-finite value.
__device__ __forceinline__ bool rhs_entry_s(const StepArgs& a, int64_t lin, int s) {
  const int M = a.M, MM = M * M, n = a.n;
  const int c = div_idx(lin, MM), ab = (int)(lin - (int64_t)c * MM);
  const int ia = ab / M, ib = ab - ia * M;
  const double* Lb = a.L + tri(n, c) * MM * 2;
  const double* Rb = a.R + tri(n, c) * MM * 2;
  double2 acc = ldd(a.I + (((int64_t)s * (n + 1) + c) * MM + ab) * 2);
  for (int x = 0; x < M; ++x) {
    const double2 e = ldd(a.eps + 2 * (ia * M + x));
    const double2 l = ldd(Lb + 2 * (x * M + ib));
    double gr = l.x, gi = l.y;
    if (s) {
      const double2 r = ldd(Rb + 2 * (x * M + ib));
      gr = r.x + l.x;
      gi = r.y + l.y;
    }
    acc.x = fma(e.x, gr, acc.x); acc.x = fma(-e.y, gi, acc.x);
    acc.y = fma(e.x, gi, acc.y); acc.y = fma(e.y, gr, acc.y);
  }
  const double2 f = make_double2(acc.y, -acc.x);
  std2(const_cast<double*>(ring_at(a, n, s, c, ab)), f);
  return isfinite(f.x) && isfinite(f.y);
}

}  // namespace rk
}  // namespace kbe
