// adjoint.cu -- reverse-mode (vector-Jacobian) kernels of the KBE step.
//
// Cotangents follow the convention of PyTorch for a real loss F of a complex
// z = x + iy: zbar = dF/dx + i dF/dy.  With it, y = A z gives zbar += A^+ ybar,
// y = conj(z) gives zbar += conj(ybar), y = Im z gives zbar += i ybar, and a
// real parameter p gets sum Re(conj(ybar) dy/dp).
//
// History slice (Eq. KBE2), I^s(c) = sum_m A1[m] G^s(m,c) + sum_{m<=c} w_{c,m} S^s[m] G^A(m,c),
// A1[m] = w_{n,m} (S^>[m] - S^<[m]):
//   A1bar[m]  = sum_{s,c} Ibar^s(c) G^s(m,c)^+
//   Bbar^s[m] = sum_{c>=m} w_{c,m} Ibar^s(c) G^A(m,c)^+ = sum_{c>=m} w_{c,m} Ibar^s(c) R(c,m)
//   S^>bar[m] = w_{n,m} A1bar[m] + Bbar^>[m],  S^<bar[m] = -w_{n,m} A1bar[m] + Bbar^<[m]
// and for a stored block (r,q), r >= q, of a row that carries a cotangent
// (J = Ibar^< + Ibar^>):
//   Lbar(r,q) += A1[r]^+ J(q) - [q<r] J(r)^+ A1[q]
//   Rbar(r,q) += A1[r]^+ Ibar^>(q) - [q<r] Ibar^>(r)^+ A1[q] + [q<r] w_{r,q} sum_s Ibar^s(r)^+ S^s[q].
// (R(r,r) = -i*1 is a constant of the method and carries no cotangent.)

#include "dfloat.cuh"
#include "kbe_internal.h"

namespace kbe {
namespace {

struct Cz {
  double re, im;
};
__device__ __forceinline__ Cz ldz(const double* p) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  return Cz{v.x, v.y};
}
__device__ __forceinline__ void stz(double* p, Cz v) { *reinterpret_cast<double2*>(p) = make_double2(v.re, v.im); }
__device__ __forceinline__ void addz(double* p, Cz v) {
  double2 o = *reinterpret_cast<double2*>(p);
  o.x += v.re;
  o.y += v.im;
  *reinterpret_cast<double2*>(p) = o;
}
__device__ __forceinline__ Cz operator+(Cz a, Cz b) { return Cz{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ Cz operator-(Cz a, Cz b) { return Cz{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ Cz operator*(Cz a, Cz b) { return Cz{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ Cz cj(Cz a) { return Cz{a.re, -a.im}; }
__device__ __forceinline__ Cz sc(double s, Cz a) { return Cz{s * a.re, s * a.im}; }
__device__ __forceinline__ Cz mi(Cz a) { return Cz{a.im, -a.re}; }  // -i a
__device__ __forceinline__ Cz pi_(Cz a) { return Cz{-a.im, a.re}; } // i a
// acc += a * b
__device__ __forceinline__ void mac(Cz& acc, Cz a, Cz b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc += a * conj(b)
__device__ __forceinline__ void mac_cj(Cz& acc, Cz a, Cz b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(-a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
__device__ __forceinline__ void mac_ca(Cz& acc, Cz a, Cz b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256); }

// Rows the slice adjoints read in their inner loops, formed once:
// Js = Ibar^< + Ibar^>, A1 = w_{n,m} (S^> - S^<)(n,m); both [n+1][M][M].
__global__ void __launch_bounds__(256) adj_prep(int M, int n, const double* __restrict__ Ib,
                                                const double* __restrict__ Sl, const double* __restrict__ Sg,
                                                WeightsView w, double* __restrict__ Js, double* __restrict__ A1) {
  const int MM = M * M;
  const int64_t srow = (int64_t)(n + 1) * MM;
  const int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lin >= srow) return;
  stz(Js + lin * 2, ldz(Ib + lin * 2) + ldz(Ib + (srow + lin) * 2));
  stz(A1 + lin * 2, sc(w.at(n, (int)(lin / MM)), ldz(Sg + lin * 2) - ldz(Sl + lin * 2)));
}

// ------------------------------------------------ history slice: Sigma ---
// Partial sums over a chunk of output columns c of A1bar[m] and Bbar^s[m]
// for every (m, a, x): part[chunk][3][n+1][M][M].
__global__ void __launch_bounds__(256) adj_hist_small(int M, int n, int chunk_len, const double* __restrict__ L,
                                                      const double* __restrict__ R, const double* __restrict__ Ib,
                                                      const double* __restrict__ Js, WeightsView w,
                                                      double* __restrict__ part) {
  const int MM = M * M;
  const int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lin >= (int64_t)(n + 1) * MM) return;
  const int m = (int)(lin / MM), ax = (int)(lin - (int64_t)m * MM);
  const int a = ax / M, x = ax - a * M;
  const int c0 = blockIdx.y * chunk_len, c1 = min(n + 1, c0 + chunk_len);
  const int64_t srow = (int64_t)(n + 1) * MM;  // stride of s in Ibar
  Cz A{0, 0}, Bl{0, 0}, Bg{0, 0};
  for (int c = c0; c < c1; ++c) {
    const double* il = Ib + ((int64_t)c * MM + a * M) * 2;
    const double* ig = Ib + (srow + (int64_t)c * MM + a * M) * 2;
    const double* is = Js + ((int64_t)c * MM + a * M) * 2;  // Ibar^< + Ibar^>
    // jl conj(G^<) + jg conj(G^>) = (jl + jg) conj(L) + jg conj(R), as G^> = R + L
    if (c <= m) {  // G^<(m,c) = L(m,c), G^> = (R+L)(m,c): conj(G(m,c)[x][b])
      const double* lb = L + (tri(m, c) * MM + x * M) * 2;
      const double* rb = R + (tri(m, c) * MM + x * M) * 2;
      for (int b = 0; b < M; ++b) {
        mac_cj(A, ldz(is + 2 * b), ldz(lb + 2 * b));
        mac_cj(A, ldz(ig + 2 * b), ldz(rb + 2 * b));
      }
    } else {       // G(m,c)[x][b] = -conj(X(c,m)[b][x]): conj -> -X(c,m)[b][x]
      const int64_t blk = tri(c, m) * MM;
      for (int b = 0; b < M; ++b) {
        const Cz l = ldz(L + (blk + b * M + x) * 2), r = ldz(R + (blk + b * M + x) * 2);
        mac(A, ldz(is + 2 * b), Cz{-l.re, -l.im});
        mac(A, ldz(ig + 2 * b), Cz{-r.re, -r.im});
      }
    }
    if (c >= m) {  // term 2: w_{c,m} Ibar^s(c)[a][b] R(c,m)[b][x]
      const double wcm = w.at(c, m);
      const int64_t blk = tri(c, m) * MM;
      Cz tl{0, 0}, tg{0, 0};
      for (int b = 0; b < M; ++b) {
        const Cz r = ldz(R + (blk + b * M + x) * 2);
        mac(tl, ldz(il + 2 * b), r);
        mac(tg, ldz(ig + 2 * b), r);
      }
      Bl = Bl + sc(wcm, tl);
      Bg = Bg + sc(wcm, tg);
    }
  }
  double* out = part + ((int64_t)blockIdx.y * 3 * srow + lin) * 2;
  stz(out, A);
  stz(out + srow * 2, Bl);
  stz(out + 2 * srow * 2, Bg);
}

// The same partial sums in double-float on the FP32 pipe (the reverse sweep
// of KBE_DF64 steps): the cotangent rows Ibar^<, Ibar^> and Js come as
// double-float rows (Ibf [2][n+1][MM], Jsf [n+1][MM]), the history entries
// are converted where they are read, every sum is a compensated pair.
__global__ void __launch_bounds__(256) adj_prep_df(int64_t n2, const double* __restrict__ Ib,
                                                   const double* __restrict__ Js, float4* __restrict__ Ibf,
                                                   float4* __restrict__ Jsf, int64_t srow) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n2) return;
  Ibf[e] = df::c2f(reinterpret_cast<const double2*>(Ib)[e]);
  if (e < srow) Jsf[e] = df::c2f(reinterpret_cast<const double2*>(Js)[e]);
}

__global__ void __launch_bounds__(256) adj_hist_small_df(int M, int n, int chunk_len, const double* __restrict__ L,
                                                         const double* __restrict__ R,
                                                         const float4* __restrict__ Ibf,
                                                         const float4* __restrict__ Jsf, WeightsView w,
                                                         double* __restrict__ part) {
  const int MM = M * M;
  const int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lin >= (int64_t)(n + 1) * MM) return;
  const int m = (int)(lin / MM), ax = (int)(lin - (int64_t)m * MM);
  const int a = ax / M, x = ax - a * M;
  const int c0 = blockIdx.y * chunk_len, c1 = min(n + 1, c0 + chunk_len);
  const int64_t srow = (int64_t)(n + 1) * MM;
  const double2* L2 = reinterpret_cast<const double2*>(L);
  const double2* R2 = reinterpret_cast<const double2*>(R);
  df::Acc Ar{0.f, 0.f}, Ai{0.f, 0.f}, Blr{0.f, 0.f}, Bli{0.f, 0.f}, Bgr{0.f, 0.f}, Bgi{0.f, 0.f};
  for (int c = c0; c < c1; ++c) {
    const float4* il = Ibf + (int64_t)c * MM + a * M;
    const float4* ig = Ibf + srow + (int64_t)c * MM + a * M;
    const float4* is = Jsf + (int64_t)c * MM + a * M;
    if (c <= m) {  // conj(G(m,c)[x][b]): conj(L), conj(R) of block (m,c) row x
      const int64_t blk = tri(m, c) * MM + x * M;
      for (int b = 0; b < M; ++b) {
        df::cmac(Ar, Ai, is[b], df::cconj(df::c2f(L2[blk + b])));
        df::cmac(Ar, Ai, ig[b], df::cconj(df::c2f(R2[blk + b])));
      }
    } else {       // -X(c,m)[b][x]
      const int64_t blk = tri(c, m) * MM;
      for (int b = 0; b < M; ++b) {
        df::cmac(Ar, Ai, is[b], df::cneg(df::c2f(L2[blk + b * M + x])));
        df::cmac(Ar, Ai, ig[b], df::cneg(df::c2f(R2[blk + b * M + x])));
      }
    }
    if (c >= m) {  // term 2: w_{c,m} sum_b Ibar^s(c)[a][b] R(c,m)[b][x]
      const df::F2 wf = df::from_double_fast(w.at(c, m));
      const int64_t blk = tri(c, m) * MM;
      df::Acc tlr{0.f, 0.f}, tli{0.f, 0.f}, tgr{0.f, 0.f}, tgi{0.f, 0.f};
      for (int b = 0; b < M; ++b) {
        const float4 r = df::c2f(R2[blk + b * M + x]);
        df::cmac(tlr, tli, il[b], r);
        df::cmac(tgr, tgi, ig[b], r);
      }
      df::acc_prod(Blr, wf.hi, wf.lo, tlr.s, tlr.c);
      df::acc_prod(Bli, wf.hi, wf.lo, tli.s, tli.c);
      df::acc_prod(Bgr, wf.hi, wf.lo, tgr.s, tgr.c);
      df::acc_prod(Bgi, wf.hi, wf.lo, tgi.s, tgi.c);
    }
  }
  double* out = part + ((int64_t)blockIdx.y * 3 * srow + lin) * 2;
  stz(out, Cz{df::acc_value(Ar), df::acc_value(Ai)});
  stz(out + srow * 2, Cz{df::acc_value(Blr), df::acc_value(Bli)});
  stz(out + 2 * srow * 2, Cz{df::acc_value(Bgr), df::acc_value(Bgi)});
}

// Sl_bar, Sg_bar from the ordered sum of the chunk partials.
__global__ void __launch_bounds__(256) adj_hist_small_reduce(int M, int n, int nchunk, const double* __restrict__ part,
                                                             WeightsView w, double* __restrict__ dSl,
                                                             double* __restrict__ dSg) {
  const int MM = M * M;
  const int64_t srow = (int64_t)(n + 1) * MM;
  const int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lin >= srow) return;
  const int m = (int)(lin / MM);
  Cz A{0, 0}, Bl{0, 0}, Bg{0, 0};
  for (int k = 0; k < nchunk; ++k) {
    const double* p = part + ((int64_t)k * 3 * srow + lin) * 2;
    A = A + ldz(p);
    Bl = Bl + ldz(p + srow * 2);
    Bg = Bg + ldz(p + 2 * srow * 2);
  }
  const double wn = w.at(n, m);
  stz(dSg + lin * 2, sc(wn, A) + Bg);
  stz(dSl + lin * 2, Bl - sc(wn, A));
}

// ---------------------------------------------- history slice: G rows ---
// Cotangents of the stored blocks (r,q) of rows r in [row_lo, n]: rows r < n
// accumulate into dL, dR (triangles); row n goes to gL, gR (row buffers of
// the current iterate, [n+1][M][M]).
__global__ void __launch_bounds__(256) adj_hist_rows(int M, int n, int row_lo, const double* __restrict__ Js,
                                                     const double* __restrict__ A1, const double* __restrict__ Sl,
                                                     const double* __restrict__ Sg, const double* __restrict__ Ib,
                                                     WeightsView w, double* __restrict__ dL, double* __restrict__ dR,
                                                     double* __restrict__ gL, double* __restrict__ gR) {
  // dL, dR hold rows row_lo.. : block p at p - tri(row_lo, 0)
  const int MM = M * M;
  const int64_t srow = (int64_t)(n + 1) * MM;
  const int64_t base = tri(row_lo, 0);
  const int64_t total = (tri(n + 1, 0) - base) * MM;
  const int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lin >= total) return;
  const int64_t p = base + lin / MM;
  const int xy = (int)(lin % MM);
  const int x = xy / M, y = xy - x * M;
  // row r of block p
  int r = (int)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
  while ((int64_t)r * (r + 1) / 2 > p) --r;
  while ((int64_t)(r + 1) * (r + 2) / 2 <= p) ++r;
  const int q = (int)(p - (int64_t)r * (r + 1) / 2);
  // A1[m][a][x] = w_{n,m} (Sg - Sl)[m][a][x] and Js = Ibar^< + Ibar^> are precomputed rows
  Cz dl{0, 0}, dr{0, 0}, t2{0, 0};
  for (int a = 0; a < M; ++a) {
    const Cz a1r = ldz(A1 + ((int64_t)r * MM + a * M + x) * 2);
    mac_ca(dl, a1r, ldz(Js + ((int64_t)q * MM + a * M + y) * 2));
    mac_ca(dr, a1r, ldz(Ib + (srow + (int64_t)q * MM + a * M + y) * 2));
    if (q < r) {
      const Cz na1q = sc(-1.0, ldz(A1 + ((int64_t)q * MM + a * M + y) * 2));
      const Cz jgr = ldz(Ib + (srow + (int64_t)r * MM + a * M + x) * 2);
      mac_ca(dl, ldz(Js + ((int64_t)r * MM + a * M + x) * 2), na1q);
      mac_ca(dr, jgr, na1q);
      mac_ca(t2, ldz(Ib + ((int64_t)r * MM + a * M + x) * 2), ldz(Sl + ((int64_t)q * MM + a * M + y) * 2));
      mac_ca(t2, jgr, ldz(Sg + ((int64_t)q * MM + a * M + y) * 2));
    }
  }
  if (q < r) dr = dr + sc(w.at(r, q), t2);
  if (r < n) {
    addz(dL + ((p - base) * MM + xy) * 2, dl);
    if (q < r) addz(dR + ((p - base) * MM + xy) * 2, dr);
  } else {
    addz(gL + ((int64_t)q * MM + xy) * 2, dl);
    if (q < r) addz(gR + ((int64_t)q * MM + xy) * 2, dr);
  }
}

// ---------------------------------------------------------- self-energy --
// Off-diagonal blocks c < n: elementwise.  gL, gR += cotangents of row n;
// dUp[c*MM + ab] receives the U contributions of entry (a,b) split as
// (to U_a, to U_b) so that a later ordered reduction stays deterministic.
__global__ void __launch_bounds__(256) adj_sigma_off(int M, int n, const double* __restrict__ Lrow,
                                                     const double* __restrict__ Rrow, const double* __restrict__ U,
                                                     const double* __restrict__ dSl, const double* __restrict__ dSg,
                                                     double* __restrict__ gL, double* __restrict__ gR,
                                                     double* __restrict__ dUp) {
  const int MM = M * M;
  const int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lin >= (int64_t)n * MM) return;
  const int ab = (int)(lin % MM), a = ab / M, b = ab - a * M;
  const Cz l = ldz(Lrow + lin * 2), r = ldz(Rrow + lin * 2);
  const Cz g = l + r;
  const Cz tl{-l.re, l.im}, tg{-g.re, g.im};  // -conj(l), -conj(g)
  const double uu = U[a] * U[b];
  const Cz sbg = ldz(dSg + lin * 2), sbl = ldz(dSl + lin * 2);
  // S^> = uu g^2 tl ; S^< = uu l^2 tg
  const Cz g2 = g * g, l2 = l * l;
  Cz gb{0, 0}, lb{0, 0};
  mac_ca(gb, sc(2.0 * uu, g * tl), sbg);      // conj(2 uu g tl) Sbar^>
  const Cz tlb = cj(sc(uu, g2)) * sbg;        // tl-bar
  lb = lb - cj(tlb);                          // tl = -conj(l)
  mac_ca(lb, sc(2.0 * uu, l * tg), sbl);
  const Cz tgb = cj(sc(uu, l2)) * sbl;
  gb = gb - cj(tgb);
  lb = lb + gb;
  addz(gL + lin * 2, lb);
  addz(gR + lin * 2, gb);
  // d/dU_a of uu = U_b, d/dU_b = U_a
  const Cz dsg = g2 * tl, dsl = l2 * tg;
  const double re = sbg.re * dsg.re + sbg.im * dsg.im + sbl.re * dsl.re + sbl.im * dsl.im;  // Re(conj(Sbar) dS/duu)
  dUp[lin * 2] = re * U[b];
  dUp[lin * 2 + 1] = re * U[a];
}

// Diagonal block c = n: the third factor is the transposed entry of the
// same block, so entry (a,b) also receives the cross terms of entry (b,a).
__global__ void adj_sigma_diag(int M, const double* __restrict__ Lnn, const double* __restrict__ Rnn,
                               const double* __restrict__ U, const double* __restrict__ dSl,
                               const double* __restrict__ dSg, double* __restrict__ gLnn, double* __restrict__ dUp) {
  const int MM = M * M;
  for (int ab = threadIdx.x; ab < MM; ab += blockDim.x) {
    const int a = ab / M, b = ab - a * M, ba = b * M + a;
    const Cz l = ldz(Lnn + ab * 2), g = l + ldz(Rnn + ab * 2);
    const Cz lt = ldz(Lnn + ba * 2), gt = lt + ldz(Rnn + ba * 2);
    const double uu = U[a] * U[b];
    const Cz sbg = ldz(dSg + ab * 2), sbl = ldz(dSl + ab * 2);
    const Cz sbg_t = ldz(dSg + ba * 2), sbl_t = ldz(dSl + ba * 2);
    // S^>_ab = uu g_ab^2 L_ba,  S^<_ab = uu l_ab^2 G^>_ba;  R(n,n) is fixed, so
    // G^> cotangents go to L.
    Cz lb{0, 0};
    mac_ca(lb, sc(2.0 * uu, g * lt), sbg);
    mac_ca(lb, sc(2.0 * uu, l * gt), sbl);
    // entry (b,a): S^>_ba = uu g_ba^2 L_ab,  S^<_ba = uu l_ba^2 G^>_ab
    mac_ca(lb, sc(uu, gt * gt), sbg_t);
    mac_ca(lb, sc(uu, lt * lt), sbl_t);
    addz(gLnn + ab * 2, lb);
    const Cz dsg = (g * g) * lt, dsl = (l * l) * gt;
    const double re = sbg.re * dsg.re + sbg.im * dsg.im + sbl.re * dsl.re + sbl.im * dsl.im;
    dUp[ab * 2] = re * U[b];
    dUp[ab * 2 + 1] = re * U[a];
  }
}

// dU[a] += sum over (c, b) of the split contributions (ordered, one block per a).
__global__ void adj_reduce_dU(int M, int n, const double* __restrict__ dUp, double* __restrict__ dU) {
  const int a = blockIdx.x;
  const int MM = M * M;
  __shared__ double red[256];
  double acc = 0.0;
  // entries (c, a, b) give dUp[...][0] to U_a; entries (c, b', a) give dUp[...][1] to U_a
  for (int64_t k = threadIdx.x; k < (int64_t)(n + 1) * M; k += blockDim.x) {
    const int c = (int)(k / M), b = (int)(k % M);
    acc += dUp[((int64_t)c * MM + a * M + b) * 2] + dUp[((int64_t)c * MM + b * M + a) * 2 + 1];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) dU[a] += red[0];
}

// ------------------------------------------------------ right-hand side --
// F^s(n,c) = -i (eps G^s(n,c) + I^s(n,c)).  With Y = i Fbar:
// Ibar = Y, Gbar^s(c) += eps^+ Y^s(c) (eps Hermitian), epsbar = sum Y G^+.
__global__ void __launch_bounds__(256) adj_rhs(int M, int n, const double* __restrict__ eps,
                                               const double* __restrict__ Fb, int64_t fs, double* __restrict__ Ib,
                                               double* __restrict__ gL, double* __restrict__ gR) {
  const int MM = M * M;
  const int64_t srow = (int64_t)(n + 1) * MM;
  const int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lin >= srow) return;
  const int c = (int)(lin / MM), xb = (int)(lin % MM);
  const int x = xb / M, b = xb - x * M;
  const double* Fg = Fb + fs;
  stz(Ib + lin * 2, pi_(ldz(Fb + lin * 2)));
  stz(Ib + (srow + lin) * 2, pi_(ldz(Fg + lin * 2)));
  Cz gl{0, 0}, gg{0, 0};
  for (int a = 0; a < M; ++a) {
    const Cz e = ldz(eps + (a * M + x) * 2);
    mac_ca(gl, e, pi_(ldz(Fb + ((int64_t)c * MM + a * M + b) * 2)));
    mac_ca(gg, e, pi_(ldz(Fg + ((int64_t)c * MM + a * M + b) * 2)));
  }
  addz(gL + lin * 2, gl + gg);
  if (c < n) addz(gR + lin * 2, gg);
}

// epsbar[a][x] = sum_{s,c,b} Y^s(c)[a][b] conj(G^s(c)[x][b]); one block per (a,x);
// then the Hartree and field parts of eps (see kbe_internal.h, StepArgs).
__global__ void adj_eps(int M, int n, const double* __restrict__ Fb, int64_t fs, const double* __restrict__ Lrow,
                        const double* __restrict__ Rrow, double* __restrict__ epsb) {
  const int MM = M * M;
  const int ax = blockIdx.x, a = ax / M, x = ax - a * M;
  const double* Fg = Fb + fs;
  __shared__ double rr[256], ri[256];
  Cz acc{0, 0};
  for (int64_t k = threadIdx.x; k < (int64_t)(n + 1) * M; k += blockDim.x) {
    const int c = (int)(k / M), b = (int)(k % M);
    const Cz yl = pi_(ldz(Fb + ((int64_t)c * MM + a * M + b) * 2));
    const Cz yg = pi_(ldz(Fg + ((int64_t)c * MM + a * M + b) * 2));
    const Cz l = ldz(Lrow + ((int64_t)c * MM + x * M + b) * 2);
    const Cz r = ldz(Rrow + ((int64_t)c * MM + x * M + b) * 2);
    mac_cj(acc, yl, l);
    mac_cj(acc, yg, l + r);
  }
  rr[threadIdx.x] = acc.re;
  ri[threadIdx.x] = acc.im;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) { rr[threadIdx.x] += rr[threadIdx.x + s]; ri[threadIdx.x] += ri[threadIdx.x + s]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { epsb[ax * 2] = rr[0]; epsb[ax * 2 + 1] = ri[0]; }
}

// eps = h0 + E(t) diag(v) + diag(U_a Im L(n,n)_aa):
//   dU[a] += Re(epsbar_aa) Im L_aa;  gL(n,n)_aa += i Re(epsbar_aa) U_a;
//   dE0 += g(t_n) sum_a Re(epsbar_aa) v_a   (E(t) = E0 g(t)).
__global__ void adj_eps_params(int M, int n, const double* __restrict__ epsb, const double* __restrict__ Lnn,
                               const double* __restrict__ U, const double* __restrict__ v, double shape,
                               double* __restrict__ gLnn, double* __restrict__ dU, double* __restrict__ dE0) {
  if (threadIdx.x != 0) return;
  double de = 0.0;
  for (int a = 0; a < M; ++a) {
    const double e = epsb[(a * M + a) * 2];
    dU[a] += e * Lnn[(a * M + a) * 2 + 1];
    gLnn[(a * M + a) * 2 + 1] += e * U[a];
    de += e * v[a];
  }
  dE0[0] += de * shape;
}

// ------------------------------------------------- predictor / corrector --
// G^s(n,c) = G^s(n-1,c) + sum_p w_p F^s(j_p, c) with L = G^<, R = G^> - G^<
// (c < n), and L(n,n) = L(n-1,n-1) + sum_p w_p (F^<(j,j) - F^<(j,j)^+).
// Given the cotangent (gL, gR) of row n: dL/dR of row n-1 and the F-row
// cotangents.  F rows j < n live at Fb_rows + (j - j0) * fstride; the node
// j = n (corrector only) goes to Fb_cur.  Off-diagonal columns here, the
// diagonal in adj_step_lin_diag (separate launch: both touch F^<(j,j)).
__global__ void __launch_bounds__(256) adj_step_lin_off(AdjLinArgs a) {
  const int M = a.M, MM = M * M, n = a.n;
  const int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lin >= (int64_t)n * MM) return;
  const int c = (int)(lin / MM), ab = (int)(lin % MM);
  const Cz gl = ldz(a.gL + lin * 2), gr = ldz(a.gR + lin * 2);
  const Cz Gl = gl - gr, Gg = gr;  // cotangents of G^< and G^> of row n
  if (a.write_prev) {  // L(n-1,c) enters G^< and G^>, R(n-1,c) enters G^>
    const int64_t p = tri(n - 1, c) - a.tri_base;
    addz(a.dL + (p * MM + ab) * 2, Gl + Gg);
    addz(a.dR + (p * MM + ab) * 2, Gg);
  }
  // predictor: nodes n-q..n-1; corrector: nodes n-kap..n (q, kap = min(k_n, n-c))
  const int cnt = min(a.kn, n - c);
  const double* w = a.wtab + (cnt - 1) * kWTab;
  const int np = a.corrector ? cnt + 1 : cnt;
  const int64_t off = ((int64_t)c * MM + ab) * 2;
  for (int p = 0; p < np; ++p) {
    const int j = n - cnt + p;
    double* fr = j == n ? a.Fb_cur : a.Fb_rows + (int64_t)(j - a.j0) * a.fstride;
    addz(fr + off, sc(w[p], Gl));
    addz(fr + a.fs + off, sc(w[p], Gg));
  }
}

// Diagonal block: L(n,n) = L(n-1,n-1) + sum_p w_p D(j_p), D = F^<(j,j) - F^<(j,j)^+,
// so Fbar^<(j,j) += w_p (Dbar - Dbar^+) with Dbar = Lbar(n,n); R(n,n) is fixed.
__global__ void adj_step_lin_diag(AdjLinArgs a) {
  const int M = a.M, MM = M * M, n = a.n;
  const int cnt = min(a.kn, n);
  const double* w = a.wtab + (cnt - 1) * kWTab;
  const int np = a.corrector ? cnt + 1 : cnt;
  for (int ab = threadIdx.x; ab < MM; ab += blockDim.x) {
    const int x = ab / M, y = ab - x * M;
    const Cz gl = ldz(a.gL + ((int64_t)n * MM + ab) * 2);
    const Cz glt = ldz(a.gL + ((int64_t)n * MM + y * M + x) * 2);
    if (a.write_prev) addz(a.dL + ((tri(n - 1, n - 1) - a.tri_base) * MM + ab) * 2, gl);
    const Cz dd = gl - cj(glt);
    for (int p = 0; p < np; ++p) {
      const int j = n - cnt + p;
      double* fr = j == n ? a.Fb_cur : a.Fb_rows + (int64_t)(j - a.j0) * a.fstride;
      addz(fr + ((int64_t)j * MM + ab) * 2, sc(w[p], dd));
    }
  }
}

}  // namespace

// ------------------------------------------------------------- launchers --
cudaError_t launch_adjoint_history(const AdjHistArgs& h, cudaStream_t s, int* launches) {
  *launches = 0;
  const int M = h.M, MM = M * M, n = h.n;
  const int64_t srow = (int64_t)(n + 1) * MM;
  int64_t want = ((int64_t)sm_count() * 2048 + srow - 1) / srow;
  int nchunk = (int)(want < 1 ? 1 : (want > kMaxSplit ? kMaxSplit : want));
  if (nchunk > n + 1) nchunk = n + 1;
  // the workspace holds the chunk partials [nchunk][3][srow], then the rows Js
  // and A1 (and, for the double-float sums, Ibar^<, Ibar^> and Js as
  // double-float rows)
  const int extra = h.df ? 5 : 2;
  while (nchunk > 1 && (size_t)(nchunk * 3 + extra) * srow * 16 > h.work_bytes) --nchunk;
  if ((size_t)(nchunk * 3 + extra) * srow * 16 > h.work_bytes) return cudaErrorInvalidValue;
  const int chunk_len = (n + 1 + nchunk - 1) / nchunk;
  nchunk = (n + 1 + chunk_len - 1) / chunk_len;
  double* Js = h.work + (size_t)nchunk * 3 * srow * 2;
  double* A1 = Js + srow * 2;
  adj_prep<<<blocks_for(srow), 256, 0, s>>>(M, n, h.Ib, h.Sl, h.Sg, h.w, Js, A1);
  int nl = 3;
  if (h.df) {
    float4* Ibf = reinterpret_cast<float4*>(A1 + srow * 2);
    float4* Jsf = Ibf + 2 * srow;
    adj_prep_df<<<blocks_for(2 * srow), 256, 0, s>>>(2 * srow, h.Ib, Js, Ibf, Jsf, srow);
    adj_hist_small_df<<<dim3(blocks_for(srow), nchunk), 256, 0, s>>>(M, n, chunk_len, h.L, h.R, Ibf, Jsf, h.w,
                                                                     h.work);
    ++nl;
  } else {
    adj_hist_small<<<dim3(blocks_for(srow), nchunk), 256, 0, s>>>(M, n, chunk_len, h.L, h.R, h.Ib, Js, h.w,
                                                                  h.work);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  adj_hist_small_reduce<<<blocks_for(srow), 256, 0, s>>>(M, n, nchunk, h.work, h.w, h.dSl, h.dSg);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t rows_total = (tri(n + 1, 0) - tri(h.row_lo, 0)) * MM;
  adj_hist_rows<<<blocks_for(rows_total), 256, 0, s>>>(M, n, h.row_lo, Js, A1, h.Sl, h.Sg, h.Ib, h.w, h.dL, h.dR,
                                                       h.gL, h.gR);
  *launches = nl + 1;
  return cudaGetLastError();
}

cudaError_t launch_adjoint_sigma(const AdjSigmaArgs& a, cudaStream_t s, int* launches) {
  const int M = a.M, MM = M * M, n = a.n;
  *launches = 0;
  if (n > 0) {
    adj_sigma_off<<<blocks_for((int64_t)n * MM), 256, 0, s>>>(M, n, a.Lrow, a.Rrow, a.U, a.dSl, a.dSg, a.gL, a.gR,
                                                              a.dUp);
    ++*launches;
  }
  const int64_t dn = (int64_t)n * MM * 2;
  adj_sigma_diag<<<1, 256, 0, s>>>(M, a.Lrow + dn, a.Rrow + dn, a.U, a.dSl + dn, a.dSg + dn, a.gL + dn,
                                   a.dUp + dn);
  adj_reduce_dU<<<M, 256, 0, s>>>(M, n, a.dUp, a.dU);
  *launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_adjoint_rhs(const AdjRhsArgs& a, cudaStream_t s, int* launches) {
  const int M = a.M, MM = M * M, n = a.n;
  const int64_t srow = (int64_t)(n + 1) * MM;
  adj_rhs<<<blocks_for(srow), 256, 0, s>>>(M, n, a.eps, a.Fb, a.fs, a.Ib, a.gL, a.gR);
  adj_eps<<<MM, 256, 0, s>>>(M, n, a.Fb, a.fs, a.Lrow, a.Rrow, a.epsb);
  const int64_t dn = (int64_t)n * MM * 2;
  adj_eps_params<<<1, 32, 0, s>>>(M, n, a.epsb, a.Lrow + dn, a.U, a.v, a.shape, a.gL + dn, a.dU, a.dE0);
  *launches = 3;
  return cudaGetLastError();
}

cudaError_t launch_adjoint_lin(const AdjLinArgs& a, cudaStream_t s, int* launches) {
  *launches = 0;
  if (a.n > 0) {
    adj_step_lin_off<<<blocks_for((int64_t)a.n * a.M * a.M), 256, 0, s>>>(a);
    ++*launches;
  }
  adj_step_lin_diag<<<1, 256, 0, s>>>(a);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace kbe
