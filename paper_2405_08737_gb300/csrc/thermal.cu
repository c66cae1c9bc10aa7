// thermal.cu -- the thermal branch of the KBE step (Sec. 2, Eq. KBE3 and the
// tau terms of Eq. KBE2), FP64, local interaction.
//
// State: the mixed rows G^|(t_r, tau_k), [n_max][N][M][M], on a uniform tau
// grid tau_k = k beta / (N-1).  Conventions (fermions):
//   G^|-(tau, t) = [G^|(t, beta - tau)]^+,  G^M(s - tau) = -G^M(beta + s - tau) for s < tau,
//   Sigma^|_ab(t,tau) = U_a U_b G^|_ab(t,tau)^2 G^|-_ba(tau,t)           (Eq. SE, local U).
// Kernels for row n:
//   th_sigma   Sigma^|(t_n, tau_k), elementwise, with the weighted copies the
//              contractions read (w_k Sigma^|, w_{n,m} Sigma^R): four FMAs per
//              complex product there instead of six to eight;
//   th_mixed   adds -i sum_k w_k Sigma^|(n,k) G^|-(tau_k, t_c) to both history
//              integrals I^<>(n,c), c = 0..n;
//   th_rhs     F^|(n,j) = -i [eps G^|(n,j) + sum_m w_{n,m} Sigma^R(n,m) G^|(m,j)
//              + int_0^beta Sigma^|(n,s) G^M(s - tau_j) ds], the Matsubara
//              convolution split at s = tau_j;
//   th_adams   predictor or corrector of the mixed row with the weights of
//              the diagonal (q = min(k_n, n) points).
// With a.df set (the split and double-float precisions of the step) the two
// long sums, the mixed term of th_mixed and the history term of th_rhs, run
// in double-float on the FP32 pipe (dfloat.cuh: operands as hi + lo floats,
// compensated sums, about 2^-47 of the terms' sizes); the Matsubara
// convolution and everything else stay FP64.
// tau weights: left[j][k], k <= j, integrate over [0, tau_j]; [tau_j, beta]
// uses the mirrored row left[N-1-j][N-1-k]; the full interval is row N-1.

#include "dfloat.cuh"
#include "kbe_internal.h"

namespace kbe {
namespace {

constexpr int kThThreads = 256;

__device__ __forceinline__ double2 ld2(const double* p) { return *reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ void st2(double* p, double2 v) { *reinterpret_cast<double2*>(p) = v; }

__device__ __forceinline__ void cfma(double2& acc, double w, double2 x, double2 y) {  // acc += w x y
  const double xr = w * x.x, xi = w * x.y;
  acc.x = fma(xr, y.x, acc.x);
  acc.x = fma(-xi, y.y, acc.x);
  acc.y = fma(xr, y.y, acc.y);
  acc.y = fma(xi, y.x, acc.y);
}

__device__ __forceinline__ void cfma4(double2& acc, double2 x, double2 y) {  // acc += x y
  acc.x = fma(x.x, y.x, acc.x);
  acc.x = fma(-x.y, y.y, acc.x);
  acc.y = fma(x.x, y.y, acc.y);
  acc.y = fma(x.y, y.x, acc.y);
}

// Sigma^| row n and its copy scaled by the full-interval tau weights; the
// threads past N M^2 form the weighted Sigma^R row w_{n,m} (S^> - S^<)(n,m)
// of the KBE3 history term.
__global__ void __launch_bounds__(kThThreads) th_sigma(ThermalArgs a) {
  const int M = a.M, MM = M * M, N = a.N;
  const int64_t e = (int64_t)blockIdx.x * kThThreads + threadIdx.x;
  if (e >= (int64_t)N * MM) {
    const int64_t r = e - (int64_t)N * MM;
    if (r >= (int64_t)(a.n + 1) * MM) return;
    const int m = (int)(r / MM);
    const double w = a.w.at(a.n, m);
    const double2 g = ld2(a.Sg + r * 2), l = ld2(a.Sl + r * 2);
    const double2 v = make_double2(w * (g.x - l.x), w * (g.y - l.y));
    st2(a.Aw + r * 2, v);
    a.Awf[r] = df::c2f(v);
    return;
  }
  const int k = (int)(e / MM), ab = (int)(e - (int64_t)k * MM), ia = ab / M, ib = ab - ia * M;
  const double* row = a.Gx + (int64_t)a.n * N * MM * 2;
  const double2 g = ld2(row + ((int64_t)k * MM + ab) * 2);
  const double2 h = ld2(row + ((int64_t)(N - 1 - k) * MM + ab) * 2);  // G^|-_ba(tau_k, t_n) = conj(h)
  const double uu = a.U[ia] * a.U[ib];
  const double g2r = g.x * g.x - g.y * g.y, g2i = 2.0 * g.x * g.y;
  const double2 s = make_double2(uu * (g2r * h.x + g2i * h.y), uu * (g2i * h.x - g2r * h.y));
  st2(a.Smix + e * 2, s);
  const double wk = a.left[(int64_t)(N - 1) * N + k];
  const double2 sw = make_double2(wk * s.x, wk * s.y);
  st2(a.Smw + e * 2, sw);
  a.Smwf[e] = df::c2f(sw);
  if (!(isfinite(s.x) && isfinite(s.y))) atomicOr(a.status, kStatusNumeric);
}

// th_mixed and th_rhs: a block serves 32 consecutive output entries (one per
// lane, so that the lanes of a warp read neighbouring entries) and its warps
// split the long sum (warp w takes every kParts-th point); the warps' sums
// are added in a fixed order through shared memory.
constexpr int kParts = 8;
constexpr int kPartThreads = 32 * kParts;
// th_rhs in double-float: 16 parts (more warps per SM for its 256 blocks)
constexpr int kPartsDf = 16;

template <int NP>
__device__ __forceinline__ bool reduce_parts(double2& acc) {
  __shared__ double2 red[NP][32];
  red[threadIdx.x >> 5][threadIdx.x & 31] = acc;
  __syncthreads();
  if (threadIdx.x >= 32) return false;
  acc = red[0][threadIdx.x];
  for (int w = 1; w < NP; ++w) {
    acc.x += red[w][threadIdx.x].x;
    acc.y += red[w][threadIdx.x].y;
  }
  return true;
}

// Double-float sums with kChains independent accumulator pairs (term x goes
// to chain x mod kChains, unrolled so the chains stay in registers), so that consecutive products do not wait on one
// another's TwoSum; the chains are added in FP64 in a fixed order.
constexpr int kChains = 4;
struct DfSum {
  df::Acc re[kChains], im[kChains];
  __device__ __forceinline__ DfSum() {
#pragma unroll
    for (int i = 0; i < kChains; ++i) re[i] = im[i] = df::Acc{0.f, 0.f};
  }
  __device__ __forceinline__ double2 value() const {
    double2 v = make_double2(0.0, 0.0);
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      v.x += df::acc_value(re[i]);
      v.y += df::acc_value(im[i]);
    }
    return v;
  }
};

template <bool DF>
__global__ void __launch_bounds__(kPartThreads) th_mixed(ThermalArgs a) {
  constexpr int kParts = 8;
  const int M = a.M, MM = M * M, N = a.N, n = a.n;
  const int part = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
  const bool live = e < (int64_t)(n + 1) * MM;
  const int64_t ee = live ? e : 0;
  const int c = (int)(ee / MM), ab = (int)(ee - (int64_t)c * MM), ia = ab / M, ib = ab - ia * M;
  const double* gc = a.Gx + (int64_t)c * N * MM * 2;
  double2 acc = make_double2(0.0, 0.0);
  if (DF) {
    DfSum sum;
    for (int k = live ? part : N; k < N; k += kParts) {
      const float4* sk = a.Smwf + (int64_t)k * MM + ia * M;
      const double* gk = gc + ((int64_t)(N - 1 - k) * MM + ib * M) * 2;
      for (int x0 = 0; x0 < M; x0 += kChains)
#pragma unroll
        for (int i = 0; i < kChains; ++i)
          if (x0 + i < M) df::cmac(sum.re[i], sum.im[i], sk[x0 + i], df::cconj(df::c2f(ld2(gk + 2 * (x0 + i)))));
    }
    acc = sum.value();
  } else {
    for (int k = live ? part : N; k < N; k += kParts) {
      const double* sk = a.Smw + ((int64_t)k * MM + ia * M) * 2;         // w_k Sigma^|(n,k)
      const double* gk = gc + ((int64_t)(N - 1 - k) * MM + ib * M) * 2;  // G^|-(tau_k,t_c)_xb = conj(G^|(t_c,beta-tau_k)_bx)
      for (int x = 0; x < M; ++x) {
        const double2 g = ld2(gk + 2 * x);
        cfma4(acc, ld2(sk + 2 * x), make_double2(g.x, -g.y));
      }
    }
  }
  if (!reduce_parts<kParts>(acc) || !live) return;
  // -i (x + i y) = y - i x, added to I^< and I^>
  for (int s = 0; s < 2; ++s) {
    double* o = a.I + (((int64_t)s * (n + 1) + c) * MM + ab) * 2;
    const double2 v = ld2(o);
    st2(o, make_double2(v.x + acc.y, v.y - acc.x));
  }
}

template <bool DF>
__global__ void __launch_bounds__(32 * (DF ? kPartsDf : kParts)) th_rhs(ThermalArgs a) {
  constexpr int kParts = DF ? kPartsDf : ::kbe::kParts;
  const int M = a.M, MM = M * M, N = a.N, n = a.n;
  const int part = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * 32 + (threadIdx.x & 31);
  const bool live = e < (int64_t)N * MM;
  const int64_t ee = live ? e : 0;
  const int j = (int)(ee / MM), ab = (int)(ee - (int64_t)j * MM), ia = ab / M, ib = ab - ia * M;
  double2 acc = make_double2(0.0, 0.0);
  // history term: sum_m w_{n,m} Sigma^R(n,m)_ax G^|(m,j)_xb
  if (DF) {
    DfSum sum;
    for (int m = live ? part : n + 1; m <= n; m += kParts) {
      const float4* aw = a.Awf + (int64_t)m * MM + ia * M;
      const double* gx = a.Gx + (((int64_t)m * N + j) * MM) * 2;
      for (int x0 = 0; x0 < M; x0 += kChains)
#pragma unroll
        for (int i = 0; i < kChains; ++i)
          if (x0 + i < M) df::cmac(sum.re[i], sum.im[i], aw[x0 + i], df::c2f(ld2(gx + 2 * ((x0 + i) * M + ib))));
    }
    acc = sum.value();
  } else {
    for (int m = live ? part : n + 1; m <= n; m += kParts) {
      const double* aw = a.Aw + ((int64_t)m * MM + ia * M) * 2;  // w_{n,m} Sigma^R(n,m)
      const double* gx = a.Gx + (((int64_t)m * N + j) * MM) * 2;
      for (int x = 0; x < M; ++x) cfma4(acc, ld2(aw + 2 * x), ld2(gx + 2 * (x * M + ib)));
    }
  }
  // Matsubara convolution, split at s = tau_j
  for (int k = live ? part : N; k < N; k += kParts) {
    const double* sk = a.Smix + ((int64_t)k * MM + ia * M) * 2;
    if (k <= j) {  // G^M(tau_k - tau_j) = -G^M(tau_{N-1+k-j})
      const double w = -a.left[(int64_t)j * N + k];
      const double* gm = a.GM + (int64_t)(N - 1 + k - j) * MM * 2;
      for (int x = 0; x < M; ++x) cfma(acc, w, ld2(sk + 2 * x), ld2(gm + 2 * (x * M + ib)));
    }
    if (k >= j) {
      const double w = a.left[(int64_t)(N - 1 - j) * N + (N - 1 - k)];
      const double* gm = a.GM + (int64_t)(k - j) * MM * 2;
      for (int x = 0; x < M; ++x) cfma(acc, w, ld2(sk + 2 * x), ld2(gm + 2 * (x * M + ib)));
    }
  }
  if (!reduce_parts<kParts>(acc) || !live) return;
  const double* gn = a.Gx + (((int64_t)n * N + j) * MM) * 2;
  for (int x = 0; x < M; ++x) cfma(acc, 1.0, ld2(a.eps + 2 * (ia * M + x)), ld2(gn + 2 * (x * M + ib)));
  double* out = a.Fx + (((int64_t)(n % kRing) * N + j) * MM + ab) * 2;
  st2(out, make_double2(acc.y, -acc.x));  // -i (...)
  if (!(isfinite(acc.x) && isfinite(acc.y))) atomicOr(a.status, kStatusNumeric);
}

__global__ void __launch_bounds__(kThThreads) th_adams(ThermalArgs a, int corrector) {
  const int M = a.M, MM = M * M, N = a.N, n = a.n;
  const int64_t e = (int64_t)blockIdx.x * kThThreads + threadIdx.x;
  if (e >= (int64_t)N * MM) return;
  const int q = a.kn < n ? a.kn : n;
  const double* w = (corrector ? a.corr : a.pred) + (q - 1) * kWTab;
  double2 g = ld2(a.Gx + ((int64_t)(n - 1) * N * MM + e) * 2);
  for (int p = 0; p < q + corrector; ++p) {
    const int jr = n - q + p;
    const double2 f = ld2(a.Fx + ((int64_t)(jr % kRing) * N * MM + e) * 2);
    g.x = fma(w[p], f.x, g.x);
    g.y = fma(w[p], f.y, g.y);
  }
  st2(a.Gx + ((int64_t)n * N * MM + e) * 2, g);
}

unsigned blocks_for(int64_t threads) { return (unsigned)((threads + kThThreads - 1) / kThThreads); }

}  // namespace

cudaError_t launch_th_sigma(const ThermalArgs& a, cudaStream_t s) {
  th_sigma<<<blocks_for((int64_t)(a.N + a.n + 1) * a.M * a.M), kThThreads, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_th_mixed(const ThermalArgs& a, cudaStream_t s) {
  const unsigned blocks = (unsigned)(((int64_t)(a.n + 1) * a.M * a.M + 31) / 32);
  if (a.df)
    th_mixed<true><<<blocks, kPartThreads, 0, s>>>(a);
  else
    th_mixed<false><<<blocks, kPartThreads, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_th_rhs(const ThermalArgs& a, cudaStream_t s) {
  const unsigned blocks = (unsigned)(((int64_t)a.N * a.M * a.M + 31) / 32);
  if (a.df)
    th_rhs<true><<<blocks, 32 * kPartsDf, 0, s>>>(a);
  else
    th_rhs<false><<<blocks, kPartThreads, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_th_adams(const ThermalArgs& a, bool corrector, cudaStream_t s) {
  th_adams<<<blocks_for((int64_t)a.N * a.M * a.M), kThThreads, 0, s>>>(a, corrector ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace kbe
