// adaptive.cu -- adaptive history orders (Sec. 3.2) on the device.
//
// In every fixed-point sweep of step n, after the self-energy row, the order
// of the history quadrature over [t_{n-1}, t_n] is chosen.  A wide kernel
// forms the test integrand (one warp per point and entry, lanes over the
// contracted orbital index) into a small scratch array; one block then forms
//   u(t_l) = G^R(t_n, t_l) Sigma^<(t_l, t_n) + G^<(t_n, t_l) Sigma^A(t_l, t_n),
// l = n-kmax .. n (kmax = min(K, n)), the test integrals of every order
//   I^(k) = sum_j w^(k)_j u(t_{n-k+j}),  k = 1..kmax,
// and takes k_opt = argmin_{k >= 2} |I^(k) - I^(k-1)| (max norm over the
// M x M entries), the lowest order among differences within 64 eps of the
// largest test integral from the minimum.  Then it writes the band row n of
// the composite weights from row n-1 and the local weights of order k_opt
// (the row recursion of Sec. 3.2), and the settled weight of the point that
// leaves the band.

#include "kbe_internal.h"

namespace kbe {
namespace {

constexpr int kSelThreads = 256;

struct Cz {
  double re, im;
};
__device__ __forceinline__ Cz ldz(const double* p) { return Cz{p[0], p[1]}; }

// u(t_l)_ab for l = n-kmax+i, i = 0..kmax: warp w = i * M^2 + ab.
__global__ void __launch_bounds__(kSelThreads) select_u_kernel(SelectArgs a) {
  const int M = a.M, MM = M * M, n = a.n;
  const int kmax = a.K < n ? a.K : n;
  const int lane = threadIdx.x & 31;
  const int w = (int)(((int64_t)blockIdx.x * kSelThreads + threadIdx.x) >> 5);
  if (w >= (kmax + 1) * MM) return;  // whole warps leave together
  const int i = w / MM, e = w - i * MM, ia = e / M, ib = e - ia * M;
  const int l = n - kmax + i;
  const double* Rb = a.R + tri(n, l) * MM * 2;
  const double* Lb = a.L + tri(n, l) * MM * 2;
  const double* sl = a.Sl + (int64_t)l * MM * 2;
  const double* sg = a.Sg + (int64_t)l * MM * 2;
  Cz acc{0.0, 0.0};
  for (int x = lane; x < M; x += 32) {
    const Cz r = ldz(Rb + 2 * (ia * M + x)), g = ldz(Lb + 2 * (ia * M + x));
    // Sigma^<(t_l, t_n)_xb: the stored entry on the diagonal, -conj(S^<(n,l)_bx) below it
    Cz s;
    if (l == n) s = ldz(sl + 2 * (x * M + ib));
    else { const Cz v = ldz(sl + 2 * (ib * M + x)); s = Cz{-v.re, v.im}; }
    // Sigma^A(t_l, t_n)_xb = conj(Sigma^R(n,l)_bx), Sigma^R = S^> - S^<
    const Cz vg = ldz(sg + 2 * (ib * M + x)), vl = ldz(sl + 2 * (ib * M + x));
    const Cz q{vg.re - vl.re, -(vg.im - vl.im)};
    acc.re += r.re * s.re - r.im * s.im + g.re * q.re - g.im * q.im;
    acc.im += r.re * s.im + r.im * s.re + g.re * q.im + g.im * q.re;
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc.re += __shfl_down_sync(0xffffffffu, acc.re, o);
    acc.im += __shfl_down_sync(0xffffffffu, acc.im, o);
  }
  if (lane == 0) {
    a.u[2 * w] = acc.re;
    a.u[2 * w + 1] = acc.im;
  }
}

__global__ void __launch_bounds__(kSelThreads) select_order_kernel(SelectArgs a) {
  const int M = a.M, MM = M * M, n = a.n;
  const int kmax = a.K < n ? a.K : n;
  __shared__ double red[kSelThreads];
  __shared__ double dk[kMaxOrder + 1];
  __shared__ double s_mag;
  __shared__ int s_k;
  double my_d[kMaxOrder + 1];
  double my_mag = 0.0;
  for (int k = 0; k <= kMaxOrder; ++k) my_d[k] = 0.0;
  if (kmax >= 2) {
    for (int e = threadIdx.x; e < MM; e += blockDim.x) {
      Cz u[kMaxOrder + 1];
      for (int i = 0; i <= kmax; ++i) u[i] = ldz(a.u + 2 * (i * MM + e));
      Cz prev{0.0, 0.0};
      for (int k = 1; k <= kmax; ++k) {
        const double* w = a.hist + (k - 1) * kWTab;
        Cz I{0.0, 0.0};
        for (int j = 0; j <= k; ++j) {
          const Cz v = u[kmax - k + j];
          I.re += w[j] * v.re;
          I.im += w[j] * v.im;
        }
        my_mag = fmax(my_mag, sqrt(I.re * I.re + I.im * I.im));
        if (k >= 2) {
          const double dr = I.re - prev.re, di = I.im - prev.im;
          my_d[k] = fmax(my_d[k], sqrt(dr * dr + di * di));
        }
        prev = I;
      }
    }
  }
  // block maxima of the differences and of the test integrals
  for (int k = 2; k <= kmax + 1; ++k) {
    red[threadIdx.x] = k <= kmax ? my_d[k] : my_mag;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      if (k <= kmax) dk[k] = red[0];
      else s_mag = red[0];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int kopt = 1;
    if (kmax >= 2) {
      double dmin = dk[2];
      for (int k = 3; k <= kmax; ++k) dmin = fmin(dmin, dk[k]);
      const double tol = 64.0 * 2.220446049250313e-16 * s_mag;
      kopt = kmax;
      for (int k = 2; k <= kmax; ++k)
        if (dk[k] <= dmin + tol) { kopt = k; break; }
    }
    s_k = kopt;
    a.korder[n] = kopt;
    // band row n from row n-1 plus the local weights of order kopt
    const int bw = a.band_w;
    const double* wk = a.hist + (kopt - 1) * kWTab;
    for (int d = 0; d < bw; ++d) {
      const int m = n - d;
      double v = 0.0;
      if (m >= 0) {
        if (d >= 1) v = a.band[(int64_t)(n - 1) * bw + (d - 1)];
        if (d <= kopt) v += wk[kopt - d];
      }
      a.band[(int64_t)n * bw + d] = v;
    }
    if (n - bw >= 0) a.wbar[n - bw] = a.band[(int64_t)(n - 1) * bw + (bw - 1)];  // final from now on
  }
}

}  // namespace

cudaError_t launch_select_order(const SelectArgs& a, cudaStream_t s, int* launches) {
  const int kmax = a.K < a.n ? a.K : a.n;
  *launches = 1;
  if (kmax >= 2) {
    const int64_t warps = (int64_t)(kmax + 1) * a.M * a.M;
    select_u_kernel<<<(unsigned)((warps * 32 + kSelThreads - 1) / kSelThreads), kSelThreads, 0, s>>>(a);
    *launches = 2;
  }
  select_order_kernel<<<1, kSelThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace kbe
