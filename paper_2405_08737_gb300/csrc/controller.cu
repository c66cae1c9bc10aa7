// controller.cu -- device work of the adaptive time stepping (Sec. 3.1).
//
// The state of step n is row n: G^<(t_n,t_c) for c <= n and G^>(t_n,t_c) for
// c < n (G^>(t_n,t_n) is fixed by Eq. BC).  A component (s, c) starts the
// step from row n-1 at column min(c, n-1): the new column n-1 starts from
// the diagonal value G(t_{n-1},t_{n-1}), and the diagonal lesser block
// continues the diagonal.  Derivative data of component (s, c) at t_j are
// the stored right-hand sides F^s(j, c) of Eq. (KBE2) -- for j < c the
// reconstructed values above the diagonal -- and, for the diagonal block,
// D(j) = F^<(j,j) - F^<(j,j)^+.  Right-hand-side rows live in a ring of
// kRing rows [kRing][2][n_max][M][M]; row j holds its columns c <= j from the
// row evaluation and its columns c > j from the reconstruction.
//
// Kernels:
//   ctl_predict     y(0) = y_{n-1} + sum_i wp_i f_{n-q+i}        (Eq. predictor)
//   ctl_correct     y(m) = y_{n-1} + sum_i wc_i f_{n-q+1+i}      (Eq. corrector)
//                   with the weighted squares of y(m) - y(m-1) and
//                   y(m) - y(0) summed per block (WRMS norms, Eq. wrms_norm)
//   ctl_divdiff     weighted squares of two divided differences of the
//                   derivative data (error estimates at orders q-1, q+1)
//   ctl_reduce      the per-block sums in a fixed order (deterministic)
//   ctl_reconstruct F^s(j, n) for t_j < t_n: Eq. (KBE2) at points above the
//                   diagonal, one warp per output entry
// Error weights are w = 1 / (rtol |y_{n-1}| + atol) per complex entry
// (Eq. ewt, complex modulus).

#include "kbe_internal.h"

namespace kbe {
namespace {

constexpr int kCtlThreads = 256;

__device__ __forceinline__ double2 ld2(const double* p) { return *reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ void st2(double* p, double2 v) { *reinterpret_cast<double2*>(p) = v; }

struct View {
  int M, MM, n, n_max;
  const double* L;
  const double* R;
  const double* F;
  // F^s(j, c)_ab from the ring
  __device__ __forceinline__ double2 f(int s, int j, int c, int ab) const {
    return ld2(F + ((((int64_t)(j % kRing) * 2 + s) * n_max + c) * MM + ab) * 2);
  }
  // derivative of component (s, c) of row n at t_j
  __device__ __forceinline__ double2 deriv(int s, int j, int c, int a, int b) const {
    if (s == 0 && c == n) {
      const double2 x = f(0, j, j, a * M + b), y = f(0, j, j, b * M + a);
      return make_double2(x.x - y.x, x.y + y.y);  // F - F^+ of the block
    }
    return f(s, j, c, a * M + b);
  }
  // starting value of component (s, c): row n-1, column min(c, n-1)
  __device__ __forceinline__ double2 y0(int s, int c, int ab) const {
    const int cc = c < n - 1 ? c : n - 1;
    const int64_t off = (tri(n - 1, cc) * MM + ab) * 2;
    const double2 l = ld2(L + off);
    if (s == 0) return l;
    const double2 r = ld2(R + off);
    return make_double2(r.x + l.x, r.y + l.y);
  }
};

__device__ __forceinline__ double weight(double2 y, double rtol, double atol) {
  return 1.0 / (rtol * sqrt(y.x * y.x + y.y * y.y) + atol);
}

// deterministic block sum of two values; thread 0 writes partial[blockIdx]
__device__ __forceinline__ void block_sum2(double a, double b, double* partial) {
  __shared__ double sa[kCtlThreads], sb[kCtlThreads];
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int s = kCtlThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sa[threadIdx.x] += sa[threadIdx.x + s];
      sb[threadIdx.x] += sb[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = sa[0];
    partial[2 * blockIdx.x + 1] = sb[0];
  }
}

__global__ void __launch_bounds__(kCtlThreads) ctl_predict(CtlArgs a) {
  const View v{a.M, a.M * a.M, a.n, a.n_max, a.L, a.R, a.F};
  const int64_t e = (int64_t)blockIdx.x * kCtlThreads + threadIdx.x;
  if (e >= (int64_t)(a.n + 1) * v.MM) return;
  const int c = (int)(e / v.MM), ab = (int)(e - (int64_t)c * v.MM), ia = ab / a.M, ib = ab - ia * a.M;
  const int n = a.n, q = a.q;
  double2 y[2];
  y[1] = make_double2(0.0, 0.0);
  for (int s = 0; s < 2; ++s) {
    if (s == 1 && c == n) break;
    double2 acc = v.y0(s, c, ab);
    for (int i = 0; i < q; ++i) {
      const double2 d = v.deriv(s, n - q + i, c, ia, ib);
      acc.x = fma(a.wp[i], d.x, acc.x);
      acc.y = fma(a.wp[i], d.y, acc.y);
    }
    y[s] = acc;
    st2(a.ypred + (((int64_t)s * (n + 1) + c) * v.MM + ab) * 2, acc);
    st2(a.ycur + (((int64_t)s * (n + 1) + c) * v.MM + ab) * 2, acc);
  }
  const int64_t off = (tri(n, c) * v.MM + ab) * 2;
  st2(a.L + off, y[0]);
  if (c < n) st2(a.R + off, make_double2(y[1].x - y[0].x, y[1].y - y[0].y));
  else st2(a.R + off, make_double2(0.0, ia == ib ? -1.0 : 0.0));
}

__global__ void __launch_bounds__(kCtlThreads) ctl_correct(CtlArgs a) {
  const View v{a.M, a.M * a.M, a.n, a.n_max, a.L, a.R, a.F};
  const int64_t e = (int64_t)blockIdx.x * kCtlThreads + threadIdx.x;
  double dsq = 0.0, esq = 0.0;
  if (e < (int64_t)(a.n + 1) * v.MM) {
    const int c = (int)(e / v.MM), ab = (int)(e - (int64_t)c * v.MM), ia = ab / a.M, ib = ab - ia * a.M;
    const int n = a.n, q = a.q;
    double2 y[2];
    y[1] = make_double2(0.0, 0.0);
    bool ok = true;
    for (int s = 0; s < 2; ++s) {
      if (s == 1 && c == n) break;
      const double2 start = v.y0(s, c, ab);
      double2 acc = start;
      for (int i = 0; i < q; ++i) {
        const double2 d = v.deriv(s, n - q + 1 + i, c, ia, ib);
        acc.x = fma(a.wc[i], d.x, acc.x);
        acc.y = fma(a.wc[i], d.y, acc.y);
      }
      y[s] = acc;
      const double w = weight(start, a.rtol, a.atol);
      double* pc = a.ycur + (((int64_t)s * (n + 1) + c) * v.MM + ab) * 2;
      const double2 prev = ld2(pc), pred = ld2(a.ypred + (((int64_t)s * (n + 1) + c) * v.MM + ab) * 2);
      const double dx = (acc.x - prev.x) * w, dy = (acc.y - prev.y) * w;
      const double ex = (acc.x - pred.x) * w, ey = (acc.y - pred.y) * w;
      dsq += dx * dx + dy * dy;
      esq += ex * ex + ey * ey;
      st2(pc, acc);
      ok &= isfinite(acc.x) && isfinite(acc.y);
    }
    const int64_t off = (tri(n, c) * v.MM + ab) * 2;
    st2(a.L + off, y[0]);
    if (c < n) st2(a.R + off, make_double2(y[1].x - y[0].x, y[1].y - y[0].y));
    if (!ok) atomicOr(a.status, kStatusNumeric);
  }
  block_sum2(dsq, esq, a.partial);
}

__global__ void __launch_bounds__(kCtlThreads) ctl_divdiff(CtlArgs a) {
  const View v{a.M, a.M * a.M, a.n, a.n_max, a.L, a.R, a.F};
  const int64_t e = (int64_t)blockIdx.x * kCtlThreads + threadIdx.x;
  double s1 = 0.0, s2 = 0.0;
  if (e < (int64_t)(a.n + 1) * v.MM) {
    const int c = (int)(e / v.MM), ab = (int)(e - (int64_t)c * v.MM), ia = ab / a.M, ib = ab - ia * a.M;
    const int n = a.n;
    for (int s = 0; s < 2; ++s) {
      if (s == 1 && c == n) break;
      const double w = weight(v.y0(s, c, ab), a.rtol, a.atol);
      double2 u = make_double2(0.0, 0.0), z = make_double2(0.0, 0.0);
      for (int i = 0; i <= a.q1; ++i) {
        const double2 d = v.deriv(s, n - i, c, ia, ib);
        u.x = fma(a.wp[i], d.x, u.x);
        u.y = fma(a.wp[i], d.y, u.y);
      }
      for (int i = 0; i <= a.q2; ++i) {
        const double2 d = v.deriv(s, n - i, c, ia, ib);
        z.x = fma(a.wc[i], d.x, z.x);
        z.y = fma(a.wc[i], d.y, z.y);
      }
      if (a.q1 >= 0) s1 += (u.x * u.x + u.y * u.y) * w * w;
      if (a.q2 >= 0) s2 += (z.x * z.x + z.y * z.y) * w * w;
    }
  }
  block_sum2(s1, s2, a.partial);
}

__global__ void __launch_bounds__(kCtlThreads) ctl_reduce(const double* partial, int n_part, double* out) {
  __shared__ double sa[kCtlThreads], sb[kCtlThreads];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n_part; i += kCtlThreads) {
    a += partial[2 * i];
    b += partial[2 * i + 1];
  }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int s = kCtlThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sa[threadIdx.x] += sa[threadIdx.x + s];
      sb[threadIdx.x] += sb[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sa[0];
    out[1] = sb[0];
  }
}

// One warp per output entry (j, s, a, b), j = jlo .. n-1:
//   I^s(j,n) = sum_{m<=j} w_{j,m} Sigma^R(j,m) G^s(m,n) + sum_{m<=n} w_{n,m} Sigma^s(j,m) G^A(m,n),
//   F^s(j,n) = -i (eps(t_j) G^s(j,n) + I^s(j,n)),
// with G^s(m,n) = -G^s(n,m)^+ (m < n), G^A(m,n) = G^R(n,m)^+, Sigma^s(j,m) = -Sigma^s(m,j)^+ (m > j).
__global__ void __launch_bounds__(kCtlThreads) ctl_reconstruct(ReconArgs r) {
  const int M = r.M, MM = M * M, n = r.n;
  const int lane = threadIdx.x & 31;
  const int64_t item = ((int64_t)blockIdx.x * kCtlThreads + threadIdx.x) >> 5;
  const int64_t n_items = (int64_t)(n - r.jlo) * 2 * MM;
  if (item >= n_items) return;  // whole warps leave together
  const int jj = (int)(item / (2 * MM));
  const int rem = (int)(item - (int64_t)jj * 2 * MM);
  const int s = rem / MM, ab = rem - s * MM, ia = ab / M, ib = ab - ia * M;
  const int j = r.jlo + jj;
  const int64_t sstride = (int64_t)r.n_max * MM * 2;  // doubles per s-row of the self-energy ring
  auto sig = [&](int ss, int row, int col, int x, int y) -> double2 {  // Sigma^ss(t_row, t_col)_xy, col <= row
    return ld2(r.Sring + ((int64_t)(row % kRing) * 2 + ss) * sstride + ((int64_t)col * MM + x * M + y) * 2);
  };
  auto gnm = [&](int ss, int m, int x, int y) -> double2 {  // G^ss(t_n, t_m)_xy, m <= n
    const int64_t off = (tri(n, m) * MM + x * M + y) * 2;
    const double2 l = ld2(r.L + off);
    if (ss == 0) return l;
    const double2 rr = ld2(r.R + off);
    return make_double2(rr.x + l.x, rr.y + l.y);
  };
  double re = 0.0, im = 0.0;
  for (int m = lane; m <= n; m += 32) {
    if (m <= j) {  // Sigma^R(j,m) G^s(m,n), G^s(m,n)_xb = -conj(G^s(n,m)_bx)
      const double w = r.w.at(j, m);
      for (int x = 0; x < M; ++x) {
        const double2 sg = sig(1, j, m, ia, x), sl = sig(0, j, m, ia, x);
        const double2 A = make_double2(sg.x - sl.x, sg.y - sl.y);
        const double2 g = gnm(s, m, ib, x);
        const double2 B = make_double2(-g.x, g.y);
        re = fma(w * A.x, B.x, re);
        re = fma(-w * A.y, B.y, re);
        im = fma(w * A.x, B.y, im);
        im = fma(w * A.y, B.x, im);
      }
    }
    {  // Sigma^s(j,m) G^A(m,n), G^A(m,n)_xb = conj(R(n,m)_bx)
      const double w = r.w.at(n, m);
      for (int x = 0; x < M; ++x) {
        double2 A;
        if (m <= j) {
          A = sig(s, j, m, ia, x);
        } else {
          const double2 t = sig(s, m, j, x, ia);
          A = make_double2(-t.x, t.y);
        }
        const double2 rr = ld2(r.R + (tri(n, m) * MM + ib * M + x) * 2);
        const double2 B = make_double2(rr.x, -rr.y);
        re = fma(w * A.x, B.x, re);
        re = fma(-w * A.y, B.y, re);
        im = fma(w * A.x, B.y, im);
        im = fma(w * A.y, B.x, im);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, o);
    im += __shfl_down_sync(0xffffffffu, im, o);
  }
  if (lane != 0) return;
  // eps(t_j) G^s(j,n), G^s(j,n)_xb = -conj(G^s(n,j)_bx)
  const double* eps = r.eps_ring + (int64_t)(j % kRing) * MM * 2;
  for (int x = 0; x < M; ++x) {
    const double2 A = ld2(eps + (ia * M + x) * 2);
    const double2 g = gnm(s, j, ib, x);
    const double2 B = make_double2(-g.x, g.y);
    re += A.x * B.x - A.y * B.y;
    im += A.x * B.y + A.y * B.x;
  }
  // F = -i (eps G + I), stored in ring row j at column n
  double* out = r.F + ((((int64_t)(j % kRing) * 2 + s) * r.n_max + n) * MM + ab) * 2;
  st2(out, make_double2(im, -re));
  if (!(isfinite(re) && isfinite(im))) atomicOr(r.status, kStatusNumeric);
}

int row_blocks(int n, int M) { return (int)(((int64_t)(n + 1) * M * M + kCtlThreads - 1) / kCtlThreads); }

}  // namespace

int ctl_partial_count(int n_max, int M) { return row_blocks(n_max - 1, M); }

cudaError_t launch_ctl_predict(const CtlArgs& a, cudaStream_t s) {
  ctl_predict<<<row_blocks(a.n, a.M), kCtlThreads, 0, s>>>(a);
  return cudaGetLastError();
}

// correction; then out[0] = sum |dy w|^2 over the row, out[1] = sum |(y - y(0)) w|^2
cudaError_t launch_ctl_correct(const CtlArgs& a, double* out, cudaStream_t s) {
  const int nb = row_blocks(a.n, a.M);
  ctl_correct<<<nb, kCtlThreads, 0, s>>>(a);
  ctl_reduce<<<1, kCtlThreads, 0, s>>>(a.partial, nb, out);
  return cudaGetLastError();
}

// out[0], out[1]: weighted squares of the divided differences with
// coefficients a.wp[0..q1] and a.wc[0..q2] over t_n, t_{n-1}, ... (q < 0: skipped)
cudaError_t launch_ctl_divdiff(const CtlArgs& a, double* out, cudaStream_t s) {
  const int nb = row_blocks(a.n, a.M);
  ctl_divdiff<<<nb, kCtlThreads, 0, s>>>(a);
  ctl_reduce<<<1, kCtlThreads, 0, s>>>(a.partial, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_ctl_reconstruct(const ReconArgs& r, cudaStream_t s) {
  const int64_t items = (int64_t)(r.n - r.jlo) * 2 * r.M * r.M;
  if (items <= 0) return cudaSuccess;
  const int64_t blocks = (items * 32 + kCtlThreads - 1) / kCtlThreads;
  ctl_reconstruct<<<(unsigned)blocks, kCtlThreads, 0, s>>>(r);
  return cudaGetLastError();
}

}  // namespace kbe
