// stepper.cu -- right-hand side, predictor and corrector of one KBE step.
//
// Row n of the lower triangle is advanced along t at fixed t_c (the
// t-derivative of Eq. (KBE2)):
//   dG^s(t,t_c)/dt = F^s = -i ( eps(t) G^s(t,t_c) + I^s(t,t_c) ),
// and the diagonal with the total derivative of G^<(t,t), which by the
// anti-Hermitian symmetry is D = F^< - (F^<)^+ = -i[eps,G^<] - i(I^< + I^<^+).
// The step is the integral form of a variable-order Adams method on the
// nonuniform grid: G(n,c) = G(n-1,c) + int_{t_{n-1}}^{t_n} F, with F
// interpolated through stored right-hand-side rows (predictor: rows
// n-q..n-1, corrector: rows n-kap..n, kap = min(k_n, n-c) so that only
// points on or below the diagonal are used).  The weights come from the
// same Vandermonde solves as the history weights (Sec. 3.2).
//
// All kernels here are elementwise over the (2n+1) M^2 entries of a row.

#include "kbe_internal.h"

namespace kbe {
namespace {

__device__ __forceinline__ double2 ldd(const double* p) { return *reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ void std2(double* p, double2 v) { *reinterpret_cast<double2*>(p) = v; }

__device__ __forceinline__ const double* ring_at(const StepArgs& a, int j, int s, int c, int ab) {
  const int MM = a.M * a.M;
  const int64_t slot = (j - a.f_base) % a.f_rows;
  return a.F + (((slot * 2 + s) * a.n_max + c) * MM + ab) * 2;
}

// eps(t_n) = h0 + E(t_n) diag(v) + diag(U_a Im L(n,n)_aa)
__global__ void fock_kernel(StepArgs a) {
  const int M = a.M, MM = M * M;
  const double* Lnn = a.L + tri(a.n, a.n) * MM * 2;
  for (int ab = threadIdx.x; ab < MM; ab += blockDim.x) {
    const int i = ab / M, j = ab - i * M;
    double2 e = ldd(a.h0 + 2 * ab);
    if (i == j) e.x += a.field * a.v[i] + a.U[i] * Lnn[2 * ab + 1];
    std2(a.eps + 2 * ab, e);
  }
}

__global__ void __launch_bounds__(256) predictor_kernel(StepArgs a) {
  const int M = a.M, MM = M * M, n = a.n;
  const int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lin >= (int64_t)(n + 1) * MM) return;
  const int c = (int)(lin / MM), ab = (int)(lin - (int64_t)c * MM);
  const int ia = ab / M, ib = ab - ia * M;
  double* Ln = a.L + (tri(n, c) * MM + ab) * 2;
  double* Rn = a.R + (tri(n, c) * MM + ab) * 2;
  if (c < n) {
    const int q = min(a.kn, n - c);
    const double* w = a.pred + (q - 1) * kWTab;
    const double2 l0 = ldd(a.L + (tri(n - 1, c) * MM + ab) * 2);
    const double2 r0 = ldd(a.R + (tri(n - 1, c) * MM + ab) * 2);
    double2 gl = l0, gg = make_double2(r0.x + l0.x, r0.y + l0.y);
    for (int p = 0; p < q; ++p) {
      const int j = n - q + p;
      const double2 fl = ldd(ring_at(a, j, 0, c, ab)), fg = ldd(ring_at(a, j, 1, c, ab));
      gl.x = fma(w[p], fl.x, gl.x); gl.y = fma(w[p], fl.y, gl.y);
      gg.x = fma(w[p], fg.x, gg.x); gg.y = fma(w[p], fg.y, gg.y);
    }
    std2(Ln, gl);
    std2(Rn, make_double2(gg.x - gl.x, gg.y - gl.y));
  } else {
    const int q = min(a.kn, n);
    const double* w = a.pred + (q - 1) * kWTab;
    double2 gl = ldd(a.L + (tri(n - 1, n - 1) * MM + ab) * 2);
    const int ba = ib * M + ia;
    for (int p = 0; p < q; ++p) {
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

// F^s(n,c)_ab = -i ( sum_x eps_ax G^s(n,c)_xb + I^s(n,c)_ab ),  G^> = R + L
__global__ void __launch_bounds__(256) rhs_kernel(StepArgs a) {
  const int M = a.M, MM = M * M, n = a.n;
  const int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lin >= (int64_t)(n + 1) * MM) return;
  const int c = (int)(lin / MM), ab = (int)(lin - (int64_t)c * MM);
  const int ia = ab / M, ib = ab - ia * M;
  const double* Lb = a.L + tri(n, c) * MM * 2;
  const double* Rb = a.R + tri(n, c) * MM * 2;
  double2 sl = ldd(a.I + ((int64_t)c * MM + ab) * 2);
  double2 sg = ldd(a.I + (((int64_t)(n + 1) + c) * MM + ab) * 2);
  bool bad = false;
  for (int x = 0; x < M; ++x) {
    const double2 e = ldd(a.eps + 2 * (ia * M + x));
    const double2 l = ldd(Lb + 2 * (x * M + ib));
    const double2 r = ldd(Rb + 2 * (x * M + ib));
    const double gr = r.x + l.x, gi = r.y + l.y;
    sl.x += e.x * l.x - e.y * l.y; sl.y += e.x * l.y + e.y * l.x;
    sg.x += e.x * gr - e.y * gi;   sg.y += e.x * gi + e.y * gr;
  }
  // -i (x + i y) = y - i x
  const double2 fl = make_double2(sl.y, -sl.x), fg = make_double2(sg.y, -sg.x);
  bad = !(isfinite(fl.x) && isfinite(fl.y) && isfinite(fg.x) && isfinite(fg.y));
  std2(const_cast<double*>(ring_at(a, n, 0, c, ab)), fl);
  std2(const_cast<double*>(ring_at(a, n, 1, c, ab)), fg);
  if (bad) atomicOr(a.status, kStatusNumeric);
}

__global__ void __launch_bounds__(256) corrector_kernel(StepArgs a) {
  const int M = a.M, MM = M * M, n = a.n;
  const int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lin >= (int64_t)(n + 1) * MM) return;
  const int c = (int)(lin / MM), ab = (int)(lin - (int64_t)c * MM);
  const int ia = ab / M, ib = ab - ia * M;
  double* Ln = a.L + (tri(n, c) * MM + ab) * 2;
  double* Rn = a.R + (tri(n, c) * MM + ab) * 2;
  if (c < n) {
    const int kap = min(a.kn, n - c);
    const double* w = a.corr + (kap - 1) * kWTab;
    const double2 l0 = ldd(a.L + (tri(n - 1, c) * MM + ab) * 2);
    const double2 r0 = ldd(a.R + (tri(n - 1, c) * MM + ab) * 2);
    double2 gl = l0, gg = make_double2(r0.x + l0.x, r0.y + l0.y);
    for (int p = 0; p <= kap; ++p) {
      const int j = n - kap + p;
      const double2 fl = ldd(ring_at(a, j, 0, c, ab)), fg = ldd(ring_at(a, j, 1, c, ab));
      gl.x = fma(w[p], fl.x, gl.x); gl.y = fma(w[p], fl.y, gl.y);
      gg.x = fma(w[p], fg.x, gg.x); gg.y = fma(w[p], fg.y, gg.y);
    }
    std2(Ln, gl);
    std2(Rn, make_double2(gg.x - gl.x, gg.y - gl.y));
  } else {
    const int kap = min(a.kn, n);
    const double* w = a.corr + (kap - 1) * kWTab;
    double2 gl = ldd(a.L + (tri(n - 1, n - 1) * MM + ab) * 2);
    const int ba = ib * M + ia;
    for (int p = 0; p <= kap; ++p) {
      const int j = n - kap + p;
      const double2 f = ldd(ring_at(a, j, 0, j, ab)), ft = ldd(ring_at(a, j, 0, j, ba));
      gl.x = fma(w[p], f.x - ft.x, gl.x);
      gl.y = fma(w[p], f.y + ft.y, gl.y);
    }
    std2(Ln, gl);
    std2(Rn, make_double2(0.0, ia == ib ? -1.0 : 0.0));
  }
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

cudaError_t launch_fock(const StepArgs& a, cudaStream_t s) {
  fock_kernel<<<1, 256, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_predictor(const StepArgs& a, cudaStream_t s) {
  predictor_kernel<<<blocks_for((int64_t)(a.n + 1) * a.M * a.M), 256, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_rhs(const StepArgs& a, cudaStream_t s) {
  rhs_kernel<<<blocks_for((int64_t)(a.n + 1) * a.M * a.M), 256, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_rhs_corrector(const StepArgs& a, cudaStream_t s) {
  rhs_kernel<<<blocks_for((int64_t)(a.n + 1) * a.M * a.M), 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  corrector_kernel<<<blocks_for((int64_t)(a.n + 1) * a.M * a.M), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace kbe
