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

#include "row_kernels.cuh"

namespace kbe {
namespace {

__global__ void fock_kernel(StepArgs a) {
  for (int ab = threadIdx.x; ab < a.M * a.M; ab += blockDim.x) rk::fock_entry(a, ab);
}

__global__ void __launch_bounds__(256) predictor_kernel(StepArgs a) {
  const int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lin < (int64_t)(a.n + 1) * a.M * a.M) rk::adams_entry(a, lin, false);
}

__global__ void __launch_bounds__(256) rhs_kernel(StepArgs a) {
  const int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lin >= (int64_t)(a.n + 1) * a.M * a.M) return;
  if (!rk::rhs_entry(a, lin)) atomicOr(a.status, kStatusNumeric);
}

__global__ void __launch_bounds__(256) corrector_kernel(StepArgs a) {
  const int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (lin < (int64_t)(a.n + 1) * a.M * a.M) rk::adams_entry(a, lin, true);
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256); }

// Row 0 of an uncorrelated start: G^<(0,0) = i rho0 and G^R(0,0) = -i 1
// (Eq. BC with theta(0) = 1).
__global__ void init_row0_kernel(int M, const double2* __restrict__ rho, double2* __restrict__ L,
                                 double2* __restrict__ R) {
  for (int ab = threadIdx.x; ab < M * M; ab += blockDim.x) {
    const double2 p = rho[ab];
    L[ab] = make_double2(-p.y, p.x);
    R[ab] = make_double2(0.0, ab / M == ab % M ? -1.0 : 0.0);
  }
}

}  // namespace

cudaError_t launch_init_row0(int M, const double* rho, double* L, double* R, cudaStream_t s) {
  init_row0_kernel<<<1, 256, 0, s>>>(M, (const double2*)rho, (double2*)L, (double2*)R);
  return cudaGetLastError();
}

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
