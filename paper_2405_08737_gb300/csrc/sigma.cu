// sigma.cu -- second-Born self-energy, Sec. 2, Eq. (SE), local interaction.
//
// With U_abcd = U_a delta_abcd the exchange tensor is UEx = U and Eq. (SE)
// becomes Sigma^<>_ab(t,t') = U_a U_b G^<>_ab(t,t')^2 G^><_ba(t',t).  The
// anti-Hermitian symmetry gives G^><_ba(t',t) = -conj(G^><_ab(t,t')), so
// every entry of Sigma needs only the entry (a,b) of the same block:
//   S^>_ab = -U_a U_b (G^>_ab)^2 conj(G^<_ab),
//   S^<_ab = -U_a U_b (G^<_ab)^2 conj(G^>_ab),   G^> = R + L.
// On a diagonal block (t' = t) the third factor is the stored entry
// G^><_ba(t,t) itself, as Eq. (SE) reads; it equals -conj(G^><_ab) when the
// block is exactly anti-Hermitian.
// The kernel is a pure stream over complex128 entries: 32 bytes read and
// 32 bytes written per entry.  One thread per entry per pass of a
// grid-stride loop; 16-byte (double2) accesses, fully coalesced.

#include "row_kernels.cuh"

namespace kbe {
namespace {

// Row r of triangle block p (r(r+1)/2 <= p < (r+1)(r+2)/2).
__device__ __forceinline__ int64_t tri_row(int64_t p) {
  int64_t r = (int64_t)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
  while (r * (r + 1) / 2 > p) --r;
  while ((r + 1) * (r + 2) / 2 <= p) ++r;
  return r;
}

// first_block: triangle index of the first block of the launch; diag_block:
// the one diagonal block of a row launch (relative index), or -1 when the
// launch covers whole rows of a triangle (the diagonal blocks are found
// from the triangle index).
__global__ void __launch_bounds__(256) sigma_kernel(int MM, int M, int64_t n_elem, int64_t first_block,
                                                    int64_t diag_block, const double2* __restrict__ L,
                                                    const double2* __restrict__ R,
                                                    const double* __restrict__ U,
                                                    double2* __restrict__ Sl,
                                                    double2* __restrict__ Sg, int* status) {
  bool ok = true;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_elem;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blk = e / MM;
    bool diag;
    if (diag_block >= 0) {
      diag = blk == diag_block;
    } else {
      const int64_t p = first_block + blk;
      const int64_t r = tri_row(p);
      diag = (p - r * (r + 1) / 2) == r;
    }
    ok &= rk::sigma_entry(M, MM, e, diag, L, R, U, Sl, Sg);
  }
  if (!ok) atomicOr(status, kStatusNumeric);
}

}  // namespace

// Row launch: first_block = p(n,0), n_blocks = n+1, diagonal at n.
// Whole-triangle launch: first_block = 0, n_blocks = tri(N), diag_rel = -1.
cudaError_t launch_sigma(int M, int64_t first_block, int64_t n_blocks, int64_t diag_rel, const double* L,
                         const double* R, const double* U, double* Sl, double* Sg, int* status, cudaStream_t s) {
  const int MM = M * M;
  const int64_t n_elem = n_blocks * MM;
  const int64_t off = first_block * MM;
  if (n_elem == 0) return cudaSuccess;
  int64_t blocks = (n_elem + 255) / 256;
  const int64_t cap = 152 * 16;  // a grid-stride loop beyond ~16 CTAs per SM
  if (blocks > cap) blocks = cap;
  sigma_kernel<<<(unsigned)blocks, 256, 0, s>>>(MM, M, n_elem, first_block, diag_rel, (const double2*)L + off,
                                                (const double2*)R + off, U, (double2*)Sl, (double2*)Sg, status);
  return cudaGetLastError();
}

}  // namespace kbe
