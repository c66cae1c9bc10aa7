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
// 32 bytes written per entry, 16-byte (double2) accesses, fully coalesced;
// the products run in double-float on the FP32 pipe (row_kernels.cuh).

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
// from the triangle index).  Each CTA streams one contiguous range of
// entries, blockDim at a time; a thread keeps (block, ab) and, for whole
// triangles, the index of the next diagonal block by increments.  Five CTAs
// per SM (at most 51 registers), each thread with the next entry's loads in
// flight, keep enough bytes moving for HBM.
__global__ void __launch_bounds__(256, 5) sigma_kernel(int MM, int M, int64_t n_elem, int64_t first_block,
                                                    int64_t diag_block, const double2* __restrict__ L,
                                                    const double2* __restrict__ R,
                                                    const double* __restrict__ U,
                                                    double2* __restrict__ Sl,
                                                    double2* __restrict__ Sg, int* status) {
  const int64_t per_cta = ((n_elem + gridDim.x - 1) / gridDim.x + blockDim.x - 1) / blockDim.x * blockDim.x;
  const int64_t e_end = min(n_elem, (int64_t)(blockIdx.x + 1) * per_cta);
  int64_t e = (int64_t)blockIdx.x * per_cta + threadIdx.x;
  if (e >= e_end) return;
  int64_t blk = e / MM;
  int ab = (int)(e - blk * MM);
  const int sblk = (int)(blockDim.x / MM);
  const int sab = (int)(blockDim.x - sblk * MM);
  // whole triangles: next diagonal block index at or after the current block
  int64_t r = 0, next_diag = 0;
  if (diag_block < 0) {
    const int64_t p = first_block + blk;
    r = tri_row(p);
    next_diag = r * (r + 1) / 2 + r;
  }
  bool ok = true;
  int uu_ab = ab;
  df::F2 uu = rk::sigma_uu(M, ab, U);
  // the next entry's loads are issued before this entry's arithmetic: two
  // entries' 32 bytes in flight per thread
  double2 l_next = L[e], r_next = R[e];
  for (; e < e_end; e += blockDim.x) {
    const double2 l64 = l_next, r64 = r_next;
    if (e + blockDim.x < e_end) {
      l_next = L[e + blockDim.x];
      r_next = R[e + blockDim.x];
    }
    if (ab != uu_ab) {  // never for M dividing 16: blockDim is a multiple of M^2
      uu = rk::sigma_uu(M, ab, U);
      uu_ab = ab;
    }
    bool diag;
    if (diag_block >= 0) {
      diag = blk == diag_block;
    } else {
      const int64_t p = first_block + blk;
      while (p > next_diag) {  // rows advance by at most a few blocks per iteration
        ++r;
        next_diag += r + 1;
      }
      diag = p == next_diag;
    }
    ok &= rk::sigma_entry_v(M, e, ab, diag, uu, l64, r64, L, R, Sl, Sg);
    blk += sblk;
    ab += sab;
    if (ab >= MM) {
      ab -= MM;
      ++blk;
    }
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
  const int64_t cap = (int64_t)sm_count() * 16;  // a grid-stride loop beyond ~16 CTAs per SM
  if (blocks > cap) blocks = cap;
  sigma_kernel<<<(unsigned)blocks, 256, 0, s>>>(MM, M, n_elem, first_block, diag_rel, (const double2*)L + off,
                                                (const double2*)R + off, U, (double2*)Sl, (double2*)Sg, status);
  return cudaGetLastError();
}

}  // namespace kbe
