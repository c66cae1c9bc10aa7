// sigma_dense.cu -- second-Born self-energy, Sec. 2, Eq. (SE), for a general
// real four-index interaction U_ifde (chemists' order, no symmetry assumed).
//
// For one block (t_n, t_c) and one component s, with A = G^s(t_n,t_c) and
// C = G^s'(t_c,t_n) (s' the other component),
//   Sigma^s_ij = sum_{f,d,e,a,b,c} U_ifde UEx_jabc A_fb A_ea C_cd,
//   UEx_jabc = 2 U_jbac - U_jabc.
// The six-index sum is factored per pair (d,b) of the indices that link the
// two tensors:
//   T^{db}_ie = sum_f U_ifde A_fb            (real x complex, M^3 per pair)
//   P^{db}_ia = sum_e T^{db}_ie A_ea         (complex x complex)
//   Q^{db}_ja = sum_c UEx_jabc C_cd          (real x complex)
//   Sigma_ij += sum_a P^{db}_ia Q^{db}_ja    (complex x complex)
// which is 12 M^5 FP64 fused multiply-adds per (block, component) instead of
// the M^6 terms of the plain sum.  The off-diagonal third factor is
// C = -G^s'(t_n,t_c)^+ (the anti-Hermitian symmetry of Sec. 2); on the
// diagonal block it is the stored G^s'(t_n,t_n).
//
// GB300 has 2 FP64 FMA lanes per SM per clock, so this kernel is bound by the
// FP64 pipe at every M >= 3 (operands come from shared memory and L1, whose
// bandwidth is an order of magnitude above the FP64 rate).  One CTA handles
// one (block, component) unit at a time: A and C are staged in shared
// memory, and the M^2 pairs run in tiles of g pairs so that each phase has
// about 256 independent outputs for the 128 threads.  The tensors are read
// from global memory (L1/L2 resident) in layouts with the contracted index
// innermost:  Ut[d][i][e][f] = U_ifde  and  Xt[b][j][a][c] = UEx_jabc.

#include "kbe_internal.h"

namespace kbe {
namespace {

constexpr int kThreads = 128;
constexpr int kMaxAcc = (kDenseMaxM * kDenseMaxM + kThreads - 1) / kThreads;

__device__ __forceinline__ int64_t tri_row(int64_t p) {
  int64_t r = (int64_t)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
  while (r * (r + 1) / 2 > p) --r;
  while ((r + 1) * (r + 2) / 2 <= p) ++r;
  return r;
}

__device__ __forceinline__ void cfma(double2& acc, double2 x, double2 y) {
  acc.x = fma(x.x, y.x, acc.x);
  acc.x = fma(-x.y, y.y, acc.x);
  acc.y = fma(x.x, y.y, acc.y);
  acc.y = fma(x.y, y.x, acc.y);
}

__global__ void __launch_bounds__(kThreads) sigma_dense_kernel(DenseSigmaArgs a) {
  extern __shared__ double2 sm[];
  const int M = a.M, MM = M * M, g = a.g, G3 = a.g3;
  double2* sA = sm;
  double2* sC = sA + MM;
  double2* sT = sC + MM;
  double2* sQ = sT + g * MM;
  double2* sP = sQ + g * MM;
  const int tid = threadIdx.x;
  const int64_t n_units = 2 * a.n_blocks;
  bool ok = true;
  for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x) {
    const int64_t blk = u >> 1;
    const int s = (int)(u & 1);
    bool diag;
    if (a.diag_rel >= 0) {
      diag = blk == a.diag_rel;
    } else {
      const int64_t p = a.first_block + blk, r = tri_row(p);
      diag = p == r * (r + 1) / 2 + r;
    }
    const double2* Lb = a.L + blk * MM;
    const double2* Rb = a.R + blk * MM;
    for (int k = tid; k < MM; k += kThreads) {
      const double2 l = Lb[k], r = Rb[k];
      const double2 gt = make_double2(r.x + l.x, r.y + l.y);
      sA[k] = s == 0 ? l : gt;
      const double2 o = s == 0 ? gt : l;  // entry (x,y) of the other component of block (n,c)
      if (diag) {
        sC[k] = o;
      } else {
        const int x = k / M, y = k - x * M;
        sC[y * M + x] = make_double2(-o.x, o.y);
      }
    }
    __syncthreads();
    double2 acc[kMaxAcc];
#pragma unroll
    for (int k = 0; k < kMaxAcc; ++k) acc[k] = make_double2(0.0, 0.0);
    for (int q0 = 0; q0 < MM; q0 += g) {
      const int gc = min(g, MM - q0);
      const int nT = gc * MM;
      // T^{db} and Q^{db} for the pairs of this tile
      for (int o = tid; o < 2 * nT; o += kThreads) {
        const bool isQ = o >= nT;
        const int oo = isQ ? o - nT : o;
        const int p = oo / MM, rc = oo - p * MM;
        const int q = q0 + p, d = q / M, b = q - d * M;
        double2 v = make_double2(0.0, 0.0);
        if (!isQ) {
          const double* w = a.Ut + ((int64_t)d * MM + rc) * M;  // U_{i f d e}, f = 0..M-1
          for (int f = 0; f < M; ++f) {
            const double c = __ldg(w + f);
            const double2 x = sA[f * M + b];
            v.x = fma(c, x.x, v.x);
            v.y = fma(c, x.y, v.y);
          }
          sT[oo] = v;
        } else {
          const double* w = a.Xt + ((int64_t)b * MM + rc) * M;  // UEx_{j a b c}, c = 0..M-1
          for (int c = 0; c < M; ++c) {
            const double cw = __ldg(w + c);
            const double2 x = sC[c * M + d];
            v.x = fma(cw, x.x, v.x);
            v.y = fma(cw, x.y, v.y);
          }
          sQ[oo] = v;
        }
      }
      __syncthreads();
      // P^{db}_ia = sum_e T^{db}_ie A_ea
      for (int o = tid; o < nT; o += kThreads) {
        const int p = o / MM, rc = o - p * MM, i = rc / M, ca = rc - i * M;
        const double2* t = sT + p * MM + i * M;
        double2 v = make_double2(0.0, 0.0);
        for (int e = 0; e < M; ++e) cfma(v, t[e], sA[e * M + ca]);
        sP[o] = v;
      }
      __syncthreads();
      // Sigma_ij += sum_a P^{db}_ia Q^{db}_ja, pairs split over G3 groups
#pragma unroll
      for (int k = 0; k < kMaxAcc; ++k) {
        const int item = tid + k * kThreads;
        if (item < G3 * MM) {
          const int grp = item / MM, ij = item - grp * MM, i = ij / M, j = ij - i * M;
          double2 v = acc[k];
          for (int p = grp; p < gc; p += G3) {
            const double2* pp = sP + p * MM + i * M;
            const double2* qq = sQ + p * MM + j * M;
            for (int c = 0; c < M; ++c) cfma(v, pp[c], qq[c]);
          }
          acc[k] = v;
        }
      }
      __syncthreads();
    }
    double2* out = (s == 0 ? a.Sl : a.Sg) + blk * MM;
    if (G3 == 1) {
#pragma unroll
      for (int k = 0; k < kMaxAcc; ++k) {
        const int item = tid + k * kThreads;
        if (item < MM) {
          out[item] = acc[k];
          ok &= isfinite(acc[k].x) && isfinite(acc[k].y);
        }
      }
    } else {
      double2* red = sT;  // G3 * MM <= g * MM entries
#pragma unroll
      for (int k = 0; k < kMaxAcc; ++k) {
        const int item = tid + k * kThreads;
        if (item < G3 * MM) red[item] = acc[k];
      }
      __syncthreads();
      for (int ij = tid; ij < MM; ij += kThreads) {
        double2 v = red[ij];
        for (int grp = 1; grp < G3; ++grp) {
          v.x += red[grp * MM + ij].x;
          v.y += red[grp * MM + ij].y;
        }
        out[ij] = v;
        ok &= isfinite(v.x) && isfinite(v.y);
      }
    }
    __syncthreads();
  }
  if (!ok) atomicOr(a.status, kStatusNumeric);
}

struct Tiling {
  int g, g3;
  size_t smem;
};

Tiling tiling(int M) {
  const int MM = M * M;
  Tiling t;
  t.g = std::max(1, std::min(MM, 256 / MM));
  t.g3 = std::max(1, std::min(t.g, kThreads / MM));
  t.smem = (size_t)(2 + 3 * t.g) * MM * sizeof(double2);
  return t;
}

}  // namespace

size_t dense_sigma_smem(int M) { return tiling(M).smem; }

cudaError_t dense_sigma_prepare(int M) {
  const size_t smem = tiling(M).smem;
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(sigma_dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t launch_sigma_dense(int M, int64_t first_block, int64_t n_blocks, int64_t diag_rel, const double* L,
                               const double* R, const double* Ut, const double* Xt, double* Sl, double* Sg,
                               int* status, cudaStream_t s) {
  if (n_blocks == 0) return cudaSuccess;
  const Tiling t = tiling(M);
  DenseSigmaArgs a;
  a.M = M;
  a.first_block = first_block;
  a.n_blocks = n_blocks;
  a.diag_rel = diag_rel;
  a.L = (const double2*)L + first_block * M * M;
  a.R = (const double2*)R + first_block * M * M;
  a.Ut = Ut;
  a.Xt = Xt;
  a.Sl = (double2*)Sl;
  a.Sg = (double2*)Sg;
  a.status = status;
  a.g = t.g;
  a.g3 = t.g3;
  int64_t blocks = 2 * n_blocks;
  const int64_t cap = (int64_t)sm_count() * 16;
  if (blocks > cap) blocks = cap;
  sigma_dense_kernel<<<(unsigned)blocks, kThreads, t.smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace kbe
