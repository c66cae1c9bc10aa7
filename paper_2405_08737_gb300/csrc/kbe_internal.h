// kbe_internal.h -- definitions shared by the translation units of libkbe.
#pragma once

#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/kbe.h"

namespace kbe {

constexpr int kMaxOrder = KBE_MAX_ORDER;
constexpr int kRing = KBE_RING_ROWS;
constexpr int kMaxNorb = 64;
constexpr int kMaxSplit = 16;      // largest split of the history index m
constexpr int kMaxSplitSmall = 64; // ... for rows of at most kRunMaxRow entries (history_f64_split)
constexpr int kWTab = kMaxOrder + 1;  // row stride of the stepper weight tables
constexpr int kDenseMaxM = KBE_DENSE_MAX_NORB;  // largest norb of the dense-interaction self-energy

__host__ __device__ inline int64_t tri(int64_t r, int64_t c) { return r * (r + 1) / 2 + c; }

// Device status bits (reported by kbe_sync_status).
constexpr int kStatusNumeric = 1;
constexpr int kStatusTimeout = 2;
constexpr int kStatusInternal = 4;  // a kernel found an inconsistent launch geometry

// Read-only view of the composite weights on the device:
//   w_{c,m} = band[c * band_w + (c - m)]  if c - m < band_w,
//           = wbar[m]                     otherwise
// (Sec. 3.2: rows agree with the settled sums for m < c - K).
struct WeightsView {
  const double* wbar;
  const double* band;
  int band_w;
  __device__ __forceinline__ double at(int c, int m) const {
    const int d = c - m;
    return d < band_w ? band[(int64_t)c * band_w + d] : wbar[m];
  }
};

// Host-side grid data (FP64), also the source of the device tables.
struct HostGrid {
  int n_t = 0;
  int K = 0;                      // largest effective order on the grid
  std::vector<double> t;
  std::vector<int> order;         // order[l], l >= 1 (order[0] = 0)
  std::vector<double> wbar;       // settled composite weights, [n_t]
  std::vector<double> band;       // w_{c, c-j}, [n_t][K+1]
  std::vector<double> corr;       // corrector weights [n_t][kMaxOrder][kWTab]
  std::vector<double> pred;       // predictor weights [n_t][kMaxOrder][kWTab]
};

// Host FP64 weight routines (weights.cpp).  Return KBE_OK or an error code
// with a message in *err.
kbe_status local_weights(const double* tau, int k, double lo, double hi, double* w, std::string* err);
kbe_status build_grid(const double* t, const int* order, int n_t, HostGrid* g, std::string* err);

// Layout of the digit-plane buffer of the split path (history_split.cu).
struct SplitPlanes {
  int cpt_stride = 0, col_tiles = 0, qu_slots = 0;
  size_t bytes = 0;
};

// Record a context-free error message (returned by kbe_last_error(NULL) on
// the calling host thread).
void set_global_error(const char* msg);

// Streaming multiprocessors of the current device (queried once per device;
// launch heuristics size their grids from it).
int sm_count();

struct Model {
  bool set = false;
  std::vector<double> h0;   // complex MxM interleaved
  std::vector<double> U, v;
  double E0 = 0, t0 = 0, sigma = 1, omega = 0;
  double field(double t) const;   // E(t) = E0 * shape(t)
  double shape(double t) const;   // Gaussian envelope times the carrier
};

}  // namespace kbe

// The context behind the opaque handle.
struct kbe_ctx {
  int M = 0;
  int n_max = 0;
  std::string err;
  int last_launches = 0;
  kbe::HostGrid grid;
  bool grid_set = false;
  kbe::Model model;
  // device state
  int device = 0;
  double* d_wbar = nullptr;
  double* d_band = nullptr;
  double* d_corr = nullptr;
  double* d_pred = nullptr;
  double* d_h0 = nullptr;     // complex MxM
  double* d_U = nullptr;      // M
  double* d_v = nullptr;      // M
  double* d_eps = nullptr;    // complex MxM (Fock matrix of the current row)
  double* d_part = nullptr;   // FP64 slice workspace: prep rows, chunk partials [chunks][2][n_max][M][M] complex
  void* d_split = nullptr;    // split-precision workspace (digit planes of the small operands, partials)
  size_t split_bytes = 0;
  void* d_planes = nullptr;   // digit planes of the history (split path), allocated by the first split slice
  kbe::SplitPlanes planes_layout;
  bool planes_failed = false; // allocation failed once: the in-kernel conversion path is used
  bool split_planes = true;   // keep the digit-plane cache (kbe_set_split_planes)
  // Cache of the planes across KBE steps: rows < planes_rows of the arrays
  // planes_L / planes_R are encoded with their final values.
  const void* planes_L = nullptr;
  const void* planes_R = nullptr;
  int planes_rows = 0;
  // failure-path test of the next split contraction (kbe_debug_withhold_split)
  long long dbg_withhold = -1;
  long long dbg_spin = 0;
  int dbg_run_withhold = -1;     // kbe_debug_withhold_run: next cooperative run launch only
  long long dbg_run_spin = 0;
  int* d_status = nullptr;
  unsigned* d_runbar = nullptr;  // barrier counter of the cooperative small-row run kernel
  bool run_coop_refused = false; // the device refused the cooperative launch once: per-kernel steps only
  size_t part_bytes = 0;
  // reverse-mode workspace, allocated by the first adjoint call that needs it
  double* d_adj = nullptr;
  size_t adj_bytes = 0;
  // adaptive history orders (Sec. 3.2): 0 = the grid's orders; else the
  // largest order the selection may choose
  int adaptive_K = 0;
  int band_w = 0;             // width of the composite-weight band on the device
  int adaptive_rows = 0;      // band rows 0 .. adaptive_rows-1 are set
  double* d_hist = nullptr;   // local weights of every order per interval [n_max][kMaxOrder][kWTab]
  int* d_korder = nullptr;    // chosen history order per interval [n_max]
  // general four-index interaction (Eq. SE, Eq. eps); unset: the local U
  bool dense = false;
  double* d_Ut = nullptr;     // [d][i][e][f] = U_ifde
  double* d_Xt = nullptr;     // [b][j][a][c] = UEx_jabc = 2 U_jbac - U_jabc
  double* d_HF = nullptr;     // [(i,j)][(b,a)] = U_iabj - 2 U_ijba (Fock matrix)
  // adaptive time stepping: self-energy and Fock rings, iterates, sums
  double* d_ctl = nullptr;
  size_t ctl_bytes = 0;
  // thermal branch (Eq. KBE3): tau grid of th_N points on [0, th_beta]
  bool thermal = false;
  int th_N = 0, th_k = 0;
  double th_beta = 0.0;
  double* d_th = nullptr;     // GM | left | Smix | Smw | Aw [n_max][MM] | Fx [kRing][N][MM] | Gx [n_max][N][MM]
  // measurement: event pairs around each contraction kernel
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  // kbe_step_host: copy stream for the history upload and its events
  cudaStream_t up_stream = nullptr;
  cudaEvent_t up_start = nullptr;
  cudaEvent_t up_ev[16] = {};
};

namespace kbe {

// ---- launchers (each returns cudaGetLastError() after the launch) -------
cudaError_t launch_sigma(int M, int64_t first_block, int64_t n_blocks, int64_t diag_rel, const double* L,
                         const double* R, const double* U, double* Sl, double* Sg, int* status, cudaStream_t s);

// Dense-interaction self-energy (sigma_dense.cu): same launch geometry as
// launch_sigma; Ut, Xt are the reordered tensors of the context.
struct DenseSigmaArgs {
  int M;
  int64_t first_block, n_blocks, diag_rel;
  const double2* L;   // block first_block of the triangles
  const double2* R;
  const double* Ut;
  const double* Xt;
  double2* Sl;        // outputs, relative block index
  double2* Sg;
  int* status;
  int g, g3;          // pairs per tile, accumulator groups
};
cudaError_t launch_sigma_dense(int M, int64_t first_block, int64_t n_blocks, int64_t diag_rel, const double* L,
                               const double* R, const double* Ut, const double* Xt, double* Sl, double* Sg,
                               int* status, cudaStream_t s);
cudaError_t dense_sigma_prepare(int M);  // shared-memory opt-in, outside stream capture
size_t dense_sigma_smem(int M);

struct HistoryArgs {
  int M, n;
  const double* L;
  const double* R;
  const double* Sl;
  const double* Sg;
  WeightsView w;
  double* out;       // [2][n+1][M][M]
  double* part;      // workspace
  size_t part_bytes;
  int* status;
  cudaEvent_t ev_begin = nullptr;  // optional timing of the contraction kernel
  cudaEvent_t ev_end = nullptr;
  int band_lo = 0;                 // contributions of the stored rows [band_lo, band_hi) only
  int band_hi = 0x7fffffff;
};
// FP64 history slice; sets *launches to the number of kernels enqueued.
cudaError_t launch_history_f64(const HistoryArgs& a, cudaStream_t s, int* launches);
// The history slice in double-float on the FP32 pipe (KBE_DF64), same
// workspace and outputs as launch_history_f64.
cudaError_t launch_history_df(const HistoryArgs& a, cudaStream_t s, int* launches);
// Chunk partials [nchunk][2][row] summed in order into out (one launch).
cudaError_t launch_history_finish(int nchunk, int64_t row, const double* partials, double* out, int* status,
                                  cudaStream_t s, int* launches);
// The same with the output columns contracted in nranges launches, range k
// (columns [c_lo[k], c_hi[k])) after the stream waits for wait[k] (if wait
// and wait[k] are set); bitwise the same results as one launch.
cudaError_t launch_history_f64_ranges(const HistoryArgs& a, int nranges, const int* c_lo, const int* c_hi,
                                      const cudaEvent_t* wait, cudaStream_t s, int* launches);

// Split-precision history slice (history_split.cu).
struct SplitGeomHost {
  int M, n, CT, parts, cpt, tiles;
  long long U;
  int G, S;
};
struct SplitLaunch {
  int M, n;
  const double* L;
  const double* R;
  const double* Sl;
  const double* Sg;
  WeightsView w;
  double* out;
  void* work;
  size_t work_bytes;
  int* status;
  cudaEvent_t ev_begin = nullptr;
  cudaEvent_t ev_end = nullptr;
  long long withhold = -1;   // failure-path test (kbe_debug_withhold_split): unit never supplied
  long long spin_limit = 0;  // polls of a work wait before it gives up (0: the default)
};
bool split_geometry(int M, int n, SplitGeomHost* h);

// Fused split path: one persistent contraction over the work units of one or
// many systems, converting the FP64 history into digit planes inside the
// kernel (no plane buffer), then a reduction over all systems' columns.
struct FusedSystem {
  int M, n;
  const double* L;
  const double* R;
  const double* Sl;
  const double* Sg;
  WeightsView w;
  double* out;   // [2][n+1][M][M]
  void* small;   // the system's split workspace: small-operand digit planes, then their exponents
};
struct FusedPlanHost {
  std::vector<unsigned char> image;  // device image of the work list (upload before launching)
  int G = 0, n_ent = 0, max_parts = 0;
  long long total_chunks = 0, total_cols = 0, slots = 0, segments = 0;
  size_t off_sys = 0, off_lo = 0, off_tile0 = 0, off_segb = 0, off_slot = 0;
};
bool fused_build(const FusedSystem* in, int n_sys, FusedPlanHost* p);
size_t fused_part_bytes(const FusedPlanHost& p);  // partial slots the launch writes
cudaError_t launch_history_fused(const FusedPlanHost& p, const void* plan_dev, double* part, int* status,
                                 cudaStream_t s, int* launches, cudaEvent_t ev_begin = nullptr,
                                 cudaEvent_t ev_end = nullptr, long long withhold = -1, long long spin = 0);
size_t split_workspace_bytes(int M, int n_max);
cudaError_t launch_history_split(const SplitLaunch& l, cudaStream_t s, int* launches);
cudaError_t split_prepare();  // one-time kernel attributes of the current device
// Planes path: digit planes of the history encoded by a separate kernel and
// streamed into the contraction (single systems; needs split_planes_bytes).
bool split_planes_layout(int M, int n_max, SplitPlanes* p);
// Encodes the units that involve rows >= r0 (r0 = 0: all), then contracts.
cudaError_t launch_history_split2(const SplitLaunch& l, const SplitPlanes& layout, void* planes, int r0,
                                  cudaStream_t s, int* launches);

struct StepArgs {
  int M, n, K;
  int kn;            // order of interval n
  double field;      // E(t_n)
  double* L;
  double* R;
  double* F;         // right-hand-side rows [f_rows][2][n_max][M][M]; row j in slot (j - f_base) % f_rows
  int n_max;
  int f_base;        // 0 for the ring (f_rows = kRing); the first stored row for a row store
  int f_rows;
  const double* I;   // [2][n+1][M][M]
  const double* h0;
  const double* U;
  const double* HF;    // dense Fock tensor [(i,j)][(b,a)] or NULL for the local U
  const double* v;
  double* eps;
  const double* corr;  // weights of interval n: [kMaxOrder][kWTab]
  const double* pred;
  int* status;
};
cudaError_t launch_predictor(const StepArgs& a, cudaStream_t s);
// Split of the history index of the FP64 slice of row n (chunks and their
// length), as every FP64 slice launch takes it; false when the workspace
// holds no split.
bool history_f64_split(int M, int n, size_t part_bytes, int band_hi, int* nchunk, int* chunk_len);

// Consecutive FP64 KBE steps of a small system in one cooperative launch
// (run_small.cu): the rows n[0..nsteps), each with its interval's order,
// field and history split; the rest as in kbe_step's launches.
constexpr int kRunMaxSteps = 64;
constexpr int kRunThreads = 256;
constexpr int kRunMaxRow = 4096;  // rows of at most this many entries ((n+1) M^2) run in the cooperative kernel
struct RunSmallHost {
  StepArgs base;                 // n, kn, field, corr, pred are set per row
  double* Sl;
  double* Sg;
  double* I;
  WeightsView w;
  double* part;
  const double* corr0;
  const double* pred0;
  unsigned* bar;                 // one counter of device memory
  long long spin;
  int withhold = -1;             // barrier at which block 0 leaves without arriving (failure-path test)
  int P, nsteps;
  int n[kRunMaxSteps], kn[kRunMaxSteps], chunk_len[kRunMaxSteps], nchunk[kRunMaxSteps];
  double field[kRunMaxSteps];
};
cudaError_t launch_run_small(const RunSmallHost& h, cudaStream_t s, int* launches);
// L(0,0) = i rho, R(0,0) = -i 1 from the device matrix rho (complex MxM).
cudaError_t launch_init_row0(int M, const double* rho, double* L, double* R, cudaStream_t s);
cudaError_t launch_fock(const StepArgs& a, cudaStream_t s);
cudaError_t launch_rhs(const StepArgs& a, cudaStream_t s);          // F row n only
cudaError_t launch_rhs_corrector(const StepArgs& a, cudaStream_t s);  // F row n, then new row n

// ---- adaptive history orders (adaptive.cu) -------------------------------
struct SelectArgs {
  int M, n, K;
  const double* L;     // triangles (row n = the current iterate)
  const double* R;
  const double* Sl;    // self-energy row n
  const double* Sg;
  const double* hist;  // local weights of interval n for orders 1..K: [kMaxOrder][kWTab]
  double* band;        // composite-weight band [n_t][band_w] (row n written)
  double* wbar;        // settled weights (entry n - band_w written)
  int band_w;
  int* korder;         // chosen order per interval (entry n written)
  double* u = nullptr; // scratch: test integrand [kMaxOrder+1][M][M] complex
};
cudaError_t launch_select_order(const SelectArgs& a, cudaStream_t s, int* launches);
// d_hist holds the local weights [n_max][kMaxOrder][kWTab], then the scratch u
inline size_t hist_doubles(int n_max, int M) {
  return (size_t)n_max * kMaxOrder * kWTab + 2 * (size_t)(kMaxOrder + 1) * M * M;
}

// ---- adaptive time stepping (controller.cu) -----------------------------
struct CtlArgs {
  int M, n, q, n_max;
  double* L;           // triangles; row n is written
  double* R;
  const double* F;     // right-hand-side ring [kRing][2][n_max][M][M]
  double wp[kWTab];    // predictor weights (nodes t_{n-q..n-1}); divided differences: coefficients over t_{n..n-q1}
  double wc[kWTab];    // corrector weights (nodes t_{n-q+1..n}); divided differences: over t_{n..n-q2}
  int q1, q2;          // orders of the two divided differences (-1: none)
  double rtol, atol;
  double* ypred;       // [2][n+1][M][M] predicted row
  double* ycur;        // [2][n+1][M][M] current iterate
  double* partial;     // [blocks][2] per-block sums
  int* status;
};
struct ReconArgs {
  int M, n, jlo, n_max;
  const double* L;
  const double* R;
  const double* Sring;     // self-energy rows [kRing][2][n_max][M][M] of accepted rows
  const double* eps_ring;  // Fock matrices [kRing][M][M] of accepted rows
  WeightsView w;
  double* F;               // right-hand-side ring; row j gets column n
  int* status;
};
int ctl_partial_count(int n_max, int M);
cudaError_t launch_ctl_predict(const CtlArgs& a, cudaStream_t s);
cudaError_t launch_ctl_correct(const CtlArgs& a, double* out, cudaStream_t s);
cudaError_t launch_ctl_divdiff(const CtlArgs& a, double* out, cudaStream_t s);
cudaError_t launch_ctl_reconstruct(const ReconArgs& r, cudaStream_t s);

// ---- thermal branch (thermal.cu) ----------------------------------------
struct ThermalArgs {
  int M, N, n, kn;
  const double* U;       // local interaction
  const double* Sl;      // self-energy row n
  const double* Sg;
  WeightsView w;
  const double* eps;     // eps(t_n)
  const double* GM;      // [N][M][M]
  const double* left;    // tau weights [N][N]
  double* Gx;            // mixed rows [n_max][N][M][M]
  double* Smix;          // Sigma^| row n [N][M][M]
  double* Smw;           // w_k Sigma^|(n, k) with the full-interval tau weights [N][M][M]
  double* Aw;            // w_{n,m} Sigma^R(n, m), m <= n [n_max][M][M]
  float4* Smwf;          // Smw and Aw as double-float (re.hi, re.lo, im.hi, im.lo)
  float4* Awf;
  int df;                // 1: the two long sums in double-float on the FP32 pipe
  double* Fx;            // mixed right-hand sides, ring [kRing][N][M][M]
  double* I;             // history slice [2][n+1][M][M]
  const double* corr;    // stepper weights of interval n
  const double* pred;
  int* status;
};
cudaError_t launch_th_sigma(const ThermalArgs& a, cudaStream_t s);  // also Smw and Aw
cudaError_t launch_th_mixed(const ThermalArgs& a, cudaStream_t s);
cudaError_t launch_th_rhs(const ThermalArgs& a, cudaStream_t s);
cudaError_t launch_th_adams(const ThermalArgs& a, bool corrector, cudaStream_t s);

// ---- reverse mode (adjoint.cu) ------------------------------------------
// Cotangent convention: for a real loss, zbar = dF/dRe z + i dF/dIm z.
struct AdjHistArgs {
  int M, n, row_lo;
  const double* L;      // triangles; row n holds the iterate the slice was taken at
  const double* R;
  const double* Sl;     // Sigma row n, [n+1][M][M]
  const double* Sg;
  const double* Ib;     // cotangent of the slice, [2][n+1][M][M]
  WeightsView w;
  double* dSl;          // cotangent of the Sigma row (overwritten)
  double* dSg;
  double* dL;           // rows row_lo..n-1 (incremented); block p at p - tri(row_lo, 0)
  double* dR;
  double* gL;           // row n (incremented), [n+1][M][M]
  double* gR;
  double* work;
  size_t work_bytes;
  int df = 0;           // 1: the Sigma-row cotangent sums in double-float (KBE_DF64 steps)
};
cudaError_t launch_adjoint_history(const AdjHistArgs& a, cudaStream_t s, int* launches);

struct AdjSigmaArgs {
  int M, n;
  const double* Lrow;   // row n of the triangles, [n+1][M][M]
  const double* Rrow;
  const double* U;
  const double* dSl;
  const double* dSg;
  double* gL;           // incremented
  double* gR;
  double* dUp;          // scratch, 2 (n+1) M^2 doubles
  double* dU;           // incremented
};
cudaError_t launch_adjoint_sigma(const AdjSigmaArgs& a, cudaStream_t s, int* launches);

struct AdjRhsArgs {
  int M, n;
  const double* eps;    // Fock matrix of the iterate
  const double* Fb;     // cotangent of F row n: entry (s, c, a, b) at Fb + s * fs + (c M^2 + a M + b) * 2
  int64_t fs;
  const double* Lrow;
  const double* Rrow;
  const double* U;
  const double* v;
  double shape;         // dE(t_n)/dE0
  double* Ib;           // cotangent of the slice (overwritten), [2][n+1][M][M]
  double* gL;           // incremented
  double* gR;
  double* epsb;         // scratch, M^2 complex
  double* dU;
  double* dE0;
};
cudaError_t launch_adjoint_rhs(const AdjRhsArgs& a, cudaStream_t s, int* launches);

struct AdjLinArgs {
  int M, n, kn, corrector;
  const double* wtab;   // predictor or corrector weights of interval n, [kMaxOrder][kWTab]
  const double* gL;     // cotangent of the new row n, [n+1][M][M]
  const double* gR;
  double* dL;           // triangles of cotangents, block p at p - tri_base
  double* dR;
  int64_t tri_base;
  int write_prev;       // 0: row n-1 is frozen, its cotangent is not formed
  double* Fb_rows;      // cotangents of F rows j < n: row j at (j - j0) * fstride, s at + s * fs
  int j0;
  int64_t fstride, fs;
  double* Fb_cur;       // cotangent of F row n (corrector), same row layout
};
cudaError_t launch_adjoint_lin(const AdjLinArgs& a, cudaStream_t s, int* launches);

}  // namespace kbe
