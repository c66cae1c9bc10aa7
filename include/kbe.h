/*
 * kbe.h -- C ABI of the GB300 (sm_103a) hot path of the adaptive
 * Kadanoff-Baym solver of Blommel, Gardner, Woodward and Gull,
 * "Adaptive Time Stepping for the Two-Time Integro-Differential
 * Kadanoff-Baym Equations" (arXiv 2405.08737).
 *
 * At each new time t_n of a nonuniform grid the library computes
 *   - the second-Born self-energy row Sigma^{<,>}(t_n, t_c), c <= n
 *     (Sec. 2, Eq. SE, for a local interaction U_abcd = U_a delta_abcd),
 *   - the history (collision) integrals of Eq. (KBE2),
 *       I^s(n,c) = sum_{m<=n} w_{n,m} Sigma^R(n,m) G^s(m,c)
 *                + sum_{m<=c} w_{c,m} Sigma^s(n,m) G^A(m,c),   s in {<,>},
 *     with the variable-order interpolatory weights w of Sec. 3.2
 *     (Eq. weights and the composite-row recursion),
 *   - one KBE step of row n (predictor, then P fixed-point sweeps of
 *     self-energy, history integrals, right-hand side and corrector;
 *     Sec. 3.1 solves each step by fixed-point iteration).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Complex numbers are interleaved (re, im) doubles (complex128).
 *  - Two-time arrays are triangle-packed: the lower triangle r >= c of the
 *    (t, t') plane, block p(r,c) = r(r+1)/2 + c, each block an MxM
 *    row-major matrix (M = norb).  The upper triangle follows from the
 *    anti-Hermitian symmetry G(t,t') = -G(t',t)^+ (Sec. 2).  Row n is the
 *    contiguous run of blocks p(n,0) .. p(n,n).
 *      L(r,c) = G^<(t_r, t_c),  R(r,c) = G^R(t_r, t_c),
 *    and R(r,r) must hold -i*1 (Eq. BC with theta(0) = 1), so that
 *    G^> = R + L on and below the diagonal.
 *  - Self-energy rows are [n+1][M][M] (c = 0..n); history slices are
 *    [2][n+1][M][M] with s = 0 for "<" and s = 1 for ">".
 *  - Device pointers are borrowed, never freed, and must be 16-byte
 *    aligned.  Host pointers are read during the call only.
 *  - "stream" is a cudaStream_t (NULL = legacy default stream).  Calls
 *    that launch kernels are asynchronous; a non-KBE_OK return means that
 *    nothing (or not everything) was enqueued.
 *  - Calls never exit, abort or trap the GPU.  Kernel-side problems
 *    (non-finite values, a device wait that ran out) set a device status
 *    word that kbe_sync_status() returns.
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef KBE_H
#define KBE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kbe_ctx kbe_ctx;
typedef int kbe_status;

#define KBE_OK 0
#define KBE_EINVAL 1   /* null or misaligned pointer, bad size or index     */
#define KBE_ERANGE 2   /* order outside [1, KBE_MAX_ORDER], n beyond grid   */
#define KBE_ENOMEM 3   /* device allocation failed                          */
#define KBE_ECUDA 4    /* a CUDA runtime call or launch failed              */
#define KBE_ENUMERIC 5 /* a kernel saw a non-finite value                   */
#define KBE_ETIMEOUT 6 /* a bounded device wait ran out                     */
#define KBE_ESTATE 7   /* call made out of order (no grid, no model, ...)   */

#define KBE_MAX_ORDER 12   /* largest per-interval quadrature order k      */
#define KBE_RING_ROWS 13   /* right-hand-side rows kept by the stepper     */
#define KBE_DENSE_MAX_NORB 32  /* largest norb for a dense interaction      */

/* precision argument of kbe_history_slice / kbe_step */
#define KBE_FP64 0        /* plain FP64 arithmetic, deterministic            */
#define KBE_SPLIT_BF16 1  /* the contraction on the 16-bit-float tensor cores */
                          /* with error-free 4-digit fixed-point splitting:   */
                          /* every value becomes round(v 2^(31-e)) in base-256 */
                          /* digits (e: exponent of its column over 16 (the   */
                          /* planes path) or 8 (the fused path) history       */
                          /* entries), each digit exact in fp16 (bf16 would   */
                          /* hold them too; fp16 takes three instructions per */
                          /* digit pair to form), the 13 digit products of    */
                          /* levels 0..4 summed exactly in FP32 and combined  */
                          /* in double-float; about 1e-9 relative to the      */
                          /* slice maximum.  norb <= 32.  Deterministic.      */
                          /* Requires R(r,r) = -i*1 exactly.                  */
#define KBE_DF64 2        /* the contraction in double-float arithmetic on    */
                          /* the FP32 pipe (hi + lo floats, about 2^-47 per   */
                          /* product, compensated sums): about 1e-14 of the   */
                          /* terms' sizes, several times the FP64 pipe's      */
                          /* rate on this part.  Deterministic.               */

/* ---------------------------------------------------------- lifecycle -- */

/* Create a context for norb orbitals and at most n_max time points.
 * Allocates device workspace only (split-reduction partials, weight tables,
 * status word); the two-time arrays belong to the caller.
 * KBE_EINVAL: out == NULL, norb < 1, norb > 64, n_max < 1, or sizes that
 * overflow 64-bit block indices.  KBE_ENOMEM / KBE_ECUDA on device errors. */
kbe_status kbe_create(int norb, int n_max, kbe_ctx** out);

/* Free the context and its workspace (NULL is accepted). */
kbe_status kbe_destroy(kbe_ctx* ctx);

/* Text of the last error on this context (static storage of the context;
 * "" when none).  A NULL ctx gives the last context-free error (kbe_create,
 * kbe_history_slice_noalloc, kbe_batch_create) of the calling host thread;
 * each thread keeps its own. */
const char* kbe_last_error(const kbe_ctx* ctx);

/* ------------------------------------------------------------- grid ---- */

/* Set the time grid t[0..n_t-1] and the per-interval orders order[1..n_t-1]
 * (order[0] is ignored).  Host arrays, copied.  Requires t[0] = 0, t
 * strictly increasing and finite (else KBE_EINVAL), 1 <= order[l] <=
 * KBE_MAX_ORDER (else KBE_ERANGE), 1 <= n_t <= n_max (else KBE_EINVAL).
 * Interval l uses order kappa_l = min(order[l], l) (backward stencils).
 * The local weights of Sec. 3.2, Eq. (weights), are computed here in host
 * FP64 by a fully pivoted LU solve of the Vandermonde system, the composite
 * rows w_{c,m} are assembled by the recursion of Sec. 3.2 and stored as a
 * settled vector plus a band, and the stepper's predictor/corrector weights
 * are tabulated; all of it is uploaded synchronously. */
kbe_status kbe_set_grid(kbe_ctx* ctx, const double* t, const int* order, int n_t);

/* Host FP64 composite weight row w_{n,0..n} of a grid (Sec. 3.2), by the
 * same LU solves and recursion kbe_set_grid uses.  No context, no GPU.
 * Same validation as kbe_set_grid; n must lie in [0, n_t-1]. */
kbe_status kbe_grid_weights(const double* t, const int* order, int n_t, int n, double* row);

/* Host FP64 weights w[0..k] of the rule that integrates over [lo, hi] the
 * degree-k interpolant through the nodes tau[0..k] (Eq. weights), by a
 * fully pivoted LU solve of V^T w = T.  No context, no GPU.
 * KBE_EINVAL for k < 0, k > KBE_MAX_ORDER, repeated nodes or NULL. */
kbe_status kbe_local_weights(const double* tau, int k, double lo, double hi, double* w);

/* ------------------------------------------------------------ model ---- */

/* Model of the stepper: h(t) = h0 + E(t) diag(v) with
 * E(t) = E0 exp(-(t-t0)^2 / (2 sigma^2)) cos(omega t), pulse = {E0, t0,
 * sigma, omega}; local interaction U[0..M-1].  The Fock matrix of Eq. (eps)
 * for this interaction is eps(t) = h(t) + diag(U_a n_a(t)) with
 * n_a = Im G^<_aa(t,t).  h0 is a host complex MxM matrix; U, v host
 * doubles.  KBE_EINVAL for NULL pointers, non-finite values or sigma <= 0. */
kbe_status kbe_set_model(kbe_ctx* ctx, const double* h0, const double* U, const double* v,
                         const double* pulse);

/* Thermal branch (Sec. 2, Eq. KBE3 and the tau terms of Eq. KBE1/KBE2): the
 * mixed component G^|(t, tau) joins the state, on the uniform grid
 * tau_k = k beta / (n_tau - 1) (the paper represents tau functions in the
 * DLR basis, which this library does not have).  GM: host, complex
 * [n_tau][M][M], the Matsubara function G^M(tau_k) supplied as the initial
 * condition (tau_0 = 0+, tau_{n_tau-1} = beta-); the call sets
 * G^|(0, tau) = -i G^M(beta - tau), and the caller sets L(0,0) = i rho
 * consistently (rho = -G^M(beta-)).  Conventions: G^|-(tau, t) =
 * [G^|(t, beta - tau)]^+, G^M antiperiodic.  Every kbe_step (and
 * kbe_rhs_row) then, in FP64 for the local interaction:
 *   Sigma^|_ab(t_n, tau) = U_a U_b G^|_ab(t_n, tau)^2 G^|-_ba(tau, t_n),
 *   adds -i int_0^beta Sigma^|(t_n, tau) G^|-(tau, t_c) dtau to I^<(n,c), I^>(n,c),
 *   F^|(n, tau) = -i [eps G^| + int_0^{t_n} Sigma^R G^|(., tau) + int_0^beta
 *                Sigma^|(t_n, s) G^M(s - tau) ds]        (Eq. KBE3),
 * and steps the mixed row with the weights of the diagonal.  tau integrals
 * over [0, tau_j] take, per interval, the interpolatory rule of order k_tau
 * (Eq. weights) through nodes centred on the interval inside the range;
 * [tau_j, beta] the mirrored rule (odd k_tau gives mirror-symmetric weights,
 * which keep the particle number exactly).  The context holds
 * (2 + 2 KBE_RING_ROWS + 2 n_max) n_tau M^2 complex entries plus n_tau^2
 * weights.  GM = NULL turns the branch off.  KBE_EINVAL for a dense
 * interaction, beta <= 0, n_tau outside [2, 4096], k_tau outside [1, 12],
 * non-finite G^M.  Batches, the reverse mode, kbe_step_rows and
 * kbe_run_controlled do not take a thermal branch (KBE_EINVAL / KBE_ESTATE). */
kbe_status kbe_set_thermal(kbe_ctx* ctx, double beta, int n_tau, int k_tau, const double* GM);

/* Copies rows 0..n_rows-1 of the mixed component [n_rows][n_tau][M][M]
 * (device buffer buf) out of the context (to_context = 0) or into it
 * (to_context = 1, e.g. to restart from a stored history), on stream. */
kbe_status kbe_copy_mixed(kbe_ctx* ctx, int n_rows, void* buf, int to_context, void* stream);

/* General four-index interaction (Sec. 2, Eq. SE and Eq. eps) in place of
 * the model's local U.  U4: host, M^4 real doubles, row-major
 * U4[((i*M + f)*M + d)*M + e] = U_ifde (chemists' order for Coulomb
 * integrals; no symmetry is assumed or used).  The self-energy becomes
 *   Sigma^<>_ij(t,t') = U_ifde UEx_jabc G^<>_fb(t,t') G^<>_ea(t,t') G^><_cd(t',t),
 *   UEx_jabc = 2 U_jbac - U_jabc,
 * evaluated in FP64 with 12 M^5 multiply-adds per block and component, and
 * the Fock matrix eps_ij = h_ij(t) + i (U_iabj - 2 U_ijba) G^<_ba(t,t).  The
 * tensor is copied (3 M^4 doubles on the device, synchronously); the
 * model's pulse and v stay in force and its U is unused.  U4 = NULL returns
 * to the local U.  KBE_ERANGE for M > KBE_DENSE_MAX_NORB, KBE_EINVAL for
 * non-finite entries.  With a dense interaction the reverse-mode calls that
 * differentiate the self-energy or the Fock matrix (kbe_adjoint_selfenergy_
 * slice, kbe_step_adjoint) and batches return KBE_ESTATE / KBE_EINVAL;
 * kbe_adjoint_slice (the history contraction alone) is unaffected. */
kbe_status kbe_set_interaction(kbe_ctx* ctx, const double* U4);

/* ------------------------------------------------------- hot path ------ */

/* Self-energy row n (Sec. 2, Eq. SE with the local interaction of the
 * model, or the tensor of kbe_set_interaction): for c = 0..n and every (a,b)
 *   S^>(n,c)_ab = -U_a U_b [G^>(n,c)_ab]^2 conj(G^<(n,c)_ab),
 *   S^<(n,c)_ab = -U_a U_b [G^<(n,c)_ab]^2 conj(G^>(n,c)_ab),
 * with G^< = L and G^> = R + L from row n.  (G^<>(t_c,t_n)_ba =
 * -conj(G^<>(t_n,t_c)_ab) turns Eq. SE's third factor into the conjugate.)
 * On the diagonal block c = n the third factor is the stored entry
 * G^><(t_n,t_n)_ba itself, as Eq. SE reads.
 * L, R: device triangles holding row n.  S_less, S_great: device rows
 * [n+1][M][M], written.  Requires a grid (n < n_t) and a model. */
kbe_status kbe_selfenergy_slice(kbe_ctx* ctx, int n, const void* L, const void* R, void* S_less,
                                void* S_great, void* stream);

/* Self-energy of every stored block of a triangle of n_rows rows (the
 * row formula above applied to each block), S triangles written.  Used for
 * whole-history evaluation.  Requires a model. */
kbe_status kbe_selfenergy_all(kbe_ctx* ctx, int n_rows, const void* L, const void* R, void* S_less,
                              void* S_great, void* stream);

/* History slice of row n, Eq. (KBE2) (formula at the top of this file):
 * I_out [2][n+1][M][M] device, written.  L, R: device triangles holding
 * rows 0..n; S_less, S_great: device self-energy row n.  precision:
 * KBE_FP64, KBE_SPLIT_BF16 or KBE_DF64.  Deterministic (fixed split and
 * reduction order).
 * Requires a grid with n < n_t.  Uses the context's workspace: calls on
 * one context must not overlap on different streams. */
kbe_status kbe_history_slice(kbe_ctx* ctx, int n, int precision, const void* L, const void* R,
                             const void* S_less, const void* S_great, void* I_out, void* stream);

/* One device's share of a history slice split across devices (the slice
 * of Eq. KBE2 by bands of stored rows): the contributions of the stored
 * blocks (r, c), row_lo <= r < row_hi, r <= n, of L and R to I(n, c) for
 * every c = 0..n -- term 1 of column c through G(r, c) (history point
 * m = r), term 1 of column r through G(c, r) = -G(r, c)^+ (m = c < r) and
 * term 2 of column r through G^A(c, r) = R(r, c)^+ (m = c).  I_out
 * [2][n+1][M][M] device, written with the band's partial sums; the sum of
 * the partials of bands that partition the rows 0..n is the slice of
 * kbe_history_slice (KBE_FP64) to rounding.  A device needs only its own
 * rows of L and R, row n (for its Sigma row) and the Sigma row itself.
 * KBE_EINVAL for row_lo < 0, row_hi < row_lo or a bad pointer; otherwise
 * as kbe_history_slice. */
kbe_status kbe_history_slice_band(kbe_ctx* ctx, int n, int row_lo, int row_hi, const void* L, const void* R,
                                  const void* S_less, const void* S_great, void* I_out, void* stream);

/* ----------------------------------------------------------- stepper --- */

/* Row 0 of a run that starts from an uncorrelated state (Sec. 2: the
 * initial density matrix enters as G^<(0,0) = i rho, and Eq. BC with
 * theta(0) = 1 fixes G^R(0,0) = -i 1): writes block p(0,0) of L (= i rho0)
 * and of R (= -i 1) on `stream`.  rho0: host complex MxM matrix (the
 * one-body density matrix per spin), read during the call.  L, R: device
 * triangles.  KBE_EINVAL for NULL or misaligned pointers or non-finite
 * entries.  Follow it with kbe_rhs_row(ctx, 0, ...) for the ring. */
kbe_status kbe_init_uncorrelated(kbe_ctx* ctx, const double* rho0, void* L, void* R, void* stream);

/* Right-hand-side row j of Eq. (KBE2), the t-derivative along row j:
 *   F^s(j,c) = -i ( eps(t_j) G^s(j,c) + I^s(j,c) ),  c = 0..j,
 * computed from rows 0..j of L, R (self-energy and history slice of row j
 * included) into slot j % KBE_RING_ROWS of F_ring.  F_ring: device
 * [KBE_RING_ROWS][2][n_max][M][M]; row j of a slot uses its first j+1
 * blocks per s.  S_less/S_great: device rows [n_max][M][M] (scratch);
 * I_work: device [2][n_max][M][M] (receives the history slice).  Used to
 * start a run (j = 0) or to rebuild stored right-hand sides at a restart. */
kbe_status kbe_rhs_row(kbe_ctx* ctx, int j, int precision, const void* L, const void* R, void* S_less,
                       void* S_great, void* I_work, void* F_ring, void* stream);

/* One KBE step of row n >= 1 (rows 0..n-1 of L, R and the right-hand-side
 * rows n-K..n-1 of F_ring present, K = largest order on the grid):
 *   predictor  G^s(n,c) = G^s(n-1,c) + sum_p wp_p F^s(n-q+p, c) over the q =
 *              min(k_n, n-c) points t_{n-q..n-1} (extrapolation rule);
 *              diagonal from D(j) = F^<(j,j) - F^<(j,j)^+, q = min(k_n, n);
 *   P times    self-energy row n, history row n, F row n, then the corrector
 *              G^s(n,c) = G^s(n-1,c) + sum_p w_p F^s(n-kap+p, c) over the
 *              kap+1 points t_{n-kap..n}, kap = min(k_n, n-c) (diagonal:
 *              min(k_n, n)), and R(n,c) = G^>(n,c) - L(n,c), R(n,n) = -i*1.
 * Row n of L, R and slot n of F_ring are written; S_less, S_great, I_work
 * hold row n's last self-energy and history slice.  1 <= P <= 16.
 * With KBE_SPLIT_BF16 the context keeps the tensor-core digit planes of the
 * history between steps on the same L and R: rows below the row of the
 * previous step are not encoded again.  A caller that rewrites those rows
 * between steps (a restart into the same buffers) calls kbe_reset_cache. */
kbe_status kbe_step(kbe_ctx* ctx, int n, int P, int precision, void* L, void* R, void* S_less,
                    void* S_great, void* I_work, void* F_ring, void* stream);

/* The KBE steps of rows n_first..n_last in order (1 <= n_first <= n_last <
 * n_max), each exactly kbe_step's (the same kernels, rows and ring slots;
 * rows 0..n_first-1 and the right-hand-side rows before n_first present as
 * kbe_step requires for row n_first): a whole run on the given grid (Sec. 3.1
 * with the grid's steps and orders) in one call, all on `stream` with no
 * host synchronisation and no call per step.  With KBE_FP64, the local
 * interaction, fixed history orders, no thermal branch and profiling off,
 * rows of at most 4096 complex entries per component ((n+1) M^2 <= 4096)
 * run up to 64 at a time in one cooperative launch (one block per SM, a
 * device-wide barrier with a bounded wait between the phases of a step; a
 * wait that runs out is reported as KBE_ETIMEOUT by kbe_sync_status); the
 * rows, slices and ring are bitwise kbe_step's.  Where the device refuses
 * the cooperative launch (fewer SMs available to the process than the
 * device has), those rows and all later ones on the context take
 * kbe_step's kernels instead, with the same results.  Errors as kbe_step; on a
 * launch error the rows before the failing launch are stepped. */
kbe_status kbe_run_steps(kbe_ctx* ctx, int n_first, int n_last, int P, int precision, void* L, void* R,
                         void* S_less, void* S_great, void* I_work, void* F_ring, void* stream);

/* The phases of one KBE_FP64 step, for callers that form the history slice
 * themselves -- one system split by row bands of the stored triangles across
 * devices (Eq. KBE2 is a sum over stored blocks, so the bands' partial slices
 * add up to the slice; the sum is the caller's, e.g. an all-reduce):
 *   kbe_step_predict       the predictor of row n (as kbe_step);
 *   kbe_step_sweep_band    self-energy row n into S_less, S_great, then the
 *                          partial slice of the stored rows [row_lo, row_hi)
 *                          into I_part ([2][n+1][M][M], kbe_history_slice_band);
 *   kbe_step_sweep_finish  from the whole slice I of row n: the Fock matrix,
 *                          the right-hand side row n (slot n of F_ring) and the
 *                          corrector, which writes row n of L and R.
 * kbe_step(ctx, n, P, KBE_FP64, ...) equals kbe_step_predict, then P times
 * {kbe_step_sweep_band over rows [0, n+1), kbe_step_sweep_finish}, bitwise.
 * A device that holds only its band of history rows needs, besides them,
 * rows n-1 and n (every device computes row n from the same reduced slice)
 * and the right-hand-side ring.  Layouts and errors as kbe_step; adaptive
 * history orders and the thermal branch are KBE_ESTATE (they need kbe_step). */
kbe_status kbe_step_predict(kbe_ctx* ctx, int n, void* L, void* R, void* F_ring, void* stream);
kbe_status kbe_step_sweep_band(kbe_ctx* ctx, int n, int row_lo, int row_hi, const void* L, const void* R,
                               void* S_less, void* S_great, void* I_part, void* stream);
kbe_status kbe_step_sweep_finish(kbe_ctx* ctx, int n, void* L, void* R, const void* I, void* F_ring, void* stream);

/* kbe_step with its inputs in host memory, for callers that keep the run on
 * the host: rows 0..n-1 of both triangles (L_host, R_host: the same packed
 * layout as L, R, at least tri(n) blocks) and the right-hand-side ring
 * (F_host: the image of F_ring) are copied into the device buffers L, R,
 * F_ring, and the new row n of L and R is copied back to L_row_host and
 * R_row_host ((n+1) M^2 complex each).  The rows are copied from row n-1
 * down in up to 5 chunks whose sizes grow geometrically (ratio 1.8, the
 * first the smallest) on a copy stream of the context; with KBE_FP64 (and no adaptive orders or thermal branch) the
 * first sweep's history slice contracts the output columns of each chunk as
 * soon as it has arrived (column c reads rows c..n only), so the copies
 * overlap the contraction; the results are bitwise those of kbe_step on the
 * same data.  Otherwise the step starts once all rows are in.  Host buffers
 * should be page-locked (cudaHostAlloc or registered) for the copies to be
 * asynchronous; none of them may be changed or freed before the stream has
 * passed the step.  The copies start after the work already queued on
 * `stream` and never touch row n or above.  Digit planes cached by
 * KBE_SPLIT_BF16 steps are dropped (the rows are rewritten).  Errors as
 * kbe_step, plus KBE_EINVAL for a NULL host pointer. */
kbe_status kbe_step_host(kbe_ctx* ctx, int n, int P, int precision, const void* L_host, const void* R_host,
                         const void* F_host, void* L, void* R, void* S_less, void* S_great, void* I_work,
                         void* F_ring, void* L_row_host, void* R_row_host, void* stream);

/* kbe_step with the right-hand-side rows in a row store instead of the
 * ring: row j lives in slot j - j0 of F_rows, device
 * [n_rows][2][n_max][M][M].  Step n reads rows n-k_n .. n-1 and writes row
 * n, so n - k_n >= j0 and n - j0 < n_rows (else KBE_ERANGE).  Keeping every
 * row of a window of steps is what the reverse sweep (kbe_step_adjoint)
 * recomputes from. */
kbe_status kbe_step_rows(kbe_ctx* ctx, int n, int P, int precision, void* L, void* R, void* S_less,
                         void* S_great, void* I_work, void* F_rows, int j0, int n_rows, void* stream);

/* --------------------------------------------------------- reverse mode -- */
/* The paper computes no gradients; these calls give vector-Jacobian
 * products of the calls above, for derivatives of observables with respect
 * to the interaction U and the pulse amplitude E0 (E(t) = E0 g(t)).
 * Cotangents use the convention of PyTorch for a real loss F of complex z:
 * zbar = dF/d(Re z) + i dF/d(Im z).  All in FP64.  Cotangent triangles
 * dL, dR cover rows row_lo.. only: block p(r,c) of rows r >= row_lo sits at
 * p(r,c) - p(row_lo,0).  Rows below row_lo are treated as constants. */

/* Vector-Jacobian product of the history slice of row n (Eq. KBE2), which
 * is bilinear in the self-energy row and the rows 0..n of G.  dI: device
 * [2][n+1][M][M], the cotangent of the slice.  dS_less, dS_great: device
 * [n+1][M][M], OVERWRITTEN with the cotangent of the self-energy row:
 *   dA1(m)  = sum_{s,c} dI^s(c) G^s(m,c)^+,  A1(m) = w_{n,m} (S^>(m) - S^<(m)),
 *   dS^>(m) = w_{n,m} dA1(m) + sum_{c>=m} w_{c,m} dI^>(c) R(c,m),
 *   dS^<(m) = -w_{n,m} dA1(m) + sum_{c>=m} w_{c,m} dI^<(c) R(c,m).
 * dL, dR: cotangent triangles of rows row_lo..n (0 <= row_lo <= n),
 * INCREMENTED by the slice's dependence on those rows (R(r,r) is fixed at
 * -i*1 and gets none).  Deterministic.  Uses the context's workspace. */
kbe_status kbe_adjoint_slice(kbe_ctx* ctx, int n, const void* L, const void* R, const void* S_less,
                             const void* S_great, const void* dI, void* dS_less, void* dS_great, void* dL,
                             void* dR, int row_lo, void* stream);

/* Vector-Jacobian product of the self-energy row n (Eq. SE, with the
 * diagonal block's third factor read from the stored block as in
 * kbe_selfenergy_slice).  dS_less, dS_great: device [n+1][M][M]
 * cotangents of the row.  dL_row, dR_row: device [n+1][M][M], INCREMENTED
 * by the cotangent of row n of L and R (R(n,n) gets none).  dU: device
 * double[M], INCREMENTED by dF/dU.  Uses the context's workspace. */
kbe_status kbe_adjoint_selfenergy_slice(kbe_ctx* ctx, int n, const void* L, const void* R, const void* dS_less,
                                        const void* dS_great, void* dL_row, void* dR_row, double* dU,
                                        void* stream);

/* Reverse sweep of one KBE step n taken by kbe_step_rows with the same
 * precision (KBE_FP64 or KBE_DF64; KBE_EINVAL otherwise), the same P and
 * the same store F_rows, j0, n_rows.  On entry L, R hold rows
 * 0..n and F_rows rows j0..n as the forward run left them (later steps do
 * not touch them); the call recomputes step n from rows 0..n-1, keeping
 * its P iterates on the device, then runs the adjoints of the corrector,
 * right-hand side (Fock matrix with its Hartree term U_a Im L(n,n)_aa and
 * the field E0 g(t_n) v_a), history slice and self-energy of each sweep in
 * reverse, and finally of the predictor.
 *   dL, dR: cotangent triangles of rows row_lo..n (1 <= n, row_lo <= n).
 *           Row n holds the cotangent of the step's result on entry and is
 *           read only; rows row_lo..n-1 are INCREMENTED.
 *   dF_rows: cotangents of the stored right-hand-side rows, layout of
 *           F_rows.  Slot n holds the cotangent of row n (from later steps)
 *           on entry; slots of rows n-k_n..n-1 are INCREMENTED.
 *   dU (device double[M]) and dE0 (device double[1]) are INCREMENTED.
 * On return L, R and F_rows hold what they held on entry.  Sweeping n =
 * n_end-1 down to n_start with the same dL, dR, dF_rows gives the gradient
 * of any function of the rows through the window [n_start, n_end).  The
 * first call allocates a reverse-mode workspace of (13 + 2 (P+1)) n_max M^2
 * complex entries held by the context (KBE_ENOMEM if that fails). */
kbe_status kbe_step_adjoint(kbe_ctx* ctx, int n, int P, int precision, void* L, void* R, void* F_rows, int j0,
                            int n_rows, void* dL, void* dR, int row_lo, void* dF_rows, double* dU, double* dE0,
                            void* stream);

/* Adaptive history orders (Sec. 3.2).  With K in 1..12, every fixed-point
 * sweep of kbe_step / kbe_step_rows chooses the order of the history
 * quadrature over [t_{n-1}, t_n] on the device: it integrates the test
 * function u(t) = G^R(t_n,t) Sigma^<(t,t_n) + G^<(t_n,t) Sigma^A(t,t_n) over
 * the interval with every order k <= min(K, n) (interpolatory rules of
 * Eq. weights through t_{n-k..n}) and takes the order that minimises the
 * max-norm change from order k-1; differences within 64 eps of the largest
 * test integral from the minimum are not distinguished (the lowest order is
 * taken).  The composite weights of row n follow from row n-1 and the local
 * weights of that order (the row recursion of Sec. 3.2).  The grid's own
 * orders keep driving the stepper's predictor and corrector.  The band of
 * the weights widens to K+1 points.  Steps must run in order from row 1
 * (kbe_step at row n requires rows 1..n-1 stepped; stepping a row again
 * restarts from it), else KBE_ESTATE.  K = 0 returns to the grid's orders.
 * Calls kbe_set_grid first; kbe_set_grid returns to the grid's orders.
 * Batches (kbe_batch_*) need the grids' orders. */
kbe_status kbe_set_adaptive_orders(kbe_ctx* ctx, int K);

/* The history order of each interval 0..n-1 (0 for row 0): the chosen ones
 * in adaptive mode (synchronises the device), else min(order[l], l). */
kbe_status kbe_get_history_orders(kbe_ctx* ctx, int* orders, int n);

/* Adaptive time stepping (Sec. 3.1): from row 0 (L(0,0) = i rho(0),
 * R(0,0) = -i, set by the caller) to t_end, the run chooses its own grid.
 * Step n takes variable-step Adams formulas of order q (1..q_max) in
 * integral form on the accepted points: the predictor integrates the
 * interpolant of the derivative data at t_{n-1..n-q}, the corrector the one
 * at t_{n..n-q+1} (Eq. predictor, Eq. corrector).  The corrector is iterated
 * with the right-hand side of Eq. (KBE2) evaluated on the device (self-
 * energy, history slice in the given precision, Fock matrix) until
 * R ||dy||_wrms < 0.1 / |C| (Eq. wrms_norm with the weights of Eq. ewt,
 * complex modulus; at most 3 iterations; R the estimated contraction rate).
 * The local error C (y_n - y_n(0)), with C = E_c / (E_p - E_c) from the
 * error integrals of the two formulas, must have WRMS norm <= 1, else the
 * step is retried smaller.  After q+1 steps at order q the orders q-1 and
 * q+1 are weighed by error estimates from divided differences of the
 * derivative data.  Step factors 1 / ((b E)^(1/(q+1)) + 1e-6) (b = 6, 6, 10
 * for q-1, q, q+1) pick the next step and order, with CVODE's safeguards:
 * no change below a factor 1.5, growth at most 1e4 on the first step, 10
 * later and none right after a failure; a failed error test shrinks the
 * step by 0.1..0.9 and the third one of a step falls back to order 1 with a
 * factor 0.1; a failed iteration shrinks it by 0.25.  When a step is
 * accepted, the derivative data of the new column at the last q+1 earlier
 * times are evaluated above the diagonal (the history reconstruction of
 * Sec. 3.1): Eq. (KBE2) at (t_j, t_n), j < n.  History quadrature: order
 * k_hist on every interval, or chosen per interval up to K_sel (Sec. 3.2,
 * as with kbe_set_adaptive_orders) when K_sel > 0.
 *   opts (host double[5]) = {rtol >= 0, atol > 0, h0 > 0 (first step),
 *                           h_max >= 0 (0: unbounded), t_end > 0};
 *   iopts (host int[4]) = {q_max 1..12, k_hist 1..12, K_sel 0..12, precision};
 *   L, R: device triangles of n_max rows; S_less, S_great: device rows
 *   [n_max][M][M]; I_work [2][n_max][M][M]; F_ring
 *   [KBE_RING_ROWS][2][n_max][M][M] (the layouts of kbe_step);
 *   t_out (double), q_out, korder_out (int): host arrays of n_max entries:
 *   the accepted times, the order of each step and the history order of
 *   each interval (0 past the last row); n_rows: accepted rows including
 *   row 0; stats (host int[5]) = {steps, error-test failures, convergence
 *   failures, right-hand-side evaluations, reconstructed blocks}.
 * Needs a model (and uses the dense interaction when one is set).  The first
 * call allocates a workspace of (2 KBE_RING_ROWS + 4) n_max M^2 complex
 * entries held by the context.  The host reads two numbers per fixed-point
 * iteration (the stream is synchronised each time).  Invalid options are
 * KBE_EINVAL (ranges above; also an unknown precision).  Returns KBE_OK at
 * t_end, KBE_ERANGE when n_max rows fill first, KBE_ENUMERIC when a step
 * fails 7 error tests or 10 iterations; the outputs describe the rows
 * accepted so far.  On KBE_OK and KBE_ERANGE the context's grid becomes the
 * accepted grid with the history orders used (as kbe_set_grid sets it). */
kbe_status kbe_run_controlled(kbe_ctx* ctx, const double* opts, const int* iopts, void* L, void* R,
                              void* S_less, void* S_great, void* I_work, void* F_ring, double* t_out,
                              int* q_out, int* korder_out, int* n_rows, int* stats, void* stream);

/* Storage of the split-precision contraction (KBE_SPLIT_BF16).  keep = 1
 * (the default): the first split slice allocates a buffer of the history's
 * digit planes (about twice the two triangles: 32 n_max^2 norb^2 bytes),
 * an encoder kernel fills it and the contraction streams it; during
 * kbe_step the planes of rows below the step's row are kept between steps
 * and only the new rows' entries are encoded again.  keep = 0: no plane
 * buffer (an existing one is freed, after a device synchronisation); every
 * split slice runs one persistent contraction that converts the FP64
 * history entries into digit planes inside the kernel, the form the batched
 * steps use.  The two round to different fixed-point grids (column
 * exponents over 16 resp. 8 history entries), each within the split
 * path's bound of the exact slice.  KBE_EINVAL unless keep is 0 or 1. */
kbe_status kbe_set_split_planes(kbe_ctx* ctx, int keep);

/* Forget per-history state kept between steps (the split path's digit
 * planes); the next step encodes every row again.  No GPU work. */
kbe_status kbe_reset_cache(kbe_ctx* ctx);

/* Synchronize stream and return the device status word accumulated since
 * the last call (then cleared): KBE_OK, KBE_ENUMERIC or KBE_ETIMEOUT. */
kbe_status kbe_sync_status(kbe_ctx* ctx, void* stream);

/* Test support for the device-side failure path (no fault is involved):
 * the next split-precision contraction launched on this context (by
 * kbe_history_slice, kbe_step, ... with KBE_SPLIT_BF16) issues no copy for
 * its work unit `unit` (a unit is one column tile of 128 / norb output
 * columns times one chunk of 16 history entries; the persistent CTA that
 * owns it stops producing there), and every wait of its pipeline gives up
 * after spin_limit polls (instead of about 2^26).  The consumers' bounded
 * waits run out, every CTA of the launch finishes the copies and MMAs it
 * had already issued, frees its tensor memory and returns, and
 * kbe_sync_status reports KBE_ETIMEOUT; the slice's output is then
 * undefined.  Later calls are unaffected (the setting applies to one launch
 * and clears itself).  A unit beyond the launch's last unit withholds
 * nothing.  KBE_EINVAL for unit < 0 or spin_limit < 1. */
kbe_status kbe_debug_withhold_split(kbe_ctx* ctx, long long unit, long long spin_limit);

/* Test support for the failure path of kbe_run_steps' cooperative launch
 * (no fault is involved): in the next such launch on this context, block 0
 * leaves the kernel at device-wide barrier number `barrier` (0 = the one
 * after the launch's first predictor, then four in the first sweep of each
 * step and three in each later sweep) without arriving,
 * and every barrier wait gives up after spin_limit polls (instead of about
 * 2^24).  The other blocks' waits run out and they return; kbe_sync_status
 * reports KBE_ETIMEOUT and the rows of that launch are undefined.  Later
 * launches are unaffected (the setting clears itself).  A barrier beyond the
 * launch's last withholds nothing.  KBE_EINVAL for barrier < 0 or
 * spin_limit < 1. */
kbe_status kbe_debug_withhold_run(kbe_ctx* ctx, int barrier, long long spin_limit);

/* Number of kernels the last kbe_* call on this context enqueued. */
int kbe_last_launch_count(const kbe_ctx* ctx);

/* Measurement support.  With profiling enabled, every history-contraction
 * kernel the context launches is bracketed by a CUDA event pair recorded on
 * its stream; kbe_set_profiling() also discards earlier records.
 * kbe_read_profiling() waits for the recorded events and returns how many
 * contraction kernels ran and their summed duration in milliseconds.
 * Event recording adds no kernels and no synchronization to the calls. */
kbe_status kbe_set_profiling(kbe_ctx* ctx, int enable);
kbe_status kbe_read_profiling(kbe_ctx* ctx, int* count, double* total_ms);

/* ------------------------------------------------------------ batching -- */
/* Many independent systems (each a context with its own norb, grid and
 * model) advanced together: one batched KBE step runs kbe_step's sequence
 * for every active system as ONE CUDA graph launch (batched elementwise
 * kernels, and for KBE_FP64 one persistent history kernel over a work list
 * of (system, tile, history chunk) items).  The paper steps one system;
 * this is a throughput form for ensembles of systems. */
typedef struct kbe_batch kbe_batch;

/* A batch over n_sys (1..1024) contexts on one device, each with its grid
 * and model already set (later kbe_set_grid / kbe_set_model calls on them
 * are not seen by the batch).  The contexts stay owned by the caller and
 * must outlive the batch; their workspaces are used by the batched calls,
 * so they must not run other calls concurrently.  Contexts with adaptive
 * history orders or a dense interaction are KBE_EINVAL. */
kbe_status kbe_batch_create(kbe_ctx* const* ctxs, int n_sys, kbe_batch** out);
kbe_status kbe_batch_destroy(kbe_batch* b);
const char* kbe_batch_last_error(const kbe_batch* b);
int kbe_batch_last_launch_count(const kbe_batch* b);  /* kernels of one batched step */

/* State of system i, with the layouts of kbe_step (triangles of the
 * context's n_max rows, self-energy rows, history slice, right-hand-side
 * ring); device pointers, borrowed. */
kbe_status kbe_batch_bind(kbe_batch* b, int i, void* L, void* R, void* S_less, void* S_great, void* I_work,
                          void* F_ring);

/* One batched step: system i advances row rows[i] (host int array of n_sys
 * entries) exactly as kbe_step(ctx_i, rows[i], P, precision, ...) would;
 * rows[i] < 1 leaves system i untouched, rows[i] >= n_t_i is KBE_ERANGE.
 * The graph of the step is captured on the first call and reused while P,
 * precision and the tile policy stay the same (KBE_SPLIT_BF16 graphs also
 * depend on the rows and are re-captured when they change).  With
 * KBE_SPLIT_BF16 every sweep contracts all active systems in ONE persistent
 * tensor-core launch over a work list of (system, column tile, history
 * chunk) units, split into contiguous ranges of about equal cost, one per
 * SM; the kernel converts each unit's FP64 history entries into digit
 * planes itself (no plane buffer), then a reduction launch adds the partial
 * sums and the band term of every system's columns.  The work list (a few
 * KB to MB) and the partial sums are held by the batch, allocated by the
 * first split step that needs them (KBE_ENOMEM if that fails), and the work
 * list is uploaded on `stream` when the rows change.  Results agree with
 * kbe_step to rounding (the history sum is chunked differently).
 * precision: KBE_FP64, KBE_SPLIT_BF16 or KBE_DF64 (each system's
 * double-float slice in its own context's workspace, graph re-captured
 * when the rows change, like KBE_SPLIT_BF16). */
kbe_status kbe_batch_step(kbe_batch* b, const int* rows, int P, int precision, void* stream);

/* Tile policy of the persistent FP64 history kernel: `block` output entries
 * per work item (128 or 256) and a target of 2^item_work_log2 complex
 * multiply-adds per item (10..40), which sets each system's history chunk
 * length.  Default (256, 20). */
kbe_status kbe_batch_set_policy(kbe_batch* b, int block, int item_work_log2);
kbe_status kbe_batch_get_policy(const kbe_batch* b, int* block, int* item_work_log2);

/* Autotuner: times the persistent history kernel of the batch at `rows`
 * for each candidate policy (block 128 or 256, item_work_log2 = 14, 16, ..,
 * 26; `reps` timed runs after one warm-up, CUDA events on `stream`), keeps
 * the fastest (kbe_batch_set_policy) and returns it with its time in ms.
 * Synchronous.  Overwrites the self-energy rows and history slices of the
 * systems active at `rows`. */
kbe_status kbe_batch_autotune(kbe_batch* b, const int* rows, int reps, void* stream, int* block_out,
                              int* item_work_log2_out, double* best_ms);

/* Synchronize stream and return (then clear) the batch's device status. */
kbe_status kbe_batch_sync_status(kbe_batch* b, void* stream);

/* ------------------------------------------------ allocation-free entry -- */

/* History slice of row n (the same Eq. KBE2 contraction and kernels as
 * kbe_history_slice, KBE_FP64) for callers that cannot allocate device
 * memory: code that runs inside another framework's memory pool or
 * allocator hooks (a nested cudaMalloc there would re-enter the allocator
 * or escape its accounting), or hosts that only hand over fixed buffers.
 * The paper has no counterpart; this entry exists for those callers.
 *
 * No context: the grid t[0..n_t-1], order[1..n_t-1] is passed on the host
 * (same validation as kbe_set_grid) and its weights are recomputed on each
 * call.  L, R, S_less, S_great, I_out are the caller's device buffers with
 * the layouts of kbe_history_slice.  All scratch lives in one static
 * device array of 64 MiB that every GPU loading the library reserves until
 * the process exits: n_t <= 8192 and (n+1)*norb^2 <= about 1.37e6 complex
 * entries, else KBE_EINVAL with a message in kbe_last_error(NULL) (the
 * last context-free error of the calling host thread).  The
 * call allocates no device memory (no cudaMalloc, cudaFree or allocating
 * library routine).  Its first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make
 * that first call before any stream capture.  The weight tables are
 * copied from pageable host memory, so the call waits for earlier work on
 * `stream`.  Every call shares the array and leaves its contents behind;
 * calls whose kernels overlap on the GPU race on it.  Non-finite values
 * are not reported (there is no context to hold a status word). */
kbe_status kbe_history_slice_noalloc(int norb, int n, const double* t, const int* order, int n_t,
                                     const void* L, const void* R, const void* S_less,
                                     const void* S_great, void* I_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* KBE_H */
