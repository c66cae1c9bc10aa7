// weights.cpp -- host FP64 quadrature weights of Sec. 3.2.
//
// Local rule (Eq. weights): the degree-k interpolant of g through the nodes
// tau_0..tau_k, integrated over [lo, hi], is sum_j w_j g(tau_j) with
//   sum_j w_j u_j^i = T_i,  u_j = (tau_j - c0)/S,
//   T_i = integral_lo^hi ((s - c0)/S)^i ds,     i = 0..k,
// i.e. V^T w = T for the Vandermonde matrix V_ji = u_j^i.  The system is
// solved by Gaussian elimination with full pivoting, as the paper does
// (Eigen's fully pivoted LU).  The paper expands in (s - t_{n-k})^i; the
// centred, scaled monomials used here (c0, S: centre and half-width of the
// nodes) give the same weights with a far better conditioned V.
//
// Composite rows (Sec. 3.2): w_{n,i} = w_{n-1,i} plus the local weights of
// interval n on i = n-k..n.  Entries below n-K never change again, so a
// settled vector and a band of width K+1 describe every row.

#include <cmath>
#include <cstring>

#include "kbe_internal.h"

namespace kbe {
namespace {

// Solve A x = b for n <= kWTab by Gaussian elimination with full pivoting.
bool solve_full_pivot(int n, double* A, double* b, double* x) {
  int col[kWTab];
  for (int i = 0; i < n; ++i) col[i] = i;
  for (int k = 0; k < n; ++k) {
    int pr = k, pc = k;
    double best = 0.0;
    for (int i = k; i < n; ++i)
      for (int j = k; j < n; ++j)
        if (std::fabs(A[i * n + j]) > best) { best = std::fabs(A[i * n + j]); pr = i; pc = j; }
    if (!(best > 0.0) || !std::isfinite(best)) return false;
    if (pr != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[pr * n + j]);
      std::swap(b[k], b[pr]);
    }
    if (pc != k) {
      for (int i = 0; i < n; ++i) std::swap(A[i * n + k], A[i * n + pc]);
      std::swap(col[k], col[pc]);
    }
    for (int i = k + 1; i < n; ++i) {
      const double f = A[i * n + k] / A[k * n + k];
      A[i * n + k] = 0.0;
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      b[i] -= f * b[k];
    }
  }
  double y[kWTab];
  for (int k = n - 1; k >= 0; --k) {
    double s = b[k];
    for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * y[j];
    y[k] = s / A[k * n + k];
  }
  for (int k = 0; k < n; ++k) x[col[k]] = y[k];
  return true;
}

}  // namespace

kbe_status local_weights(const double* tau, int k, double lo, double hi, double* w, std::string* err) {
  if (!tau || !w || k < 0 || k > kMaxOrder || !(hi > lo)) {
    if (err) *err = "local_weights: bad arguments";
    return KBE_EINVAL;
  }
  if (k == 0) { w[0] = hi - lo; return KBE_OK; }
  const int n = k + 1;
  // Monomials in u = (s - c0)/S, with c0 and S the centre and half-width of
  // the node span, keep V well conditioned (nodes in [-1, 1]); the weights
  // do not depend on the basis.
  const double c0 = 0.5 * (tau[0] + tau[k]), S = 0.5 * (tau[k] - tau[0]);
  if (!(S > 0.0)) {
    if (err) *err = "local_weights: repeated nodes";
    return KBE_EINVAL;
  }
  double A[kWTab * kWTab], T[kWTab];
  for (int j = 0; j < n; ++j) {
    const double u = (tau[j] - c0) / S;
    double p = 1.0;
    for (int i = 0; i < n; ++i) { A[i * n + j] = p; p *= u; }  // A = V^T
  }
  const double a = (lo - c0) / S, b = (hi - c0) / S;
  double pa = a, pb = b;
  for (int i = 0; i < n; ++i) {
    T[i] = S * (pb - pa) / (i + 1);
    pa *= a; pb *= b;
  }
  if (!solve_full_pivot(n, A, T, w)) {
    if (err) *err = "local_weights: singular Vandermonde system (repeated nodes)";
    return KBE_EINVAL;
  }
  return KBE_OK;
}

kbe_status build_grid(const double* t, const int* order, int n_t, HostGrid* g, std::string* err) {
  if (!t || !order || n_t < 1) { *err = "set_grid: null array or n_t < 1"; return KBE_EINVAL; }
  if (t[0] != 0.0) { *err = "set_grid: t[0] must be 0"; return KBE_EINVAL; }
  for (int l = 1; l < n_t; ++l) {
    if (!std::isfinite(t[l]) || !(t[l] > t[l - 1])) {
      *err = "set_grid: t must be finite and strictly increasing (index " + std::to_string(l) + ")";
      return KBE_EINVAL;
    }
    if (order[l] < 1 || order[l] > kMaxOrder) {
      *err = "set_grid: order[" + std::to_string(l) + "] = " + std::to_string(order[l]) +
             " outside [1, " + std::to_string(kMaxOrder) + "]";
      return KBE_ERANGE;
    }
  }
  g->n_t = n_t;
  g->t.assign(t, t + n_t);
  g->order.assign(n_t, 0);
  int K = 1;
  for (int l = 1; l < n_t; ++l) {
    g->order[l] = order[l];
    const int kap = order[l] < l ? order[l] : l;
    if (kap > K) K = kap;
  }
  g->K = K;
  const int bw = K + 1;
  g->wbar.assign(n_t, 0.0);
  g->band.assign((size_t)n_t * bw, 0.0);
  g->corr.assign((size_t)n_t * kMaxOrder * kWTab, 0.0);
  g->pred.assign((size_t)n_t * kMaxOrder * kWTab, 0.0);
  std::vector<double>& cur = g->wbar;  // running composite row
  double w[kWTab];
  for (int c = 1; c < n_t; ++c) {
    const int kap = order[c] < c ? order[c] : c;
    kbe_status st = local_weights(t + c - kap, kap, t[c - 1], t[c], w, err);
    if (st != KBE_OK) return st;
    for (int j = 0; j <= kap; ++j) cur[c - kap + j] += w[j];
    for (int j = 0; j < bw && j <= c; ++j) g->band[(size_t)c * bw + j] = cur[c - j];
    // stepper tables for row c: corrector over t_{c-kap..c}, predictor over t_{c-q..c-1}
    const int kmax = order[c] < c ? order[c] : c;
    for (int kk = 1; kk <= kmax; ++kk) {
      st = local_weights(t + c - kk, kk, t[c - 1], t[c], w, err);
      if (st != KBE_OK) return st;
      for (int j = 0; j <= kk; ++j) g->corr[((size_t)c * kMaxOrder + (kk - 1)) * kWTab + j] = w[j];
      st = local_weights(t + c - kk, kk - 1, t[c - 1], t[c], w, err);
      if (st != KBE_OK) return st;
      for (int j = 0; j < kk; ++j) g->pred[((size_t)c * kMaxOrder + (kk - 1)) * kWTab + j] = w[j];
    }
  }
  return KBE_OK;
}

double Model::shape(double t) const {
  const double x = (t - t0) / sigma;
  return std::exp(-0.5 * x * x) * std::cos(omega * t);
}

double Model::field(double t) const {
  if (E0 == 0.0) return 0.0;
  return E0 * shape(t);
}

}  // namespace kbe
