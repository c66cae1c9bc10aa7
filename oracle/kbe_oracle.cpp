// kbe_oracle.cpp -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, FP64 CPU reference for the hot path of the adaptive
// Kadanoff-Baym solver of Blommel, Gardner, Woodward and Gull
// (arXiv 2405.08737).  Only the tests, the smoke check and the CPU-baseline
// leg of the benchmark may load this library.  The product path never calls
// it and shares no code with it.
//
// Every routine follows the paper's definitions literally:
//   * quadrature weights -- Sec. 3.2, Eq. (weights): integrate the degree-k
//     interpolant through t_{l-k..l} over [t_{l-1}, t_l].  The Lagrange basis
//     polynomials are integrated by Gauss-Legendre, a route independent of the
//     paper's Vandermonde solve; both give the same numbers.
//   * composite weights -- Sec. 3.2: w_{n,m} = sum over intervals l <= n of
//     the local weights, summed directly (the recursion is not used here).
//   * self-energy -- Sec. 2, Eq. (SE), summed over the non-zero entries of
//     the four-index Coulomb tensor.
//   * Fock matrix -- Eq. (eps), for the local tensor or a general real one.
//   * thermal branch -- Sec. 2, Eq. (KBE3) and the tau terms of Eq. (KBE2) on
//     a uniform tau grid with the same kind of composite weights.
//   * history integrals -- Sec. 2, Eq. (KBE2), and Eq. (KBE1) for the adjoint
//     identity, with theta(0) = 1 and G(t,t') = -G(t',t)^+.
//   * stepper -- integral-form Adams-Moulton on the same kind of weights with
//     P fixed-point sweeps (Sec. 3.1 solves each step by fixed-point
//     iteration; Sec. 5.3 reports about two sweeps per step).
//
// Storage convention (input format, not arithmetic): two-time arrays hold
// the lower triangle r >= c; block p(r,c) = r(r+1)/2 + c is an MxM row-major
// complex128 matrix.  L(r,c) = G^<(t_r,t_c), R(r,c) = G^R(t_r,t_c), and
// R(r,r) = -i*1 (Eq. BC with theta(0) = 1).
//
// History sums are Neumaier-compensated.  The arithmetic type is a template
// parameter so that the stepper also runs on forward-mode dual numbers,
// which gives exact directional derivatives of the discrete map.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- scalars --
struct Dual {  // value and directional derivative
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double a) : v(a), d(0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline bool is_zero(double x) { return x == 0.0; }
inline bool is_zero(Dual x) { return x.v == 0.0 && x.d == 0.0; }

template <class T> struct Cx {
  T re, im;
  Cx() : re(0.0), im(0.0) {}
  Cx(T a) : re(a), im(0.0) {}
  Cx(T a, T b) : re(a), im(b) {}
};
template <class T> inline Cx<T> operator+(Cx<T> a, Cx<T> b) { return Cx<T>(a.re + b.re, a.im + b.im); }
template <class T> inline Cx<T> operator-(Cx<T> a, Cx<T> b) { return Cx<T>(a.re - b.re, a.im - b.im); }
template <class T> inline Cx<T> operator-(Cx<T> a) { return Cx<T>(-a.re, -a.im); }
template <class T> inline Cx<T> operator*(Cx<T> a, Cx<T> b) {
  return Cx<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class T> inline Cx<T> scale(T s, Cx<T> a) { return Cx<T>(s * a.re, s * a.im); }
template <class T> inline Cx<T> conj(Cx<T> a) { return Cx<T>(a.re, -a.im); }
template <class T> inline Cx<T> mul_mi(Cx<T> a) { return Cx<T>(a.im, -a.re); }  // -i * a

using C64 = Cx<double>;

// Neumaier compensated accumulation, per real component.
inline void nadd(double& s, double& c, double x) {
  double t = s + x;
  if (std::fabs(s) >= std::fabs(x)) c += (s - t) + x; else c += (x - t) + s;
  s = t;
}
template <class T> struct Acc;
template <> struct Acc<double> {
  double sr = 0, cr = 0, si = 0, ci = 0;
  void add(C64 x) { nadd(sr, cr, x.re); nadd(si, ci, x.im); }
  C64 get() const { return C64(sr + cr, si + ci); }
};
template <> struct Acc<Dual> {
  double sr = 0, cr = 0, si = 0, ci = 0, dsr = 0, dcr = 0, dsi = 0, dci = 0;
  void add(Cx<Dual> x) {
    nadd(sr, cr, x.re.v); nadd(si, ci, x.im.v);
    nadd(dsr, dcr, x.re.d); nadd(dsi, dci, x.im.d);
  }
  Cx<Dual> get() const { return Cx<Dual>(Dual(sr + cr, dsr + dcr), Dual(si + ci, dsi + dci)); }
};

inline int64_t tri(int64_t r, int64_t c) { return r * (r + 1) / 2 + c; }

// ----------------------------------------------------- quadrature weights --
// Gauss-Legendre nodes and weights on [-1,1]: Newton iteration on P_q, with
// P_q from the recurrence k P_k = (2k-1) x P_{k-1} - (k-1) P_{k-2}.
void legendre_eval(int q, double z, double* pq, double* dpq) {
  double p0 = 1.0, p1 = z;
  for (int k = 2; k <= q; ++k) {
    double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
    p0 = p1; p1 = pk;
  }
  *pq = p1;
  *dpq = (q == 1) ? 1.0 : q * (z * p1 - p0) / (z * z - 1.0);
}
void gauss_legendre(int q, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < q; ++i) {
    double z = std::cos(pi * (i + 0.75) / (q + 0.5)), p, dp;
    for (int it = 0; it < 100; ++it) {
      legendre_eval(q, z, &p, &dp);
      double dz = p / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    legendre_eval(q, z, &p, &dp);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// w[j] = integral over [lo,hi] of the Lagrange basis polynomial l_j on the
// nodes tau[0..k] -- the weights of the degree-k interpolatory rule of
// Eq. (weights).  12 Gauss-Legendre points are exact up to degree 23.
void lagrange_weights(const double* tau, int k, double lo, double hi, double* w) {
  const int q = 12;
  double gx[q], gw[q];
  gauss_legendre(q, gx, gw);
  const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
  for (int j = 0; j <= k; ++j) {
    double s = 0.0;
    for (int g = 0; g < q; ++g) {
      double x = mid + half * gx[g], lj = 1.0;
      for (int i = 0; i <= k; ++i)
        if (i != j) lj *= (x - tau[i]) / (tau[j] - tau[i]);
      s += gw[g] * lj;
    }
    w[j] = half * s;
  }
}

inline int eff_order(const int* order, int l) { return order[l] < l ? order[l] : l; }

// Composite row w_{n,m}, m = 0..n: direct sum over the intervals l = 1..n of
// the local weights of order kappa_l = min(order[l], l).
void composite_row(const double* t, const int* order, int n, double* row) {
  for (int m = 0; m <= n; ++m) row[m] = 0.0;
  double w[64];
  for (int l = 1; l <= n; ++l) {
    const int kap = eff_order(order, l);
    lagrange_weights(t + (l - kap), kap, t[l - 1], t[l], w);
    for (int j = 0; j <= kap; ++j) row[l - kap + j] += w[j];
  }
}

// ------------------------------------------- adaptive history orders ---
// Order selection of Sec. 3.2 for interval n: the test integral of u over
// [t_{n-1}, t_n] with the order-k interpolatory rule through t_{n-k..n},
//   I^(k) = sum_j w^(k)_j u(t_{n-k+j}),  k = 1..kmax (kmax = min(K, n)),
// and k_opt = argmin_{k >= 2} |I^(k) - I^(k-1)| in the max norm over the
// M x M entries (k_opt = 1 when kmax = 1).  Differences that lie within a
// rounding tolerance (64 eps times the largest |I^(k)|) of the minimum are
// not distinguished: the lowest such order is taken.
// u: [kmax+1][M*M] values at t_{n-kmax} .. t_n; diffs[k] = |I^(k) - I^(k-1)|.
int choose_order(const double* t, int n, int K, int M, const C64* u, double* diffs) {
  const int kmax = K < n ? K : n;
  if (kmax <= 1) {
    if (diffs) diffs[1] = 0.0;
    return 1;
  }
  const int MM = M * M;
  std::vector<C64> I((size_t)(kmax + 1) * MM);
  double w[64];
  double mag = 0.0;
  for (int k = 1; k <= kmax; ++k) {
    lagrange_weights(t + (n - k), k, t[n - 1], t[n], w);
    for (int e = 0; e < MM; ++e) {
      C64 acc;
      for (int j = 0; j <= k; ++j) acc = acc + scale(w[j], u[(size_t)(kmax - k + j) * MM + e]);
      I[(size_t)k * MM + e] = acc;
      mag = std::max(mag, std::hypot(acc.re, acc.im));
    }
  }
  std::vector<double> d(kmax + 1, 0.0);
  double dmin = 1e300;
  for (int k = 2; k <= kmax; ++k) {
    double m = 0.0;
    for (int e = 0; e < MM; ++e) {
      const C64 x = I[(size_t)k * MM + e] - I[(size_t)(k - 1) * MM + e];
      m = std::max(m, std::hypot(x.re, x.im));
    }
    d[k] = m;
    dmin = std::min(dmin, m);
  }
  if (diffs) for (int k = 1; k <= kmax; ++k) diffs[k] = d[k];
  const double tol = 64.0 * 2.220446049250313e-16 * mag;
  for (int k = 2; k <= kmax; ++k)
    if (d[k] <= dmin + tol) return k;
  return kmax;
}

// -------------------------------------------------- two-time plane access --
// Values anywhere in the (t,t') plane from the stored lower triangles:
// G^<> (t,t') = -G^<>(t',t)^+ (Sec. 2), G^> = G^R + G^< on and below the
// diagonal (definition of G^R with theta(0) = 1), G^A(t,t') = G^R(t',t)^+.
template <class T> struct Plane {
  int M;
  const Cx<T>* L;
  const Cx<T>* R;
  Cx<T> l_at(int r, int c, int a, int b) const { return L[tri(r, c) * M * M + a * M + b]; }
  Cx<T> r_at(int r, int c, int a, int b) const { return R[tri(r, c) * M * M + a * M + b]; }
  Cx<T> less(int r, int c, int a, int b) const {
    if (r >= c) return l_at(r, c, a, b);
    return -conj(l_at(c, r, b, a));
  }
  Cx<T> great(int r, int c, int a, int b) const {
    if (r >= c) return r_at(r, c, a, b) + l_at(r, c, a, b);
    return -conj(r_at(c, r, b, a) + l_at(c, r, b, a));
  }
  Cx<T> ret(int r, int c, int a, int b) const {
    if (r >= c) return r_at(r, c, a, b);
    return Cx<T>();
  }
  Cx<T> adv(int r, int c, int a, int b) const {
    if (r <= c) return conj(r_at(c, r, b, a));
    return Cx<T>();
  }
  Cx<T> get(int s, int r, int c, int a, int b) const { return s == 0 ? less(r, c, a, b) : great(r, c, a, b); }
};

// ------------------------------------------------------------ self-energy --
// Row n of Eq. (SE):  S^<>(n,c)_ij for c = 0..n,
//   S^<>_ij(t,t') = U_ifde UEx_jabc G^<>_fb(t,t') G^<>_ea(t,t') G^><_cd(t',t),
//   UEx_jabc = 2 U_jbac - U_jabc,
// summed over the entries where U and UEx are non-zero.
template <class T>
void sigma_row(const Plane<T>& G, const T* U4, int n, Cx<T>* Sl, Cx<T>* Sg) {
  const int M = G.M;
  auto at = [M](int a, int b, int c, int d) { return ((a * M + b) * M + c) * M + d; };
  struct E { int i, f, d, e; T u; };
  std::vector<E> nzU, nzX;  // nzX holds (j,a,b,c) in (i,f,d,e)
  for (int i = 0; i < M; ++i)
    for (int f = 0; f < M; ++f)
      for (int d = 0; d < M; ++d)
        for (int e = 0; e < M; ++e) {
          T u = U4[at(i, f, d, e)];
          T ux = T(2.0) * U4[at(i, d, f, e)] - U4[at(i, f, d, e)];  // UEx_{j a b c}: U_{j b a c}
          if (!is_zero(u)) nzU.push_back({i, f, d, e, u});
          if (!is_zero(ux)) nzX.push_back({i, f, d, e, ux});
        }
  for (int c = 0; c <= n; ++c) {
    Cx<T>* sl = Sl + (int64_t)c * M * M;
    Cx<T>* sg = Sg + (int64_t)c * M * M;
    for (int k = 0; k < M * M; ++k) { sl[k] = Cx<T>(); sg[k] = Cx<T>(); }
    for (const E& p : nzU) {       // p = (i, f, d, e)
      for (const E& q : nzX) {     // q = (j, a, b, c')
        const int i = p.i, f = p.f, d = p.d, e = p.e;
        const int j = q.i, a = q.f, b = q.d, cc = q.e;
        const T uu = p.u * q.u;
        // S^>: G^>_fb(t,t') G^>_ea(t,t') G^<_cd(t',t);  S^<: the same with < and > swapped
        Cx<T> g = G.great(n, c, f, b) * G.great(n, c, e, a) * G.less(c, n, cc, d);
        Cx<T> l = G.less(n, c, f, b) * G.less(n, c, e, a) * G.great(c, n, cc, d);
        sg[i * M + j] = sg[i * M + j] + scale(uu, g);
        sl[i * M + j] = sl[i * M + j] + scale(uu, l);
      }
    }
  }
}

// -------------------------------------------------------- history slices --
// Plane access to the self-energy of row n: S^s(n,c) stored for c <= n;
// S^s(c,n) = -S^s(n,c)^+ for c < n; Sigma^R(n,m) = S^>(n,m) - S^<(n,m) for
// m <= n (theta(0) = 1); Sigma^A(m,n) = Sigma^R(n,m)^+.
template <class T> struct SigmaRow {
  int M;
  const Cx<T>* Sl;
  const Cx<T>* Sg;
  Cx<T> s_nm(int s, int m, int a, int b) const {
    return (s == 0 ? Sl : Sg)[(int64_t)m * M * M + a * M + b];
  }
  Cx<T> ret_nm(int m, int a, int b) const { return s_nm(1, m, a, b) - s_nm(0, m, a, b); }
  Cx<T> s_mn(int s, int m, int n, int a, int b) const {  // Sigma^s(t_m, t_n), m <= n
    if (m == n) return s_nm(s, m, a, b);
    return -conj(s_nm(s, m, b, a));
  }
  Cx<T> adv_mn(int m, int a, int b) const { return conj(ret_nm(m, b, a)); }
};

inline double value_of(double x) { return x; }
inline double value_of(Dual x) { return x.v; }

// Test integrand of the order selection (Sec. 3.2) at t_bar = t_l, l <= n:
//   u(t_l) = G^R(t_n, t_l) Sigma^<(t_l, t_n) + G^<(t_n, t_l) Sigma^A(t_l, t_n),
// the integrand of Eq. (KBE1) for G^<(t_n, t_n); values only (no tangents).
template <class T>
void test_integrand(const Plane<T>& G, const SigmaRow<T>& S, int n, int l, C64* u) {
  const int M = G.M;
  for (int a = 0; a < M; ++a)
    for (int b = 0; b < M; ++b) {
      Cx<T> acc;
      for (int x = 0; x < M; ++x)
        acc = acc + G.ret(n, l, a, x) * S.s_mn(0, l, n, x, b) + G.less(n, l, a, x) * S.adv_mn(l, x, b);
      u[a * M + b] = C64(value_of(acc.re), value_of(acc.im));
    }
}

// Chooses the history order of interval n from the current rows (Sec. 3.2).
template <class T>
int select_history_order(const Plane<T>& G, const SigmaRow<T>& S, const double* t, int n, int K) {
  const int kmax = K < n ? K : n;
  if (kmax <= 1) return 1;
  const int MM = G.M * G.M;
  std::vector<C64> u((size_t)(kmax + 1) * MM);
  for (int i = 0; i <= kmax; ++i) test_integrand(G, S, n, n - kmax + i, u.data() + (size_t)i * MM);
  return choose_order(t, n, K, G.M, u.data(), nullptr);
}

// Eq. (KBE2) history integrals for row n, both s in {<, >} and c = 0..n:
//   I^s(n,c) = sum_{m=0..n} w_{n,m} Sigma^R(n,m) G^s(m,c)
//            + sum_{m=0..c} w_{c,m} Sigma^s(n,m) G^A(m,c).
// out layout [s][c][a][b].  Threads split the output columns c.
template <class T>
void history_slice(const Plane<T>& G, const SigmaRow<T>& S, const double* t, const int* order,
                   int n, Cx<T>* out, int nthreads) {
  const int M = G.M;
  std::vector<std::vector<double>> w(n + 1);
  for (int c = 0; c <= n; ++c) { w[c].resize(c + 1); composite_row(t, order, c, w[c].data()); }
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) collapse(2)
  for (int s = 0; s < 2; ++s)
    for (int c = 0; c <= n; ++c) {
      for (int a = 0; a < M; ++a)
        for (int b = 0; b < M; ++b) {
          Acc<T> acc;
          for (int m = 0; m <= n; ++m)
            for (int x = 0; x < M; ++x)
              acc.add(scale(T(w[n][m]), S.ret_nm(m, a, x) * G.get(s, m, c, x, b)));
          for (int m = 0; m <= c; ++m)
            for (int x = 0; x < M; ++x)
              acc.add(scale(T(w[c][m]), S.s_nm(s, m, a, x) * G.adv(m, c, x, b)));
          out[(((int64_t)s * (n + 1) + c) * M + a) * M + b] = acc.get();
        }
    }
}

// Eq. (KBE1), lesser form, at (t_c, t_n) for c = 0..n:
//   J(c) = sum_{m=0..c} w_{c,m} G^R(c,m) Sigma^<(m,n)
//        + sum_{m=0..n} w_{n,m} G^<(c,m) Sigma^A(m,n).
template <class T>
void kbe1_slice(const Plane<T>& G, const SigmaRow<T>& S, const double* t, const int* order,
                int n, Cx<T>* out, int nthreads) {
  const int M = G.M;
  std::vector<std::vector<double>> w(n + 1);
  for (int c = 0; c <= n; ++c) { w[c].resize(c + 1); composite_row(t, order, c, w[c].data()); }
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
  for (int c = 0; c <= n; ++c)
    for (int a = 0; a < M; ++a)
      for (int b = 0; b < M; ++b) {
        Acc<T> acc;
        for (int m = 0; m <= c; ++m)
          for (int x = 0; x < M; ++x)
            acc.add(scale(T(w[c][m]), G.ret(c, m, a, x) * S.s_mn(0, m, n, x, b)));
        for (int m = 0; m <= n; ++m)
          for (int x = 0; x < M; ++x)
            acc.add(scale(T(w[n][m]), G.less(c, m, a, x) * S.adv_mn(m, x, b)));
        out[((int64_t)c * M + a) * M + b] = acc.get();
      }
}

// ---------------------------------------------------------------- stepper --
// Model: h(t) = h0 + E(t) diag(v), E(t) = E0 exp(-(t-t0)^2/(2 sigma^2)) cos(omega t);
// local interaction U_a (Coulomb tensor U_abcd = U_a delta_abcd), or, when
// U4d is set, a general real tensor U4d[((i*M + a)*M + b)*M + j] = U_iabj.
// Fock matrix (Eq. eps):
//   eps_ij = h_ij(t) + i sum_ab (U_iabj - 2 U_ijba) G^<_ba(t,t);
// for the local tensor this is eps = h(t) + diag(U_a n_a), n_a = Im L(t,t)_aa
// (the real part of -i G^<_aa(t,t)).
template <class T> struct Model {
  int M;
  const C64* h0;
  const T* U;
  const double* v;
  T E0;
  double t0, sig, om;
  const T* U4d = nullptr;
};

template <class T> T pulse(const Model<T>& md, double t) {
  const double g = std::exp(-(t - md.t0) * (t - md.t0) / (2.0 * md.sig * md.sig)) * std::cos(md.om * t);
  return md.E0 * T(g);
}

template <class T> void fock(const Model<T>& md, double t, const Cx<T>* Lnn, Cx<T>* eps) {
  const int M = md.M;
  const T e = pulse(md, t);
  for (int a = 0; a < M; ++a)
    for (int b = 0; b < M; ++b) eps[a * M + b] = Cx<T>(T(md.h0[a * M + b].re), T(md.h0[a * M + b].im));
  if (!md.U4d) {
    for (int a = 0; a < M; ++a) {
      eps[a * M + a].re = eps[a * M + a].re + e * T(md.v[a]) + md.U[a] * Lnn[a * M + a].im;
    }
    return;
  }
  auto at = [M](int p, int q, int r, int s) { return ((p * M + q) * M + r) * M + s; };
  for (int a = 0; a < M; ++a) eps[a * M + a].re = eps[a * M + a].re + e * T(md.v[a]);
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) {
      Cx<T> hf;
      for (int a = 0; a < M; ++a)
        for (int b = 0; b < M; ++b)
          hf = hf + scale(md.U4d[at(i, a, b, j)] - T(2.0) * md.U4d[at(i, j, b, a)], Lnn[b * M + a]);
      eps[i * M + j] = eps[i * M + j] + Cx<T>(-hf.im, hf.re);  // + i * hf
    }
}

// Row of right-hand sides F^s(j,c) = -i ( eps(t_j) G^s(j,c) + I^s(j,c) ), c = 0..j
// (the t-derivative from Eq. (KBE2)); layout [s][c][a][b].
template <class T>
void rhs_row(const Model<T>& md, const Plane<T>& G, const double* t, const Cx<T>* I, int j, Cx<T>* F) {
  const int M = md.M;
  std::vector<Cx<T>> eps(M * M);
  fock(md, t[j], G.L + tri(j, j) * M * M, eps.data());
  for (int s = 0; s < 2; ++s)
    for (int c = 0; c <= j; ++c)
      for (int a = 0; a < M; ++a)
        for (int b = 0; b < M; ++b) {
          Cx<T> acc = I[(((int64_t)s * (j + 1) + c) * M + a) * M + b];
          for (int x = 0; x < M; ++x) acc = acc + eps[a * M + x] * G.get(s, j, c, x, b);
          F[(((int64_t)s * (j + 1) + c) * M + a) * M + b] = mul_mi(acc);
        }
}

// Weights of the rule that integrates, over [t_{n-1}, t_n], the interpolant
// through the points t_first .. t_last.
void span_weights(const double* t, int first, int last, int n, double* w) {
  lagrange_weights(t + first, last - first, t[n - 1], t[n], w);
}

// Unrolled access to the stored right-hand sides: ring of K+1 rows.
template <class T> struct Ring {
  int M, N, K;
  std::vector<Cx<T>> F;  // [K+1][2][N][M][M]
  Cx<T>* row(int j) { return F.data() + (int64_t)(j % (K + 1)) * 2 * N * M * M; }
  Cx<T> at(int j, int s, int c, int a, int b) {  // row j holds j+1 columns per s
    return row(j)[(((int64_t)s * (j + 1) + c) * M + a) * M + b];
  }
};

// One KBE step for row n (Sec. 3.1 structure, integral form):
//  predictor   G^s(n,c) = G^s(n-1,c) + sum_p wp_p F^s(n-q+p, c),   q = min(k_n, n-c) points
//              t_{n-q..n-1} (Adams-Bashforth type); diagonal with D(j) = F^<(j,j) - F^<(j,j)^+
//              and q = min(k_n, n).
//  P sweeps:   Sigma row n, history row n, F row n, then the corrector
//              G^s(n,c) = G^s(n-1,c) + sum_p w_p F^s(n-kap+p, c),  kap = min(k_n, n-c)
//              (Adams-Moulton type, points t_{n-kap..n}), diagonal kap = min(k_n, n).
//  G^>(n,c) for c < n comes from the stepped G^> and G^<:  R(n,c) = G^>(n,c) - L(n,c);
//  R(n,n) = -i*1.  F row n keeps the value of the last evaluation.
// hord: orders of the history quadrature per interval (the stepper's orders
// `order` are separate); with K_sel > 0, hord[n] is chosen in every sweep by
// select_history_order (Sec. 3.2), otherwise hord is read only.
template <class T>
void kbe_step(const Model<T>& md, const double* t, const int* order, int n, int P,
              const T* U4, Cx<T>* L, Cx<T>* R, Ring<T>& ring, Cx<T>* I_last, int nthreads,
              int* hord = nullptr, int K_sel = 0) {
  const int M = md.M;
  const int* horder = hord ? hord : order;
  const int MM = M * M;
  const int kn = order[n];
  Plane<T> G{M, L, R};
  std::vector<Cx<T>> Gl((n + 1) * MM), Gg((n + 1) * MM);  // stepped G^< and G^> of row n
  double w[64];
  auto old_less = [&](int c, int k) { return L[tri(n - 1, c) * MM + k]; };
  auto old_great = [&](int c, int k) { return R[tri(n - 1, c) * MM + k] + L[tri(n - 1, c) * MM + k]; };
  auto diag_D = [&](int j, int a, int b) {  // total derivative of G^<(t,t) at t_j
    return ring.at(j, 0, j, a, b) - conj(ring.at(j, 0, j, b, a));
  };
  // predictor
  for (int c = 0; c < n; ++c) {
    const int q = (kn < n - c) ? kn : (n - c);
    span_weights(t, n - q, n - 1, n, w);
    for (int k = 0; k < MM; ++k) {
      Cx<T> al = old_less(c, k), ag = old_great(c, k);
      for (int p = 0; p < q; ++p) {
        const int j = n - q + p;
        al = al + scale(T(w[p]), ring.at(j, 0, c, k / M, k % M));
        ag = ag + scale(T(w[p]), ring.at(j, 1, c, k / M, k % M));
      }
      Gl[c * MM + k] = al; Gg[c * MM + k] = ag;
    }
  }
  {
    const int q = (kn < n) ? kn : n;
    span_weights(t, n - q, n - 1, n, w);
    for (int k = 0; k < MM; ++k) {
      Cx<T> al = L[tri(n - 1, n - 1) * MM + k];
      for (int p = 0; p < q; ++p) al = al + scale(T(w[p]), diag_D(n - q + p, k / M, k % M));
      Gl[n * MM + k] = al;
    }
  }
  auto commit = [&]() {
    for (int c = 0; c < n; ++c)
      for (int k = 0; k < MM; ++k) {
        L[tri(n, c) * MM + k] = Gl[c * MM + k];
        R[tri(n, c) * MM + k] = Gg[c * MM + k] - Gl[c * MM + k];
      }
    for (int k = 0; k < MM; ++k) {
      L[tri(n, n) * MM + k] = Gl[n * MM + k];
      R[tri(n, n) * MM + k] = (k / M == k % M) ? Cx<T>(T(0.0), T(-1.0)) : Cx<T>();
    }
  };
  commit();
  std::vector<Cx<T>> Sl((n + 1) * MM), Sg((n + 1) * MM), I(2 * (n + 1) * MM);
  for (int sweep = 0; sweep < P; ++sweep) {
    sigma_row(G, U4, n, Sl.data(), Sg.data());
    SigmaRow<T> S{M, Sl.data(), Sg.data()};
    if (K_sel > 0 && hord) hord[n] = select_history_order(G, S, t, n, K_sel);
    history_slice(G, S, t, horder, n, I.data(), nthreads);
    rhs_row(md, G, t, I.data(), n, ring.row(n));
    // corrector
    for (int c = 0; c < n; ++c) {
      const int kap = (kn < n - c) ? kn : (n - c);
      span_weights(t, n - kap, n, n, w);
      for (int k = 0; k < MM; ++k) {
        Cx<T> al = old_less(c, k), ag = old_great(c, k);
        for (int p = 0; p <= kap; ++p) {
          const int j = n - kap + p;
          al = al + scale(T(w[p]), ring.at(j, 0, c, k / M, k % M));
          ag = ag + scale(T(w[p]), ring.at(j, 1, c, k / M, k % M));
        }
        Gl[c * MM + k] = al; Gg[c * MM + k] = ag;
      }
    }
    {
      const int kap = (kn < n) ? kn : n;
      span_weights(t, n - kap, n, n, w);
      for (int k = 0; k < MM; ++k) {
        Cx<T> al = L[tri(n - 1, n - 1) * MM + k];
        for (int p = 0; p <= kap; ++p) al = al + scale(T(w[p]), diag_D(n - kap + p, k / M, k % M));
        Gl[n * MM + k] = al;
      }
    }
    commit();
  }
  if (I_last) for (size_t k = 0; k < I.size(); ++k) I_last[k] = I[k];
}

template <class T>
std::vector<T> local_U4(int M, const T* U) {
  std::vector<T> U4((size_t)M * M * M * M, T(0.0));
  for (int a = 0; a < M; ++a) U4[((a * M + a) * M + a) * M + a] = U[a];
  return U4;
}


// ------------------------------------------------- adaptive time stepping --
// Sec. 3.1: variable-step, variable-order Adams methods (orders q = 1..12)
// on the growing grid, written in integral form.  With derivative data
// f_j at the grid points,
//   predictor  y_n(0) = y_{n-1} + int_{t_{n-1}}^{t_n} P,  P interpolating f at t_{n-1..n-q},
//   corrector  y_n    = y_{n-1} + int_{t_{n-1}}^{t_n} Q,  Q interpolating f at t_{n..n-q+1},
// which is the polynomial pair pi_{n-1}, pi_n of Eq. (predictor) and
// Eq. (corrector) (the Nordsieck array represents the same polynomials).
// The state of step n is row n: G^<(t_n,t_c) for c <= n (the diagonal
// evolves with D = F^< - F^<^+) and G^>(t_n,t_c) for c < n.  The component
// of column c = n-1 starts from the diagonal value G(t_{n-1},t_{n-1}), and
// its derivative data at t_j < t_c are the right-hand sides of Eq. (KBE2)
// at points above the diagonal, evaluated once row c is accepted (the
// history reconstruction of Sec. 3.1 and Sec. 4).
//   Fixed point: y(m) = corrector with f(t_n, y(m-1)); stop when
//     R ||y(m) - y(m-1)||_wrms < 0.1 / |C|   (R = max(0.3 R, ratio), R = 1 at m = 1),
//     at most 3 iterations, divergence when the change more than doubles.
//   Local error: LTE = C (y_n - y_n(0)), C = E_c / (E_p - E_c) with the
//     error integrals E_p = int prod_{i=1..q} (t - t_{n-i}), E_c = int prod_{i=0..q-1} (t - t_{n-i})
//     (Milne's device); the step passes when ||LTE||_wrms <= 1.
//   Weights: w_j = 1 / (rtol |y_{n-1,j}| + atol), complex modulus, N complex components.
//   Orders q-1 and q+1 (Sec. 3.1; considered after q+1 steps at order q):
//     LTE(q') = int prod_{i=0..q'-1} (t - t_{n-i}) * f[t_n, ..., t_{n-q'}]  (divided difference).
//   Step factors eta = 1 / ((b ||LTE||)^{1/(q'+1)} + 1e-6), b = 6 (q-1, q), 10 (q+1); the
//   largest wins (ties keep q); eta < 1.5 keeps h; growth at most 1e4 on the first step,
//   10 later and none right after a failed attempt.  Error-test failure: h *= max(0.1,
//   min(0.9, eta_q)); from the third failure of a step on, q = 1 and h *= 0.1.
//   Convergence failure: h *= 0.25.
struct CtlOpts {
  double rtol, atol, h0, h_max, t_end;
  int q_max, k_hist, K_sel, n_max;
  // replay: take exactly the points t_force[1..n_force-1] with the orders
  // q_force[n] (no error test, no step selection; the fixed-point iteration
  // and everything else as above)
  const double* t_force = nullptr;
  const int* q_force = nullptr;
  int n_force = 0;
};

// integral over [t_{n-1}, t_n] of prod_{i in nodes} (t - t_i)
double node_poly_integral(const double* t, int n, const int* nodes, int cnt) {
  const int q = 12;
  double gx[q], gw[q];
  gauss_legendre(q, gx, gw);
  const double lo = t[n - 1], hi = t[n], mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
  double s = 0.0;
  for (int g = 0; g < q; ++g) {
    const double x = mid + half * gx[g];
    double p = 1.0;
    for (int i = 0; i < cnt; ++i) p *= x - t[nodes[i]];
    s += gw[g] * p;
  }
  return half * s;
}

// Milne constant C = E_c / (E_p - E_c) of the order-q pair at step n.
double milne_constant(const double* t, int n, int q) {
  int np[13], nc[13];
  for (int i = 1; i <= q; ++i) np[i - 1] = n - i;
  for (int i = 0; i < q; ++i) nc[i] = n - i;
  const double Ep = node_poly_integral(t, n, np, q), Ec = node_poly_integral(t, n, nc, q);
  return Ec / (Ep - Ec);
}

struct CtlState {
  int M;
  std::vector<double> t;
  std::vector<int> korder, qused;
  C64* L;
  C64* R;
  std::vector<std::vector<C64>> Fb;                 // row j: [2][j+1][M*M]
  std::vector<std::map<int, std::vector<C64>>> Fa;  // row j: column c > j -> [2][M*M]
  std::vector<std::vector<C64>> Sl, Sg;             // self-energy rows of accepted rows
  int nfev = 0, nrecon = 0;
  C64 F(int s, int j, int c, int a, int b) const {
    const int MM = M * M;
    if (c <= j) return Fb[j][((size_t)s * (j + 1) + c) * MM + a * M + b];
    return Fa[j].at(c)[(size_t)s * MM + a * M + b];
  }
  // derivative of the component (s, c) of the row-n state at t_j
  C64 deriv(int s, int j, int c, int n, int a, int b) const {
    if (s == 0 && c == n) return F(0, j, j, a, b) - conj(F(0, j, j, b, a));  // diagonal: D(j)
    return F(s, j, c, a, b);
  }
};

// Value of component (s, c) of row r (c <= r; the greater diagonal is fixed).
inline C64 comp_value(const Plane<double>& G, int s, int r, int c, int a, int b) {
  return s == 0 ? G.less(r, c, a, b) : G.great(r, c, a, b);
}

// Eq. (KBE2) right-hand side at the point (t_j, t_c) above the diagonal
// (j < c, rows up to c accepted):
//   I^s(j,c) = sum_{m<=j} w_{j,m} Sigma^R(j,m) G^s(m,c) + sum_{m<=c} w_{c,m} Sigma^s(j,m) G^A(m,c),
//   F^s(j,c) = -i (eps(t_j) G^s(j,c) + I^s(j,c)),
// with Sigma^s(j,m) = -Sigma^s(m,j)^+ for m > j.
void rhs_above(const Model<double>& md, const Plane<double>& G, CtlState& st, int j, int c, C64* out) {
  const int M = st.M, MM = M * M;
  std::vector<double> wj(j + 1), wc(c + 1);
  composite_row(st.t.data(), st.korder.data(), j, wj.data());
  composite_row(st.t.data(), st.korder.data(), c, wc.data());
  auto sig = [&](int s, int r, int m, int a, int b) -> C64 {  // Sigma^s(t_r, t_m)
    const auto& S = s == 0 ? st.Sl : st.Sg;
    if (m <= r) return S[r][(size_t)m * MM + a * M + b];
    return -conj(S[m][(size_t)r * MM + b * M + a]);
  };
  std::vector<C64> eps(MM);
  fock(md, st.t[j], G.L + tri(j, j) * MM, eps.data());
  for (int s = 0; s < 2; ++s)
    for (int a = 0; a < M; ++a)
      for (int b = 0; b < M; ++b) {
        Acc<double> acc;
        for (int m = 0; m <= j; ++m)
          for (int x = 0; x < M; ++x)
            acc.add(scale(wj[m], (sig(1, j, m, a, x) - sig(0, j, m, a, x)) * G.get(s, m, c, x, b)));
        for (int m = 0; m <= c; ++m)
          for (int x = 0; x < M; ++x) acc.add(scale(wc[m], sig(s, j, m, a, x) * G.adv(m, c, x, b)));
        C64 v = acc.get();
        for (int x = 0; x < M; ++x) v = v + eps[a * M + x] * G.get(s, j, c, x, b);
        out[(size_t)s * MM + a * M + b] = mul_mi(v);
      }
  ++st.nrecon;
}

// WRMS norm over the components of row n of v(s, c, a, b) with weights
// w(s, c, a, b): lesser c <= n, greater c < n; N = (2n+1) M^2 complex entries.
template <class Fn, class Wn>
double wrms(int M, int n, Fn v, Wn w) {
  double s = 0.0;
  for (int sc = 0; sc < 2; ++sc)
    for (int c = 0; c <= n - sc; ++c)
      for (int a = 0; a < M; ++a)
        for (int b = 0; b < M; ++b) {
          const C64 x = v(sc, c, a, b);
          const double ww = w(sc, c, a, b);
          s += (x.re * x.re + x.im * x.im) * ww * ww;
        }
  return std::sqrt(s / ((2.0 * n + 1.0) * M * M));
}

// Returns 0 on success (t_end reached), 1 when n_max rows are full first,
// 2 when a step fails too often.
int run_controlled(const Model<double>& md, const double* U4, const CtlOpts& o, CtlState& st, int* n_out,
                   int* stats) {
  const int M = md.M, MM = M * M;
  Plane<double> G{M, st.L, st.R};
  auto f_eval = [&](int n) {
    std::vector<C64> Sl((n + 1) * MM), Sg((n + 1) * MM), I(2 * (n + 1) * MM);
    sigma_row(G, U4, n, Sl.data(), Sg.data());
    SigmaRow<double> S{M, Sl.data(), Sg.data()};
    if (o.K_sel > 0 && n > 0) st.korder[n] = select_history_order(G, S, st.t.data(), n, o.K_sel);
    history_slice(G, S, st.t.data(), st.korder.data(), n, I.data(), 1);
    st.Fb[n].assign(2 * (n + 1) * MM, C64());
    rhs_row(md, G, st.t.data(), I.data(), n, st.Fb[n].data());
    ++st.nfev;
  };
  auto store_sigma = [&](int n) {
    st.Sl[n].assign((n + 1) * MM, C64());
    st.Sg[n].assign((n + 1) * MM, C64());
    sigma_row(G, U4, n, st.Sl[n].data(), st.Sg[n].data());
  };
  auto finish = [&](int n, int n_err, int n_conv, int rc) {
    *n_out = n;
    stats[0] = n - 1; stats[1] = n_err; stats[2] = n_conv; stats[3] = st.nfev;
    return rc;
  };
  st.korder[0] = 0;
  f_eval(0);
  store_sigma(0);
  double h = o.h0, eta_max = 1e4;
  int q = 1, qsteps = 0, n = 1, n_err = 0, n_conv = 0;
  std::vector<C64> ypred, yprev, ycur, ynew;
  double wp[16], wc[16];
  const bool replay = o.t_force != nullptr;
  while (replay ? n < o.n_force : st.t[n - 1] < o.t_end * (1.0 - 1e-14)) {
    if (n >= o.n_max) return finish(n, n_err, n_conv, 1);
    int nef = 0, ncf = 0;
    bool failed = false;
    double E = 0.0, Cm = 0.0;
    for (;;) {  // attempts of step n
      if (o.h_max > 0.0 && h > o.h_max) h = o.h_max;
      if (st.t[n - 1] + h > o.t_end) h = o.t_end - st.t[n - 1];
      if (q > n) q = n;
      st.t[n] = st.t[n - 1] + h;
      if (replay) { st.t[n] = o.t_force[n]; q = o.q_force[n]; }
      st.korder[n] = o.k_hist;
      span_weights(st.t.data(), n - q, n - 1, n, wp);      // nodes t_{n-q} .. t_{n-1}
      span_weights(st.t.data(), n - q + 1, n, n, wc);      // nodes t_{n-q+1} .. t_n
      Cm = milne_constant(st.t.data(), n, q);
      const size_t cnt = (size_t)2 * (n + 1) * MM;          // [s][c][a][b], c <= n
      ypred.assign(cnt, C64()); yprev.assign(cnt, C64());
      auto at = [&](int s, int c, int a, int b) { return (((size_t)s * (n + 1) + c) * M + a) * M + b; };
      for (int s = 0; s < 2; ++s)
        for (int c = 0; c <= n - s; ++c)
          for (int a = 0; a < M; ++a)
            for (int b = 0; b < M; ++b) {
              // previous value from row n-1; column n-1 and the diagonal start from G(t_{n-1},t_{n-1})
              const C64 y0 = comp_value(G, s, n - 1, std::min(c, n - 1), a, b);
              C64 y = y0;
              for (int i = 0; i < q; ++i) y = y + scale(wp[i], st.deriv(s, n - q + i, c, n, a, b));
              yprev[at(s, c, a, b)] = y0;
              ypred[at(s, c, a, b)] = y;
            }
      auto weight = [&](int s, int c, int a, int b) {
        const C64 y = yprev[at(s, c, a, b)];
        return 1.0 / (o.rtol * std::sqrt(y.re * y.re + y.im * y.im) + o.atol);
      };
      auto commit = [&](const std::vector<C64>& y) {
        for (int c = 0; c <= n; ++c)
          for (int k = 0; k < MM; ++k) {
            const C64 l = y[at(0, c, k / M, k % M)];
            st.L[tri(n, c) * MM + k] = l;
            if (c < n) st.R[tri(n, c) * MM + k] = y[at(1, c, k / M, k % M)] - l;
            else st.R[tri(n, c) * MM + k] = (k / M == k % M) ? C64(0.0, -1.0) : C64();
          }
      };
      commit(ypred);
      ycur = ypred;
      bool conv = false;
      double Rr = 1.0, dprev = 0.0;
      for (int m = 1; m <= 3; ++m) {
        f_eval(n);
        ynew.assign(cnt, C64());
        for (int s = 0; s < 2; ++s)
          for (int c = 0; c <= n - s; ++c)
            for (int a = 0; a < M; ++a)
              for (int b = 0; b < M; ++b) {
                C64 y = yprev[at(s, c, a, b)];
                for (int i = 0; i < q; ++i) y = y + scale(wc[i], st.deriv(s, n - q + 1 + i, c, n, a, b));
                ynew[at(s, c, a, b)] = y;
              }
        const double d = wrms(M, n, [&](int s, int c, int a, int b) {
          return ynew[at(s, c, a, b)] - ycur[at(s, c, a, b)]; }, weight);
        if (m > 1) Rr = std::max(0.3 * Rr, d / dprev);
        commit(ynew);
        ycur = ynew;
        if (Rr * d * std::fabs(Cm) < 0.1) { conv = true; break; }
        if (m > 1 && d > 2.0 * dprev) break;
        dprev = d;
      }
      if (!conv && replay) return finish(n, n_err, n_conv, 2);
      if (!conv) {
        ++n_conv; ++ncf; failed = true;
        if (ncf > 10) return finish(n, n_err, n_conv, 2);
        h *= 0.25;
        continue;
      }
      E = std::fabs(Cm) * wrms(M, n, [&](int s, int c, int a, int b) {
        return ycur[at(s, c, a, b)] - ypred[at(s, c, a, b)]; }, weight);
      if (E > 1.0 && !replay) {
        ++n_err; ++nef; failed = true;
        if (nef > 7) return finish(n, n_err, n_conv, 2);
        if (nef >= 3) { q = 1; qsteps = 0; h *= 0.1; continue; }
        const double eta = 1.0 / (std::pow(6.0 * E, 1.0 / (q + 1)) + 1e-6);
        h *= std::max(0.1, std::min(0.9, eta));
        continue;
      }
      break;
    }
    // accepted: self-energy of the accepted row, then the derivative data of
    // column n above the diagonal
    st.qused[n] = q;
    store_sigma(n);
    const int jlo = std::max(0, n - std::min(q + 1, 12));
    for (int j = jlo; j < n; ++j) {
      std::vector<C64> blk(2 * MM);
      rhs_above(md, G, st, j, n, blk.data());
      st.Fa[j][n] = blk;
    }
    if (replay) { ++n; continue; }
    // next step size and order
    ++qsteps;
    const double addon = 1e-6;
    double eta = E > 0.0 ? 1.0 / (std::pow(6.0 * E, 1.0 / (q + 1)) + addon) : eta_max;
    int qn = q;
    if (qsteps > q) {
      auto divdiff_est = [&](int qq) {  // |int prod_{i<qq} (t - t_{n-i})| * ||f[t_n .. t_{n-qq}]||
        int nodes[14];
        for (int i = 0; i < qq; ++i) nodes[i] = n - i;
        const double P = std::fabs(node_poly_integral(st.t.data(), n, nodes, qq));
        double alpha[14];
        for (int i = 0; i <= qq; ++i) {
          double d = 1.0;
          for (int k = 0; k <= qq; ++k)
            if (k != i) d *= st.t[n - i] - st.t[n - k];
          alpha[i] = 1.0 / d;
        }
        auto w = [&](int s, int c, int a, int b) {
          const C64 y = yprev[(((size_t)s * (n + 1) + c) * M + a) * M + b];
          return 1.0 / (o.rtol * std::sqrt(y.re * y.re + y.im * y.im) + o.atol);
        };
        return P * wrms(M, n, [&](int s, int c, int a, int b) {
          C64 v;
          for (int i = 0; i <= qq; ++i) v = v + scale(alpha[i], st.deriv(s, n - i, c, n, a, b));
          return v; }, w);
      };
      if (q > 1) {
        const double Eq = divdiff_est(q - 1);
        const double e2 = Eq > 0.0 ? 1.0 / (std::pow(6.0 * Eq, 1.0 / q) + addon) : eta_max;
        if (e2 > eta) { eta = e2; qn = q - 1; }
      }
      if (q < o.q_max && n - q - 1 >= 0) {
        const double Eq = divdiff_est(q + 1);
        const double e2 = Eq > 0.0 ? 1.0 / (std::pow(10.0 * Eq, 1.0 / (q + 2)) + addon) : eta_max;
        if (e2 > eta) { eta = e2; qn = q + 1; }
      }
    }
    if (qn != q) { q = qn; qsteps = 0; }
    if (eta < 1.5) eta = 1.0;
    else eta = std::min(eta, failed ? 1.0 : eta_max);
    h *= eta;
    eta_max = 10.0;
    ++n;
  }
  return finish(n, n_err, n_conv, 0);
}


// ------------------------------------------------------- thermal branch --
// Sec. 2: with a thermal branch the mixed component G^|(t,tau) joins the
// state (Eq. KBE3) and Eq. (KBE2) gains the term -i int_0^beta dtau
// Sigma^|(t,tau) G^|-(tau,t').  Conventions (fermions):
//   G^M(tau), tau in (0, beta), antiperiodic: G^M(tau - beta) = -G^M(tau);
//   G^|-(tau, t) = [G^|(t, beta - tau)]^+;   G^|(0, tau) = -i G^M(beta - tau);
//   Sigma^|(t,tau)_ij = U_ifde UEx_jabc G^|_fb(t,tau) G^|_ea(t,tau) G^|-_cd(tau,t)  (Eq. SE);
//   i d/dt G^|(t,tau) = eps(t) G^|(t,tau) + int_0^t Sigma^R(t,s) G^|(s,tau) ds
//                       + int_0^beta Sigma^|(t,s) G^M(s - tau) ds          (Eq. KBE3).
// tau grid: tau_k = k beta / (N-1).  An integral over [0, tau_j] sums, per
// interval [tau_{l-1}, tau_l], the integral of the interpolant of degree
// kap = min(ktau, j) (Eq. weights) through kap+1 consecutive nodes that
// contain the interval, centred on it where possible and kept inside
// [0, tau_j] (all tau points exist at once, unlike the past-only stencils in
// t); integrals over [tau_j, beta] use the mirrored rule.  The Matsubara
// convolution is split at s = tau_j, where G^M(s - tau) jumps.
struct TauGrid {
  int N, ktau;
  double beta;
  std::vector<double> tau;
  std::vector<std::vector<double>> left;  // [j][k], k <= j: int_0^{tau_j}
  void build() {
    tau.resize(N);
    for (int k = 0; k < N; ++k) tau[k] = beta * k / (N - 1);
    left.resize(N);
    double w[64];
    for (int j = 0; j < N; ++j) {
      left[j].assign(j + 1, 0.0);
      const int kap = ktau < j ? ktau : j;
      for (int l = 1; l <= j; ++l) {
        int s0 = l - 1 - (kap - 1) / 2;
        if (s0 > j - kap) s0 = j - kap;
        if (s0 < 0) s0 = 0;
        lagrange_weights(tau.data() + s0, kap, tau[l - 1], tau[l], w);
        for (int i = 0; i <= kap; ++i) left[j][s0 + i] += w[i];
      }
    }
  }
  double full(int k) const { return left[N - 1][k]; }                 // int_0^beta
  double right(int j, int k) const { return left[N - 1 - j][N - 1 - k]; }  // int_{tau_j}^beta, k >= j
};

struct Mixed {
  int M, N;
  C64* G;  // [rows][N][M][M]
  C64 at(int r, int k, int a, int b) const { return G[(((int64_t)r * N + k) * M + a) * M + b]; }
  C64 adj(int k, int r, int a, int b) const { return conj(at(r, N - 1 - k, b, a)); }  // G^|-(tau_k, t_r)
};

// Sigma^|(t_n, tau_k), k = 0..N-1, for the tensor U4; out [N][M][M].
void sigma_mixed(const Mixed& X, const double* U4, int n, C64* out) {
  const int M = X.M, N = X.N;
  auto at = [M](int a, int b, int c, int d) { return ((a * M + b) * M + c) * M + d; };
  struct E { int i, f, d, e; double u; };
  std::vector<E> nzU, nzX;
  for (int i = 0; i < M; ++i)
    for (int f = 0; f < M; ++f)
      for (int d = 0; d < M; ++d)
        for (int e = 0; e < M; ++e) {
          const double u = U4[at(i, f, d, e)];
          const double ux = 2.0 * U4[at(i, d, f, e)] - U4[at(i, f, d, e)];
          if (u != 0.0) nzU.push_back({i, f, d, e, u});
          if (ux != 0.0) nzX.push_back({i, f, d, e, ux});
        }
  for (int k = 0; k < N; ++k) {
    C64* o = out + (size_t)k * M * M;
    for (int q = 0; q < M * M; ++q) o[q] = C64();
    for (const E& p : nzU)
      for (const E& q : nzX) {
        const C64 g = X.at(n, k, p.f, q.d) * X.at(n, k, p.e, q.f) * X.adj(k, n, q.e, p.d);
        o[p.i * M + q.i] = o[p.i * M + q.i] + scale(p.u * q.u, g);
      }
  }
}

// Right-hand side of Eq. (KBE3) for row n: F^|(n, j) = -i (eps G^|(n,j) + I^|(n,j)); out [N][M][M].
void rhs_mixed(const Model<double>& md, const Plane<double>& G, const Mixed& X, const TauGrid& tg,
               const double* t, const int* order, const SigmaRow<double>& S, const C64* Smix, const C64* GM, int n,
               C64* out) {
  const int M = md.M, N = tg.N, MM = M * M;
  std::vector<double> wn(n + 1);
  composite_row(t, order, n, wn.data());
  std::vector<C64> eps(MM);
  fock(md, t[n], G.L + tri(n, n) * MM, eps.data());
  for (int j = 0; j < N; ++j)
    for (int a = 0; a < M; ++a)
      for (int b = 0; b < M; ++b) {
        Acc<double> acc;
        for (int m = 0; m <= n; ++m)
          for (int x = 0; x < M; ++x) acc.add(scale(wn[m], S.ret_nm(m, a, x) * X.at(m, j, x, b)));
        for (int k = 0; k <= j; ++k)  // G^M(tau_k - tau_j) = -G^M(beta + tau_k - tau_j)
          for (int x = 0; x < M; ++x)
            acc.add(scale(-tg.left[j][k], Smix[(size_t)k * MM + a * M + x] * GM[(size_t)(N - 1 + k - j) * MM + x * M + b]));
        for (int k = j; k < N; ++k)
          for (int x = 0; x < M; ++x)
            acc.add(scale(tg.right(j, k), Smix[(size_t)k * MM + a * M + x] * GM[(size_t)(k - j) * MM + x * M + b]));
        C64 v = acc.get();
        for (int x = 0; x < M; ++x) v = v + eps[a * M + x] * X.at(n, j, x, b);
        out[((size_t)j * M + a) * M + b] = mul_mi(v);
      }
}

// The KBE2 mixed term of row n, -i sum_k w_k Sigma^|(n,k) G^|-(tau_k, t_c), added to both
// history integrals I^s(n,c), c = 0..n (layout [s][c][a][b]).
void add_mixed_term(const Mixed& X, const TauGrid& tg, const C64* Smix, int n, C64* I) {
  const int M = X.M, MM = M * M, N = tg.N;
  for (int c = 0; c <= n; ++c)
    for (int a = 0; a < M; ++a)
      for (int b = 0; b < M; ++b) {
        Acc<double> acc;
        for (int k = 0; k < N; ++k)
          for (int x = 0; x < M; ++x) acc.add(scale(tg.full(k), Smix[(size_t)k * MM + a * M + x] * X.adj(k, c, x, b)));
        const C64 v = mul_mi(acc.get());
        for (int s = 0; s < 2; ++s) {
          C64& o = I[(((size_t)s * (n + 1) + c) * M + a) * M + b];
          o = o + v;
        }
      }
}

// Right-hand sides of row j with the thermal terms: F [2][j+1][M][M], Fmix [N][M][M].
void thermal_rhs(const Model<double>& md, const double* U4, const Plane<double>& G, const Mixed& X,
                 const TauGrid& tg, const C64* GM, const double* t, const int* order, int j, C64* F, C64* Fmix,
                 int nthreads) {
  const int M = md.M, MM = M * M;
  std::vector<C64> Sl((j + 1) * MM), Sg((j + 1) * MM), I(2 * (j + 1) * MM), Smix((size_t)tg.N * MM);
  sigma_row(G, U4, j, Sl.data(), Sg.data());
  sigma_mixed(X, U4, j, Smix.data());
  SigmaRow<double> S{M, Sl.data(), Sg.data()};
  history_slice(G, S, t, order, j, I.data(), nthreads);
  add_mixed_term(X, tg, Smix.data(), j, I.data());
  rhs_row(md, G, t, I.data(), j, F);
  rhs_mixed(md, G, X, tg, t, order, S, Smix.data(), GM, j, Fmix);
}

// Integral-form Adams stepper (the structure of kbe_step, P sweeps) with the
// thermal branch: rows n = 1 .. n_t-1 of L, R and G^|.  Row 0 and G^|(0, .)
// are set by the caller.
void run_thermal(const Model<double>& md, const double* U4, const TauGrid& tg, const C64* GM, const double* t,
                 const int* order, int n_t, int P, C64* L, C64* R, C64* Gm, int nthreads) {
  const int M = md.M, MM = M * M, N = tg.N;
  Plane<double> G{M, L, R};
  Mixed X{M, N, Gm};
  std::vector<std::vector<C64>> F(n_t), Fm(n_t);
  F[0].resize(2 * MM);
  Fm[0].resize((size_t)N * MM);
  thermal_rhs(md, U4, G, X, tg, GM, t, order, 0, F[0].data(), Fm[0].data(), nthreads);
  auto Fat = [&](int j, int s, int c, int k) { return F[j][((size_t)s * (j + 1) + c) * MM + k]; };
  auto D = [&](int j, int a, int b) { return Fat(j, 0, j, a * M + b) - conj(Fat(j, 0, j, b * M + a)); };
  double w[64];
  for (int n = 1; n < n_t; ++n) {
    const int kn = order[n];
    std::vector<C64> Gl((n + 1) * MM), Gg((n + 1) * MM), Gx((size_t)N * MM);
    auto step_rows = [&](bool corr) {
      for (int c = 0; c < n; ++c) {
        const int q = std::min(kn, n - c);
        if (corr) span_weights(t, n - q, n, n, w); else span_weights(t, n - q, n - 1, n, w);
        const int cnt = corr ? q + 1 : q;
        for (int k = 0; k < MM; ++k) {
          C64 al = L[tri(n - 1, c) * MM + k], ag = R[tri(n - 1, c) * MM + k] + L[tri(n - 1, c) * MM + k];
          for (int p = 0; p < cnt; ++p) {
            al = al + scale(w[p], Fat(n - q + p, 0, c, k));
            ag = ag + scale(w[p], Fat(n - q + p, 1, c, k));
          }
          Gl[c * MM + k] = al; Gg[c * MM + k] = ag;
        }
      }
      const int q = std::min(kn, n);
      if (corr) span_weights(t, n - q, n, n, w); else span_weights(t, n - q, n - 1, n, w);
      const int cnt = corr ? q + 1 : q;
      for (int k = 0; k < MM; ++k) {
        C64 al = L[tri(n - 1, n - 1) * MM + k];
        for (int p = 0; p < cnt; ++p) al = al + scale(w[p], D(n - q + p, k / M, k % M));
        Gl[n * MM + k] = al;
      }
      for (size_t k = 0; k < (size_t)N * MM; ++k) {  // mixed row: the full history in t
        C64 x = Gm[(size_t)(n - 1) * N * MM + k];
        for (int p = 0; p < cnt; ++p) x = x + scale(w[p], Fm[n - q + p][k]);
        Gx[k] = x;
      }
      for (int c = 0; c < n; ++c)
        for (int k = 0; k < MM; ++k) {
          L[tri(n, c) * MM + k] = Gl[c * MM + k];
          R[tri(n, c) * MM + k] = Gg[c * MM + k] - Gl[c * MM + k];
        }
      for (int k = 0; k < MM; ++k) {
        L[tri(n, n) * MM + k] = Gl[n * MM + k];
        R[tri(n, n) * MM + k] = (k / M == k % M) ? C64(0.0, -1.0) : C64();
      }
      for (size_t k = 0; k < (size_t)N * MM; ++k) Gm[(size_t)n * N * MM + k] = Gx[k];
    };
    step_rows(false);
    F[n].resize(2 * (n + 1) * MM);
    Fm[n].resize((size_t)N * MM);
    for (int sweep = 0; sweep < P; ++sweep) {
      thermal_rhs(md, U4, G, X, tg, GM, t, order, n, F[n].data(), Fm[n].data(), nthreads);
      step_rows(true);
    }
  }
}
}  // namespace

// =================================================================== C ABI ==
extern "C" {

int orc_version() { return 1; }

int orc_threads_available() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Gauss-Legendre rule on [-1,1].
int orc_gauss_legendre(int q, double* x, double* w) {
  if (q < 1 || q > 64) return 1;
  gauss_legendre(q, x, w);
  return 0;
}

// Weights of the interpolatory rule on nodes tau[0..k] over [lo, hi].
int orc_lagrange_weights(const double* tau, int k, double lo, double hi, double* w) {
  if (k < 0 || k > 40) return 1;
  lagrange_weights(tau, k, lo, hi, w);
  return 0;
}

// Composite weight row w_{n,0..n}.
int orc_composite_row(const double* t, const int* order, int n, double* row) {
  if (n < 0) return 1;
  composite_row(t, order, n, row);
  return 0;
}

// Self-energy row n of Eq. (SE) for a general four-index tensor U4[M^4].
int orc_sigma_row(int M, int n, const double* U4, const void* L, const void* R, void* Sl, void* Sg) {
  if (M < 1 || n < 0) return 1;
  Plane<double> G{M, (const C64*)L, (const C64*)R};
  sigma_row(G, U4, n, (C64*)Sl, (C64*)Sg);
  return 0;
}

// History slice of Eq. (KBE2) for row n; out [2][n+1][M][M].
int orc_history_slice(int M, int n, const double* t, const int* order, const void* L, const void* R,
                      const void* Sl, const void* Sg, void* out, int nthreads) {
  if (M < 1 || n < 0 || nthreads < 1) return 1;
  Plane<double> G{M, (const C64*)L, (const C64*)R};
  SigmaRow<double> S{M, (const C64*)Sl, (const C64*)Sg};
  history_slice(G, S, t, order, n, (C64*)out, nthreads);
  return 0;
}

// History slice restricted to the output columns listed in cols (both s);
// out [2][ncols][M][M].  Used to time bounded samples of a slice.
int orc_history_columns(int M, int n, const double* t, const int* order, const void* L, const void* R,
                        const void* Sl, const void* Sg, const int* cols, int ncols, void* out, int nthreads) {
  if (M < 1 || n < 0 || nthreads < 1 || ncols < 0) return 1;
  Plane<double> G{M, (const C64*)L, (const C64*)R};
  SigmaRow<double> S{M, (const C64*)Sl, (const C64*)Sg};
  std::vector<double> wn(n + 1);
  composite_row(t, order, n, wn.data());
  C64* o = (C64*)out;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) collapse(2)
  for (int s = 0; s < 2; ++s)
    for (int ic = 0; ic < ncols; ++ic) {
      const int c = cols[ic];
      std::vector<double> wc(c + 1);
      composite_row(t, order, c, wc.data());
      for (int a = 0; a < M; ++a)
        for (int b = 0; b < M; ++b) {
          Acc<double> acc;
          for (int m = 0; m <= n; ++m)
            for (int x = 0; x < M; ++x) acc.add(scale(wn[m], S.ret_nm(m, a, x) * G.get(s, m, c, x, b)));
          for (int m = 0; m <= c; ++m)
            for (int x = 0; x < M; ++x) acc.add(scale(wc[m], S.s_nm(s, m, a, x) * G.adv(m, c, x, b)));
          o[(((int64_t)s * ncols + ic) * M + a) * M + b] = acc.get();
        }
    }
  return 0;
}

// Eq. (KBE1) lesser history integrals at (t_c, t_n), c = 0..n; out [n+1][M][M].
int orc_kbe1_slice(int M, int n, const double* t, const int* order, const void* L, const void* R,
                   const void* Sl, const void* Sg, void* out, int nthreads) {
  if (M < 1 || n < 0 || nthreads < 1) return 1;
  Plane<double> G{M, (const C64*)L, (const C64*)R};
  SigmaRow<double> S{M, (const C64*)Sl, (const C64*)Sg};
  kbe1_slice(G, S, t, order, n, (C64*)out, nthreads);
  return 0;
}

// Right-hand-side row j (history reconstruction): needs rows 0..j stored and
// the self-energy from them.  F out [2][j+1][M][M].
int orc_rhs_row(int M, int j, const double* t, const int* order, const double* h0, const double* U,
                const double* v, const double* pulse4, const void* L, const void* R, void* F, int nthreads) {
  if (M < 1 || j < 0 || nthreads < 1) return 1;
  Model<double> md{M, (const C64*)h0, U, v, pulse4[0], pulse4[1], pulse4[2], pulse4[3]};
  Plane<double> G{M, (const C64*)L, (const C64*)R};
  std::vector<double> U4 = local_U4(M, U);
  std::vector<C64> Sl((j + 1) * M * M), Sg((j + 1) * M * M), I(2 * (j + 1) * M * M);
  sigma_row(G, U4.data(), j, Sl.data(), Sg.data());
  SigmaRow<double> S{M, Sl.data(), Sg.data()};
  history_slice(G, S, t, order, j, I.data(), nthreads);
  rhs_row(md, G, t, I.data(), j, (C64*)F);
  return 0;
}

// Run KBE steps n = n_start .. n_end-1 (n_start >= 1).  L, R hold rows
// 0..n_start-1 on entry and rows up to n_end-1 on exit (triangles of n_end
// rows).  F_in holds the right-hand-side rows j = max(0, n_start-K)
// .. n_start-1, packed one after the other, each [2][j+1][M][M]; K is the
// largest order on the grid orders[1..n_end-1].  I_last (optional) receives the last history
// row [2][n_end][M][M].
int orc_run(int M, int n_start, int n_end, const double* t, const int* order, const double* h0,
            const double* U, const double* v, const double* pulse4, int P, void* L, void* R,
            const void* F_in, void* I_last, int nthreads) {
  if (M < 1 || n_start < 1 || n_end < n_start || P < 1 || nthreads < 1) return 1;
  int K = 1;
  for (int l = 1; l < n_end; ++l) if (order[l] > K) K = order[l];
  Model<double> md{M, (const C64*)h0, U, v, pulse4[0], pulse4[1], pulse4[2], pulse4[3]};
  std::vector<double> U4 = local_U4(M, U);
  Ring<double> ring{M, n_end, K, std::vector<C64>((size_t)(K + 1) * 2 * n_end * M * M)};
  const C64* f = (const C64*)F_in;
  for (int j = (n_start - K > 0 ? n_start - K : 0); j <= n_start - 1; ++j) {
    const size_t cnt = (size_t)2 * (j + 1) * M * M;
    std::memcpy((void*)ring.row(j), f, cnt * sizeof(C64));
    f += cnt;
  }
  for (int n = n_start; n < n_end; ++n)
    kbe_step(md, t, order, n, P, U4.data(), (C64*)L, (C64*)R, ring,
             (n == n_end - 1) ? (C64*)I_last : nullptr, nthreads);
  return 0;
}

// The same run with adaptive history orders (Sec. 3.2): hord[1..n_start-1]
// hold the orders chosen before n_start (the history quadrature of the given
// rows); each step n chooses hord[n] with orders up to K_sel (1..12) in every
// sweep (K_sel = 0: hord[1..n_end-1] are given and used as they are).  The
// stepper's own orders stay `order`.
int orc_run_adaptive(int M, int n_start, int n_end, const double* t, const int* order, int* hord, int K_sel,
                     const double* h0, const double* U, const double* v, const double* pulse4, int P, void* L,
                     void* R, const void* F_in, void* I_last, int nthreads) {
  if (M < 1 || n_start < 1 || n_end < n_start || P < 1 || nthreads < 1 || K_sel < 0 || K_sel > 12) return 1;
  int K = 1;
  for (int l = 1; l < n_end; ++l) if (order[l] > K) K = order[l];
  Model<double> md{M, (const C64*)h0, U, v, pulse4[0], pulse4[1], pulse4[2], pulse4[3]};
  std::vector<double> U4 = local_U4(M, U);
  Ring<double> ring{M, n_end, K, std::vector<C64>((size_t)(K + 1) * 2 * n_end * M * M)};
  const C64* f = (const C64*)F_in;
  for (int j = (n_start - K > 0 ? n_start - K : 0); j <= n_start - 1; ++j) {
    const size_t cnt = (size_t)2 * (j + 1) * M * M;
    std::memcpy((void*)ring.row(j), f, cnt * sizeof(C64));
    f += cnt;
  }
  for (int n = n_start; n < n_end; ++n)
    kbe_step(md, t, order, n, P, U4.data(), (C64*)L, (C64*)R, ring,
             (n == n_end - 1) ? (C64*)I_last : nullptr, nthreads, hord, K_sel);
  return 0;
}

// Order selection from given test-integrand values u [kmax+1][M][M] at
// t_{n-kmax} .. t_n (kmax = min(K, n)); diffs[k] = |I^(k) - I^(k-1)|_max.
int orc_choose_order(int M, int n, const double* t, int K, const void* u, double* diffs, int* kopt) {
  if (M < 1 || n < 1 || K < 1 || K > 12) return 1;
  *kopt = choose_order(t, n, K, M, (const C64*)u, diffs);
  return 0;
}

// Test integrand values u(t_l), l = n-kmax .. n, from row n of L, R and the
// self-energy row n; and the order chosen from them.
int orc_select_order(int M, int n, const double* t, int K, const void* L, const void* R, const void* Sl,
                     const void* Sg, void* u_out, int* kopt) {
  if (M < 1 || n < 1 || K < 1 || K > 12) return 1;
  Plane<double> G{M, (const C64*)L, (const C64*)R};
  SigmaRow<double> S{M, (const C64*)Sl, (const C64*)Sg};
  const int kmax = K < n ? K : n;
  for (int i = 0; i <= kmax; ++i) test_integrand(G, S, n, n - kmax + i, (C64*)u_out + (size_t)i * M * M);
  *kopt = select_history_order(G, S, t, n, K);
  return 0;
}

// Test integrand value u(t_l) for any l <= n (Sec. 3.2).
int orc_test_integrand(int M, int n, int l, const void* L, const void* R, const void* Sl, const void* Sg,
                       void* u_out) {
  if (M < 1 || n < 0 || l < 0 || l > n) return 1;
  Plane<double> G{M, (const C64*)L, (const C64*)R};
  SigmaRow<double> S{M, (const C64*)Sl, (const C64*)Sg};
  test_integrand(G, S, n, l, (C64*)u_out);
  return 0;
}

// Fock matrix of Eq. (eps) at time t from the equal-time block Lnn = G^<(t,t):
// eps [M][M].  U4 (M^4, U4[((i*M + a)*M + b)*M + j] = U_iabj) selects the
// general tensor; NULL selects the local interaction U.
int orc_fock(int M, double t, const double* h0, const double* U, const double* U4, const double* v,
             const double* pulse4, const void* Lnn, void* eps) {
  if (M < 1 || (!U && !U4)) return 1;
  Model<double> md{M, (const C64*)h0, U, v, pulse4[0], pulse4[1], pulse4[2], pulse4[3]};
  md.U4d = U4;
  fock(md, t, (const C64*)Lnn, (C64*)eps);
  return 0;
}

// Right-hand-side row j with the general tensor U4 in Eq. (SE) and Eq. (eps).
int orc_rhs_row_u4(int M, int j, const double* t, const int* order, const double* h0, const double* U4,
                   const double* v, const double* pulse4, const void* L, const void* R, void* F, int nthreads) {
  if (M < 1 || j < 0 || nthreads < 1) return 1;
  Model<double> md{M, (const C64*)h0, nullptr, v, pulse4[0], pulse4[1], pulse4[2], pulse4[3]};
  md.U4d = U4;
  Plane<double> G{M, (const C64*)L, (const C64*)R};
  std::vector<C64> Sl((j + 1) * M * M), Sg((j + 1) * M * M), I(2 * (j + 1) * M * M);
  sigma_row(G, U4, j, Sl.data(), Sg.data());
  SigmaRow<double> S{M, Sl.data(), Sg.data()};
  history_slice(G, S, t, order, j, I.data(), nthreads);
  rhs_row(md, G, t, I.data(), j, (C64*)F);
  return 0;
}

// orc_run / orc_run_adaptive with the general tensor U4 in Eq. (SE) and
// Eq. (eps).  hord = NULL: the history quadrature uses the grid's orders;
// otherwise as in orc_run_adaptive (K_sel 0..12).
int orc_run_u4(int M, int n_start, int n_end, const double* t, const int* order, int* hord, int K_sel,
               const double* h0, const double* U4, const double* v, const double* pulse4, int P, void* L, void* R,
               const void* F_in, void* I_last, int nthreads) {
  if (M < 1 || n_start < 1 || n_end < n_start || P < 1 || nthreads < 1 || K_sel < 0 || K_sel > 12) return 1;
  if (!hord && K_sel != 0) return 1;
  int K = 1;
  for (int l = 1; l < n_end; ++l) if (order[l] > K) K = order[l];
  Model<double> md{M, (const C64*)h0, nullptr, v, pulse4[0], pulse4[1], pulse4[2], pulse4[3]};
  md.U4d = U4;
  Ring<double> ring{M, n_end, K, std::vector<C64>((size_t)(K + 1) * 2 * n_end * M * M)};
  const C64* f = (const C64*)F_in;
  for (int j = (n_start - K > 0 ? n_start - K : 0); j <= n_start - 1; ++j) {
    const size_t cnt = (size_t)2 * (j + 1) * M * M;
    std::memcpy((void*)ring.row(j), f, cnt * sizeof(C64));
    f += cnt;
  }
  for (int n = n_start; n < n_end; ++n)
    kbe_step(md, t, order, n, P, U4, (C64*)L, (C64*)R, ring, (n == n_end - 1) ? (C64*)I_last : nullptr,
             nthreads, hord, K_sel);
  return 0;
}

// Adaptive time stepping (Sec. 3.1) from row 0 (L, R hold L(0,0), R(0,0)):
// opts = {rtol, atol, h0, h_max, t_end}, iopts = {q_max, k_hist, K_sel, n_max}.
// U4 = NULL selects the local interaction U.  Outputs: the triangles of the
// accepted rows (n_max rows of storage), t[0..n_max-1], q[n] (order of step
// n), korder[n] (history order of interval n), n_rows (accepted rows
// including row 0), stats = {steps, error-test failures, convergence
// failures, right-hand-side evaluations, reconstructed blocks}.
// Returns the run status (0 reached t_end, 1 storage full, 2 step failure).
// With t_force (and q_force, n_force) the run replays the given points and
// step orders instead of choosing them (rows 1..n_force-1).
int orc_run_controlled(int M, const double* opts, const int* iopts, const double* h0, const double* U,
                       const double* U4, const double* v, const double* pulse4, void* L, void* R, double* t,
                       int* q, int* korder, int* n_rows, int* stats, const double* t_force, const int* q_force,
                       int n_force) {
  if (M < 1) return -1;
  CtlOpts o{opts[0], opts[1], opts[2], opts[3], opts[4], iopts[0], iopts[1], iopts[2], iopts[3]};
  if (t_force) {
    if (!q_force || n_force < 1 || n_force > iopts[3]) return -1;
    o.t_force = t_force;
    o.q_force = q_force;
    o.n_force = n_force;
  }
  if (o.q_max < 1 || o.q_max > 12 || o.n_max < 2 || o.k_hist < 1 || o.k_hist > 12 || o.K_sel < 0 ||
      o.K_sel > 12 || !(o.h0 > 0.0) || !(o.rtol >= 0.0) || !(o.atol > 0.0))
    return -1;
  std::vector<double> U4loc;
  if (!U4) { U4loc = local_U4(M, U); U4 = U4loc.data(); }
  Model<double> md{M, (const C64*)h0, U, v, pulse4[0], pulse4[1], pulse4[2], pulse4[3]};
  if (U4loc.empty()) md.U4d = U4;
  CtlState st;
  st.M = M;
  st.t.assign(o.n_max, 0.0);
  st.korder.assign(o.n_max, 0);
  st.qused.assign(o.n_max, 0);
  st.L = (C64*)L;
  st.R = (C64*)R;
  st.Fb.resize(o.n_max);
  st.Fa.resize(o.n_max);
  st.Sl.resize(o.n_max);
  st.Sg.resize(o.n_max);
  int n_out = 0, st5[4] = {0, 0, 0, 0};
  const int rc = run_controlled(md, U4, o, st, &n_out, st5);
  for (int i = 0; i < o.n_max; ++i) { t[i] = st.t[i]; q[i] = st.qused[i]; korder[i] = st.korder[i]; }
  *n_rows = n_out;
  for (int i = 0; i < 4; ++i) stats[i] = st5[i];
  stats[4] = st.nrecon;
  return rc;
}

// Error integrals of the order-q Adams pair at step n on the nodes t:
// out = {E_p, E_c} (without the 1/q! factor) and the Milne constant.
int orc_adams_error_integrals(const double* t, int n, int q, double* out) {
  if (q < 1 || q > 12 || n < q) return 1;
  int np[13], nc[13];
  for (int i = 1; i <= q; ++i) np[i - 1] = n - i;
  for (int i = 0; i < q; ++i) nc[i] = n - i;
  out[0] = node_poly_integral(t, n, np, q);
  out[1] = node_poly_integral(t, n, nc, q);
  out[2] = milne_constant(t, n, q);
  return 0;
}

// Thermal branch (Sec. 2, Eq. KBE3): run rows 1..n_t-1 from row 0 with the
// mixed component.  tau grid of N points on [0, beta], composite weights of
// order ktau; GM [N][M][M] = G^M(tau_k) (tau_0 = 0+, tau_{N-1} = beta-);
// Gm [n_t][N][M][M] receives G^|(t_r, tau_k) (row 0 is set here to
// -i G^M(beta - tau)); L, R hold row 0 on entry.  U4 = NULL: the local U.
int orc_run_thermal(int M, int n_t, const double* t, const int* order, const double* h0, const double* U,
                    const double* U4, const double* v, const double* pulse4, int P, double beta, int N, int ktau,
                    const void* GM, void* L, void* R, void* Gm, int nthreads) {
  if (M < 1 || n_t < 1 || P < 1 || N < 2 || ktau < 1 || ktau > 12 || !(beta > 0.0)) return 1;
  std::vector<double> U4loc;
  Model<double> md{M, (const C64*)h0, U, v, pulse4[0], pulse4[1], pulse4[2], pulse4[3]};
  if (!U4) { U4loc = local_U4(M, U); U4 = U4loc.data(); } else md.U4d = U4;
  TauGrid tg{N, ktau, beta};
  tg.build();
  const C64* gm = (const C64*)GM;
  C64* X = (C64*)Gm;
  const int MM = M * M;
  for (int j = 0; j < N; ++j)
    for (int k = 0; k < MM; ++k) {
      const C64 g = gm[(size_t)(N - 1 - j) * MM + k];
      X[(size_t)j * MM + k] = C64(g.im, -g.re);  // -i G^M(beta - tau_j)
    }
  run_thermal(md, U4, tg, gm, t, order, n_t, P, (C64*)L, (C64*)R, X, nthreads);
  return 0;
}

// The split Matsubara convolution of Eq. (KBE3) alone:
// out(tau_j) = int_0^beta S(s) G^M(s - tau_j) ds on the tau grid; S, GM, out [N][M][M].
int orc_matsubara_conv(int M, int N, double beta, int ktau, const void* S, const void* GM, void* out) {
  if (M < 1 || N < 2 || ktau < 1 || ktau > 12) return 1;
  TauGrid tg{N, ktau, beta};
  tg.build();
  const C64* s = (const C64*)S;
  const C64* g = (const C64*)GM;
  C64* o = (C64*)out;
  const int MM = M * M;
  for (int j = 0; j < N; ++j)
    for (int a = 0; a < M; ++a)
      for (int b = 0; b < M; ++b) {
        Acc<double> acc;
        for (int k = 0; k <= j; ++k)
          for (int x = 0; x < M; ++x)
            acc.add(scale(-tg.left[j][k], s[(size_t)k * MM + a * M + x] * g[(size_t)(N - 1 + k - j) * MM + x * M + b]));
        for (int k = j; k < N; ++k)
          for (int x = 0; x < M; ++x)
            acc.add(scale(tg.right(j, k), s[(size_t)k * MM + a * M + x] * g[(size_t)(k - j) * MM + x * M + b]));
        o[((size_t)j * M + a) * M + b] = acc.get();
      }
  return 0;
}

// Sigma^|(t_n, tau_k) for the tensor U4 from the mixed rows Gm [rows][N][M][M].
int orc_sigma_mixed(int M, int N, int n, const double* U4, const void* Gm, void* out) {
  if (M < 1 || N < 2 || n < 0) return 1;
  Mixed X{M, N, (C64*)Gm};
  sigma_mixed(X, U4, n, (C64*)out);
  return 0;
}

// Forward-mode derivative of the same run: U_a -> U_a + eps*dU_a,
// E0 -> E0 + eps*dE0.  Rows below n_start and the given F rows are held
// fixed.  On exit Lv/Ld hold the value/derivative of the final diagonal
// block L(n_end-1, n_end-1) [M][M]; L, R receive the value triangles.
int orc_run_tangent(int M, int n_start, int n_end, const double* t, const int* order, const double* h0,
                    const double* U, const double* dU, const double* v, const double* pulse4, double dE0,
                    int P, const void* L_in, const void* R_in, const void* F_in, void* Lv, void* Ld,
                    int nthreads) {
  if (M < 1 || n_start < 1 || n_end < n_start || P < 1 || nthreads < 1) return 1;
  using D = Dual;
  int K = 1;
  for (int l = 1; l < n_end; ++l) if (order[l] > K) K = order[l];
  std::vector<D> Ud(M);
  for (int a = 0; a < M; ++a) Ud[a] = D(U[a], dU[a]);
  Model<D> md{M, (const C64*)h0, Ud.data(), v, D(pulse4[0], dE0), pulse4[1], pulse4[2], pulse4[3]};
  std::vector<D> U4 = local_U4(M, Ud.data());
  const size_t ntri = (size_t)n_end * (n_end + 1) / 2 * M * M;
  const size_t nin = (size_t)n_start * (n_start + 1) / 2 * M * M;
  std::vector<Cx<D>> L(ntri), R(ntri);
  const C64* li = (const C64*)L_in;
  const C64* ri = (const C64*)R_in;
  for (size_t k = 0; k < nin; ++k) {
    L[k] = Cx<D>(D(li[k].re), D(li[k].im));
    R[k] = Cx<D>(D(ri[k].re), D(ri[k].im));
  }
  Ring<D> ring{M, n_end, K, std::vector<Cx<D>>((size_t)(K + 1) * 2 * n_end * M * M)};
  const C64* f = (const C64*)F_in;
  for (int j = (n_start - K > 0 ? n_start - K : 0); j <= n_start - 1; ++j) {
    const size_t cnt = (size_t)2 * (j + 1) * M * M;
    Cx<D>* dst = ring.row(j);
    for (size_t k = 0; k < cnt; ++k) dst[k] = Cx<D>(D(f[k].re), D(f[k].im));
    f += cnt;
  }
  for (int n = n_start; n < n_end; ++n)
    kbe_step(md, t, order, n, P, U4.data(), L.data(), R.data(), ring, static_cast<Cx<D>*>(nullptr), nthreads);
  const Cx<D>* last = L.data() + tri(n_end - 1, n_end - 1) * M * M;
  C64* ov = (C64*)Lv;
  C64* od = (C64*)Ld;
  for (int k = 0; k < M * M; ++k) {
    ov[k] = C64(last[k].re.v, last[k].im.v);
    od[k] = C64(last[k].re.d, last[k].im.d);
  }
  return 0;
}

}  // extern "C"
