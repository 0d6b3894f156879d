// ICRS oracle: plain, single-threaded FP64 CPU implementation of image-centred
// ray shooting (microJAX, arXiv:2510.02639).
//
// TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or runs
// this file; only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
// leg use it.  It shares no code, header, table or constant generator with the
// CUDA library: it is written directly from the paper, in the paper's order,
// with no blocking, fusion or reordering beyond what the method states.
//
// Every step cites the passage it follows:
//   lens equation, Eq. (lens_eq), Sec. 2.1
//   point-source magnification and det J, Eqs. (amp_point), (detJ), Sec. 2.1
//   lens polynomial of degree 5(N-1), Eq. (lens_eq_z), Sec. 2.1
//   Ehrlich-Aberth iteration and Cauchy-circle start, Sec. 3.1
//   source-limb sampling and polar binning of image-limb points, Sec. 3.2
//   fixed N_r x N_theta polar grid per sector, Sec. 3.3
//   inclusion indicator, cubic boundary crossing, uniform and limb-darkened
//   per-point rules, radial sum, normalisation, Appendix A.1 and A.2
//   triple-lens geometry, Fig. 3 caption and Sec. 3.5
//
// Readings taken where the paper is silent, garbled or self-contradictory are
// marked "READING:" and listed in the design notes.
//
// The whole pipeline is a template over the scalar type: T = double for the
// primal, T = Dual (value + 8 tangents) for the forward-mode derivative with
// respect to (t0, tE, u0, alpha, s, q, rho, u1).  Discrete decisions (image
// validity, bins, inclusion flags) are always taken on values.
//
// Parity status: every function here is pinned by tests under tests/ against
// closed forms, brute force, library routines and invariants (no function is
// "parity unpinned").

#include <cmath>
#include <cstdint>
#include <cstring>
#include <cstdlib>
#include <vector>
#include <limits>
#include <type_traits>
#include <algorithm>

namespace {

const double PI = 3.14159265358979323846;
const int ND = 8;  // tangent slots: t0, tE, u0, alpha, s, q, rho, u1

// ----------------------------------------------------------------------------
// Scalars: double and an 8-direction forward-mode dual number.
// ----------------------------------------------------------------------------
struct Dual {
  double v;
  double d[ND];
  Dual() : v(0) { for (int i = 0; i < ND; ++i) d[i] = 0; }
  Dual(double x) : v(x) { for (int i = 0; i < ND; ++i) d[i] = 0; }
};
inline Dual operator+(const Dual& a, const Dual& b) { Dual r(a.v + b.v); for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
inline Dual operator-(const Dual& a, const Dual& b) { Dual r(a.v - b.v); for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
inline Dual operator-(const Dual& a) { Dual r(-a.v); for (int i = 0; i < ND; ++i) r.d[i] = -a.d[i]; return r; }
inline Dual operator*(const Dual& a, const Dual& b) { Dual r(a.v * b.v); for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
inline Dual operator/(const Dual& a, const Dual& b) { Dual r(a.v / b.v); for (int i = 0; i < ND; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v; return r; }
inline Dual operator+(const Dual& a, double b) { return a + Dual(b); }
inline Dual operator+(double a, const Dual& b) { return Dual(a) + b; }
inline Dual operator-(const Dual& a, double b) { return a - Dual(b); }
inline Dual operator-(double a, const Dual& b) { return Dual(a) - b; }
inline Dual operator*(const Dual& a, double b) { Dual r(a.v * b); for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b; return r; }
inline Dual operator*(double a, const Dual& b) { return b * a; }
inline Dual operator/(const Dual& a, double b) { return a * (1.0 / b); }
inline Dual operator/(double a, const Dual& b) { return Dual(a) / b; }
inline Dual sqrt(const Dual& a) { Dual r(std::sqrt(a.v)); for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] / (2.0 * r.v); return r; }
inline Dual sin(const Dual& a) { Dual r(std::sin(a.v)); double c = std::cos(a.v); for (int i = 0; i < ND; ++i) r.d[i] = c * a.d[i]; return r; }
inline Dual cos(const Dual& a) { Dual r(std::cos(a.v)); double s = -std::sin(a.v); for (int i = 0; i < ND; ++i) r.d[i] = s * a.d[i]; return r; }
inline Dual atan2(const Dual& y, const Dual& x) {
  Dual r(std::atan2(y.v, x.v));
  double den = x.v * x.v + y.v * y.v;
  for (int i = 0; i < ND; ++i) r.d[i] = (x.v * y.d[i] - y.v * x.d[i]) / den;
  return r;
}
inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
using std::sqrt; using std::sin; using std::cos; using std::atan2;

template <class T> inline T tmin(const T& a, const T& b) { return val(b) < val(a) ? b : a; }
template <class T> inline T tmax(const T& a, const T& b) { return val(b) > val(a) ? b : a; }

// ----------------------------------------------------------------------------
// Complex numbers over T.
// ----------------------------------------------------------------------------
template <class T> struct Cx { T re, im; Cx() : re(0.0), im(0.0) {} Cx(T a, T b) : re(a), im(b) {} };
template <class T> inline Cx<T> operator+(const Cx<T>& a, const Cx<T>& b) { return Cx<T>(a.re + b.re, a.im + b.im); }
template <class T> inline Cx<T> operator-(const Cx<T>& a, const Cx<T>& b) { return Cx<T>(a.re - b.re, a.im - b.im); }
template <class T> inline Cx<T> operator*(const Cx<T>& a, const Cx<T>& b) { return Cx<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
template <class T> inline Cx<T> scale(const Cx<T>& a, const T& s) { return Cx<T>(a.re * s, a.im * s); }
template <class T> inline Cx<T> conj(const Cx<T>& a) { return Cx<T>(a.re, -a.im); }
template <class T> inline T abs2(const Cx<T>& a) { return a.re * a.re + a.im * a.im; }
template <class T> inline Cx<T> cdiv(const Cx<T>& a, const Cx<T>& b) { T n = abs2(b); return Cx<T>((a.re * b.re + a.im * b.im) / n, (a.im * b.re - a.re * b.im) / n); }
template <class T> inline Cx<double> cval(const Cx<T>& a) { return Cx<double>(val(a.re), val(a.im)); }
inline double cabs(const Cx<double>& a) { return std::hypot(a.re, a.im); }
typedef Cx<double> C;

// ----------------------------------------------------------------------------
// Inputs (flat arrays so the Python side needs no shared struct definition).
// params[23] = t0, tE, u0, alpha, rho, u1, n_lens, s, q, q2, q3, s2, s3, psi,
//              u2, a1, a2, a3, a4, spot_x, spot_y, spot_r, spot_c
// grid[13]   = n_r, n_theta, n_limb, n_bins_r, n_bins_theta, max_iter,
//              uniform, delta_c, margin, img_tol, ld_split, grad_rule, s_fac
// ----------------------------------------------------------------------------
const int NPRM = 23;  // slots of one parameter set
struct Grid {
  int n_r, n_theta, n_limb, n_bins_r, n_bins_theta, max_iter, uniform, ld_split, grad_rule;
  double delta_c, margin, img_tol, s_fac;
};
Grid grid_from(const double* g) {
  Grid G;
  G.n_r = (int)g[0]; G.n_theta = (int)g[1]; G.n_limb = (int)g[2];
  G.n_bins_r = (int)g[3]; G.n_bins_theta = (int)g[4]; G.max_iter = (int)g[5];
  G.uniform = (int)g[6]; G.delta_c = g[7]; G.margin = g[8]; G.img_tol = g[9];
  G.ld_split = (int)g[10];
  G.grad_rule = (int)g[11]; G.s_fac = g[12];
  return G;
}

// Status bits (per epoch).
const uint32_t ST_NONCONV = 1u, ST_IMGCOUNT = 2u, ST_SECTCAP = 4u, ST_EDGE = 8u, ST_NAN = 16u;

// ----------------------------------------------------------------------------
// Lens configuration (Eq. lens_eq; triple-lens geometry from Fig. 3).
// Binary: eps1 = 1/(1+q), eps2 = q/(1+q); origin at the centre of mass, the
//   primary on the negative real axis: a1 = -q s/(1+q), a2 = s/(1+q).
//   READING: the paper does not say which lens sits at -x.
// Triple: eps2 = q2, eps3 = q3, eps1 = 1 - q2 - q3 (mass fractions);
//   a1, a2 on the real axis, s2 apart, origin at their barycentre;
//   a3 = (a1 + a2)/2 + s3 e^{i psi}.
//   READING: q2/q3 taken as fractions of the total mass; psi measured from
//   the binary axis at the M1-M2 midpoint (Fig. 3).
// ----------------------------------------------------------------------------
template <class T> struct Lens { int n; T eps[3]; Cx<T> a[3]; };

template <class T>
Lens<T> make_lens(const double* p, const T& s, const T& q) {
  Lens<T> L;
  int n_lens = (int)p[6];
  if (n_lens == 2) {
    L.n = 2;
    T one_q = 1.0 + q;
    L.eps[0] = 1.0 / one_q;
    L.eps[1] = q / one_q;
    L.a[0] = Cx<T>(-(q * s) / one_q, T(0.0));
    L.a[1] = Cx<T>(s / one_q, T(0.0));
  } else {
    L.n = 3;
    double q2 = p[9], q3 = p[10], s2 = p[11], s3 = p[12], psi = p[13];
    double e1 = 1.0 - q2 - q3, e2 = q2, e3 = q3;
    L.eps[0] = e1; L.eps[1] = e2; L.eps[2] = e3;
    double x1 = -s2 * e2 / (e1 + e2), x2 = s2 * e1 / (e1 + e2);
    L.a[0] = Cx<T>(T(x1), T(0.0));
    L.a[1] = Cx<T>(T(x2), T(0.0));
    L.a[2] = Cx<T>(T(0.5 * (x1 + x2) + s3 * std::cos(psi)), T(s3 * std::sin(psi)));
  }
  return L;
}

// Lens map f(z) = z - sum_i eps_i / conj(z - a_i)  (Eq. lens_eq).
template <class T>
Cx<T> lens_map(const Lens<T>& L, const Cx<T>& z) {
  Cx<T> w = z;
  for (int i = 0; i < L.n; ++i) {
    Cx<T> d = z - L.a[i];
    T n = abs2(d);
    // eps / conj(d) = eps * d / |d|^2
    w = w - scale(d, L.eps[i] / n);
  }
  return w;
}

// gamma(z) = sum_i eps_i / (z - a_i)^2; det J = 1 - |gamma|^2  (Eq. detJ).
template <class T>
Cx<T> shear(const Lens<T>& L, const Cx<T>& z) {
  Cx<T> g;
  for (int i = 0; i < L.n; ++i) {
    Cx<T> d = z - L.a[i];
    Cx<T> d2 = d * d;
    g = g + cdiv(Cx<T>(L.eps[i], T(0.0)), d2);
  }
  return g;
}

Lens<double> lens_val(const Lens<Dual>& L) {
  Lens<double> R; R.n = L.n;
  for (int i = 0; i < L.n; ++i) { R.eps[i] = L.eps[i].v; R.a[i] = cval(L.a[i]); }
  return R;
}
Lens<double> lens_val(const Lens<double>& L) { return L; }

// ----------------------------------------------------------------------------
// Lens polynomial (Eq. lens_eq_z).  The paper does not print the
// coefficients; they follow from the lens equation:
//   conj(z) = conj(w) + sum_i eps_i/(z - a_i) = H(z)/D(z),
//   D = prod_i (z - a_i),  H = conj(w) D + sum_i eps_i prod_{j!=i}(z - a_j);
// substituting into the lens equation with G_k = H - conj(a_k) D gives
//   P(z) = (z - w) prod_k G_k - D sum_k eps_k prod_{j!=k} G_j,
// of degree N^2 + 1 = 5(N-1) for N = 2, 3.
// READING: the polynomial is written in coordinates centred on the lightest
// lens (the lens equation is translation invariant); this keeps the roots
// near a low-mass companion well conditioned.  Roots are returned in the
// original frame.
// ----------------------------------------------------------------------------
typedef std::vector<C> Poly;  // low -> high order

Poly pmul(const Poly& a, const Poly& b) {
  Poly r(a.size() + b.size() - 1);
  for (size_t i = 0; i < a.size(); ++i)
    for (size_t j = 0; j < b.size(); ++j) r[i + j] = r[i + j] + a[i] * b[j];
  return r;
}
Poly padd(const Poly& a, const Poly& b) {
  Poly r(std::max(a.size(), b.size()));
  for (size_t i = 0; i < a.size(); ++i) r[i] = r[i] + a[i];
  for (size_t i = 0; i < b.size(); ++i) r[i] = r[i] + b[i];
  return r;
}
Poly pscale(const Poly& a, const C& s) { Poly r(a.size()); for (size_t i = 0; i < a.size(); ++i) r[i] = a[i] * s; return r; }

int lightest_lens(const Lens<double>& L) {
  int k = 0;
  for (int i = 1; i < L.n; ++i) if (L.eps[i] < L.eps[k]) k = i;
  return k;
}

// Coefficients of P in the frame centred at c (z' = z - c).
Poly lens_poly(const Lens<double>& L, C w, C c) {
  int N = L.n;
  C a[3];
  for (int i = 0; i < N; ++i) a[i] = L.a[i] - c;
  w = w - c;
  Poly D(1, C(1.0, 0.0));
  for (int i = 0; i < N; ++i) D = pmul(D, Poly{C(-a[i].re, -a[i].im), C(1.0, 0.0)});
  Poly H = pscale(D, conj(w));
  for (int i = 0; i < N; ++i) {
    Poly t(1, C(L.eps[i], 0.0));
    for (int j = 0; j < N; ++j) if (j != i) t = pmul(t, Poly{C(-a[j].re, -a[j].im), C(1.0, 0.0)});
    H = padd(H, t);
  }
  std::vector<Poly> G(N);
  for (int k = 0; k < N; ++k) G[k] = padd(H, pscale(D, C(-a[k].re, a[k].im)));  // H - conj(a_k) D
  Poly P(1, C(1.0, 0.0));
  for (int k = 0; k < N; ++k) P = pmul(P, G[k]);
  P = pmul(P, Poly{C(-w.re, -w.im), C(1.0, 0.0)});
  Poly S(1, C(0.0, 0.0));
  for (int k = 0; k < N; ++k) {
    Poly t(1, C(L.eps[k], 0.0));
    for (int j = 0; j < N; ++j) if (j != k) t = pmul(t, G[j]);
    S = padd(S, t);
  }
  P = padd(P, pscale(pmul(D, S), C(-1.0, 0.0)));
  P.resize(N * N + 2);  // degree N^2 + 1
  return P;
}

// ----------------------------------------------------------------------------
// Ehrlich-Aberth iteration (Sec. 3.1): all roots updated simultaneously,
//   z_k <- z_k - 1 / (P'(z_k)/P(z_k) - sum_{j!=k} 1/(z_k - z_j)),
// written as z_k - W_k / (1 - W_k S_k) with W_k = P/P' so that an exact
// root (P = 0) gives a zero step.  Start: n points uniformly on the circle of
// Cauchy-bound radius R = 1 + max_{l<n} |b_l / b_n|.
// READING: the phase offset pi/(2n) and the stopping rule are not given in the
// paper; iteration stops once every step is below 1e-14 max(1, |z|) or below
// the rounding level of P at that root (8 eps sum|b_l||z|^l / |P'|), after at
// most max_iter iterations.
// Returns 1 if converged.
// ----------------------------------------------------------------------------
int ehrlich_aberth(const Poly& b, int max_iter, C* z) {
  int n = (int)b.size() - 1;
  double R = 0.0;
  for (int l = 0; l < n; ++l) R = std::max(R, cabs(cdiv(b[l], b[n])));
  R += 1.0;
  for (int k = 0; k < n; ++k) {
    double ph = 2.0 * PI * k / n + PI / (2.0 * n);
    z[k] = C(R * std::cos(ph), R * std::sin(ph));
  }
  C dz[16];
  double noise[16];
  for (int it = 0; it < max_iter; ++it) {
    for (int k = 0; k < n; ++k) {
      C p = b[n], dp(0.0, 0.0);
      double ab = cabs(b[n]), az = cabs(z[k]);
      for (int l = n - 1; l >= 0; --l) { dp = dp * z[k] + p; p = p * z[k] + b[l]; ab = ab * az + cabs(b[l]); }
      // rounding level of the step: evaluation error of P over |P'|
      noise[k] = 8.0 * 1.1102230246251565e-16 * ab / std::max(cabs(dp), 1e-300);
      if (p.re == 0.0 && p.im == 0.0) { dz[k] = C(0.0, 0.0); continue; }
      C W = cdiv(p, dp);
      C S(0.0, 0.0);
      for (int j = 0; j < n; ++j) if (j != k) S = S + cdiv(C(1.0, 0.0), z[k] - z[j]);
      dz[k] = cdiv(W, C(1.0, 0.0) - W * S);
    }
    bool done = true;
    for (int k = 0; k < n; ++k) {
      z[k] = z[k] - dz[k];
      double step = cabs(dz[k]);
      if (!(step <= std::max(1e-14 * std::max(1.0, cabs(z[k])), noise[k]))) done = false;
    }
    if (done) return 1;
  }
  return 0;
}

// Lens shifted to the frame centred at c (a_i -> a_i - c).
template <class T>
Lens<T> shifted(const Lens<T>& L, const Cx<T>& c) {
  Lens<T> R = L;
  for (int i = 0; i < L.n; ++i) R.a[i] = L.a[i] - c;
  return R;
}

// Newton's method on a polynomial, from x, until the step is below 1e-15
// max(1, |x|) or below the rounding level of P (at most 8 steps).
void newton_polish(const Poly& b, C* x) {
  int n = (int)b.size() - 1;
  for (int it = 0; it < 8; ++it) {
    C p = b[n], dp(0.0, 0.0);
    double ab = cabs(b[n]), az = cabs(*x);
    for (int l = n - 1; l >= 0; --l) { dp = dp * (*x) + p; p = p * (*x) + b[l]; ab = ab * az + cabs(b[l]); }
    if ((p.re == 0.0 && p.im == 0.0) || (dp.re == 0.0 && dp.im == 0.0)) return;
    C step = cdiv(p, dp);
    *x = *x - step;
    double noise = 8.0 * 1.1102230246251565e-16 * ab / cabs(dp);
    if (cabs(step) <= std::max(1e-15 * std::max(1.0, cabs(*x)), noise)) return;
  }
}

// A root of the lens polynomial, stored as the offset x = z - a_j from its
// nearest lens j, so that roots beside a low-mass lens keep their relative
// precision.
struct Root { int j; C x; };

// All roots of P for source position w.  READING (numerical, not in the
// paper): EA runs on the polynomial written about the lightest lens; for a
// triple lens, each root whose nearest lens is another lens is refined by
// Newton's method on the polynomial written about that lens (the two light
// companions each carry a cluster of roots).  Returns 1 if EA converged.
int lens_roots(const Lens<double>& L, C w, int max_iter, Root* R) {
  int n = L.n * L.n + 1;
  int ll = lightest_lens(L);
  C c = L.a[ll];
  Poly b = lens_poly(L, w, c);
  C z[16];
  int ok = ehrlich_aberth(b, max_iter, z);
  Poly bj[3];
  bool have[3] = {false, false, false};
  for (int k = 0; k < n; ++k) {
    int j = 0;
    double best = cabs(z[k] - (L.a[0] - c));
    for (int i = 1; i < L.n; ++i) {
      double d = cabs(z[k] - (L.a[i] - c));
      if (d < best) { best = d; j = i; }
    }
    C x = z[k];
    if (j != ll) {
      x = z[k] - (L.a[j] - c);
      if (L.n == 3) {
        if (!have[j]) { bj[j] = lens_poly(L, w, L.a[j]); have[j] = true; }
        newton_polish(bj[j], &x);
      }
    }
    R[k].j = j;
    R[k].x = x;
  }
  return ok;
}

// All polynomial roots for source position w (original frame).
int poly_roots(const Lens<double>& L, C w, int max_iter, C* z) {
  Root R[16];
  int ok = lens_roots(L, w, max_iter, R);
  for (int k = 0; k < L.n * L.n + 1; ++k) z[k] = L.a[R[k].j] + R[k].x;
  return ok;
}

// Image validation (Sec. 2.1: every root must be substituted back into the
// lens equation).  READING: a root is an image iff |f(z) - w| <= img_tol, with
// the residual evaluated in the frame of the root's nearest lens.
bool is_image(const Lens<double>& L, const Root& R, C w, double img_tol) {
  C aj = L.a[R.j];
  C F = lens_map(shifted(L, aj), R.x) - (w - aj);
  double r = cabs(F);
  return r == r && r <= img_tol;
}

// gamma at a root, evaluated in its nearest lens's frame.
C root_shear(const Lens<double>& L, const Root& R) { return shear(shifted(L, L.a[R.j]), R.x); }

// Legal image counts: N+1 ... 5(N-1) in steps of two: binary {3, 5},
// triple {4, 6, 8, 10}  (Sec. 2.1).
bool legal_count(int n_lens, int m) {
  if (n_lens == 2) return m == 3 || m == 5;
  return m == 4 || m == 6 || m == 8 || m == 10;
}

// Images of a point source at w; returns the count.
int images(const Lens<double>& L, C w, const Grid& G, Root* out, uint32_t* st) {
  Root R[16];
  if (!lens_roots(L, w, G.max_iter, R)) *st |= ST_NONCONV;
  int n = L.n * L.n + 1, m = 0;
  for (int k = 0; k < n; ++k)
    if (is_image(L, R[k], w, G.img_tol)) out[m++] = R[k];
  if (!legal_count(L.n, m)) *st |= ST_IMGCOUNT;
  return m;
}

// Point-source magnification A = sum_j 1/|det J(z_j)|  (Eqs. amp_point, detJ).
double point_source(const Lens<double>& L, C w, const Grid& G, uint32_t* st, C* imgs, int* n_img) {
  Root z[16];
  int m = images(L, w, G, z, st);
  double A = 0.0;
  for (int j = 0; j < m; ++j) {
    double g2 = abs2(root_shear(L, z[j]));
    A += 1.0 / std::fabs(1.0 - g2);
    if (imgs) imgs[j] = L.a[z[j].j] + z[j].x;
  }
  if (n_img) *n_img = m;
  return A;
}

// ----------------------------------------------------------------------------
// Parameters -> trajectory (Sec. 3.5 parameter list; Fig. 3 for the angle).
// READING: w_c = tau (cos a, sin a) + u0 (-sin a, cos a), tau = (t - t0)/tE.
// ----------------------------------------------------------------------------
// Brightness-profile coefficients beyond u1 (not differentiated), and a
// circular spot: centre (sx, sy) rho from the source centre, radius sr rho,
// brightness times (1 - sc) inside it.
struct Prof { double u2; double a[4]; double sx, sy, sr, sc; };
template <class T> struct Par { T t0, tE, u0, alpha, s, q, rho, u1; Prof pf; };

template <class T> Par<T> par_from(const double* p, bool seed);
template <> Par<double> par_from<double>(const double* p, bool) {
  Par<double> P;
  P.t0 = p[0]; P.tE = p[1]; P.u0 = p[2]; P.alpha = p[3]; P.rho = p[4]; P.u1 = p[5];
  P.s = p[7]; P.q = p[8];
  P.pf.u2 = p[14];
  for (int k = 0; k < 4; ++k) P.pf.a[k] = p[15 + k];
  P.pf.sx = p[19]; P.pf.sy = p[20]; P.pf.sr = p[21]; P.pf.sc = p[22];
  return P;
}
template <> Par<Dual> par_from<Dual>(const double* p, bool) {
  Par<Dual> P;
  P.t0 = Dual(p[0]); P.t0.d[0] = 1.0;
  P.tE = Dual(p[1]); P.tE.d[1] = 1.0;
  P.u0 = Dual(p[2]); P.u0.d[2] = 1.0;
  P.alpha = Dual(p[3]); P.alpha.d[3] = 1.0;
  P.s = Dual(p[7]); P.s.d[4] = 1.0;
  P.q = Dual(p[8]); P.q.d[5] = 1.0;
  P.rho = Dual(p[4]); P.rho.d[6] = 1.0;
  P.u1 = Dual(p[5]); P.u1.d[7] = 1.0;
  P.pf.u2 = p[14];
  for (int k = 0; k < 4; ++k) P.pf.a[k] = p[15 + k];
  P.pf.sx = p[19]; P.pf.sy = p[20]; P.pf.sr = p[21]; P.pf.sc = p[22];
  return P;
}

template <class T>
Cx<T> source_centre(const Par<T>& P, double t) {
  T tau = (t - P.t0) / P.tE;
  T ca = cos(P.alpha), sa = sin(P.alpha);
  return Cx<T>(tau * ca - P.u0 * sa, tau * sa + P.u0 * ca);
}

// Lift an image position found on values to T with the implicit derivative
// of the lens equation F(z; p) = f(z; p) - w(p) = 0:
//   dz = -J^{-1} dF|_{z fixed}, J the real 2x2 Jacobian of f at z.
// (The root-level form of the implicit derivative of Sec. 3.5.)
// root: the image in its nearest lens's frame (for the Jacobian); z: the
// image in the original frame.
Cx<double> lift(const Lens<double>&, const Root&, const Lens<double>&, const Cx<double>& z, const Cx<double>&) { return z; }
Cx<Dual> lift(const Lens<double>& Lv, const Root& root, const Lens<Dual>& L, const Cx<double>& z, const Cx<Dual>& w) {
  Cx<Dual> zc(Dual(z.re), Dual(z.im));
  Cx<Dual> F = lens_map(L, zc) - w;  // value ~ 0, tangents = dF/dp
  // df = dz + conj(gamma) conj(dz)  -> real 2x2 Jacobian
  C g = root_shear(Lv, root);
  // [dx', dy'] = [[1 + gr, gi], [gi, 1 - gr]] [dx, dy], with conj(gamma) = gr - i gi:
  // conj(g) conj(dz) = (gr - i gi)(dx - i dy) = gr dx - gi dy - i(gi dx + gr dy)
  double j11 = 1.0 + g.re, j12 = -g.im, j21 = -g.im, j22 = 1.0 - g.re;
  double det = j11 * j22 - j12 * j21;
  Cx<Dual> out(Dual(z.re), Dual(z.im));
  for (int i = 0; i < ND; ++i) {
    double fx = F.re.d[i], fy = F.im.d[i];
    out.re.d[i] = -(j22 * fx - j12 * fy) / det;
    out.im.d[i] = -(-j21 * fx + j11 * fy) / det;
  }
  return out;
}

// ----------------------------------------------------------------------------
// Image-centred sectors from binned image-limb points (Sec. 3.2).
// ----------------------------------------------------------------------------
template <class T> struct Pt { T r, th; double rv, thv; };

template <class T> struct Box {
  T r_lo, r_hi, th_lo, width;  // theta in [th_lo, th_lo + width)
  bool periodic;
};

inline double wrap_pi(double a) {  // -> [-pi, pi)
  double x = std::fmod(a + PI, 2.0 * PI);
  if (x < 0) x += 2.0 * PI;
  return x - PI;
}

template <class T> double box_area(const Box<T>& b) {
  return 0.5 * (val(b.r_hi) * val(b.r_hi) - val(b.r_lo) * val(b.r_lo)) * val(b.width);
}

template <class T> bool boxes_overlap(const Box<T>& a, const Box<T>& b) {
  if (!(val(a.r_lo) < val(b.r_hi) && val(b.r_lo) < val(a.r_hi))) return false;
  if (a.periodic || b.periodic) return true;
  double d = std::fmod(val(b.th_lo) - val(a.th_lo), 2.0 * PI);
  if (d < 0) d += 2.0 * PI;
  return d < val(a.width) || d + val(b.width) > 2.0 * PI;
}

template <class T> Box<T> box_union(const Box<T>& a, const Box<T>& b) {
  Box<T> u;
  u.r_lo = tmin(a.r_lo, b.r_lo);
  u.r_hi = tmax(a.r_hi, b.r_hi);
  if (a.periodic || b.periodic) {
    u.periodic = true; u.th_lo = T(-PI); u.width = T(2.0 * PI);
    return u;
  }
  // Offset of b's start from a's start, measured counter-clockwise.
  double dv = std::fmod(val(b.th_lo) - val(a.th_lo), 2.0 * PI);
  if (dv < 0) dv += 2.0 * PI;
  T d = b.th_lo - a.th_lo + (dv - (val(b.th_lo) - val(a.th_lo)));  // carries tangents
  T wdt;
  T start;
  if (dv < val(a.width)) {          // b starts inside a
    start = a.th_lo;
    wdt = tmax(a.width, d + b.width);
  } else {                          // b wraps round to cover a's start
    start = a.th_lo + d - 2.0 * PI;
    wdt = tmax(a.width + 2.0 * PI - d, b.width);
  }
  if (val(wdt) >= 2.0 * PI) {
    u.periodic = true; u.th_lo = T(-PI); u.width = T(2.0 * PI);
  } else {
    u.periodic = false;
    double sv = val(start);
    u.th_lo = start + (wrap_pi(sv) - sv);
    u.width = wdt;
  }
  return u;
}

// Gap probe / origin probe: does image-plane point z map inside the source?
bool maps_inside(const Lens<double>& L, C z, C wc, double rho) {
  C w = lens_map(L, z);
  return cabs(w - wc) < rho;
}

// READING (the paper gives the idea, not the rules):
//  1. r and theta of every valid image-limb point about the coordinate origin.
//  2. theta histogram: n_bins_theta bins over [-pi, pi); runs of non-empty
//     bins (wrapping round) are the angular intervals.
//  3. For each angular interval, an r histogram of its own points: n_bins_r
//     bins over their [min r, max r]; runs of non-empty bins are the radial
//     intervals.  (Binning r per angular interval keeps a far image in another
//     direction from coarsening the bins.)
//  4. An empty r gap between two radial runs is image interior when an image
//     wraps round it (a ring): it is filled when a probe ray at the gap's
//     middle radius, at the centre of a theta bin that holds points both below
//     and above the gap, maps inside the source.
//  5. If the origin maps inside the source, the lowest radial run of every
//     angular interval starts at r = 0.
//  6. Candidate sectors are (angular interval, radial run) cells holding
//     points; their bounds are the min/max r and theta of those points,
//     widened by margin * extent on each side (r >= 0; width >= 2 pi or a
//     full angular interval -> the full circle starting at -pi).
//  7. Overlapping sectors are merged until none overlap.
//  8. At most N_deg sectors: while more, merge the pair whose union adds the
//     least area; flag SECTCAP.
template <class T>
std::vector<Box<T>> build_sectors(const std::vector<Pt<T>>& pts, const Lens<double>& Lv,
                                  C wc, double rho, const Grid& G, int cap, uint32_t* st) {
  std::vector<Box<T>> boxes;
  const int BR = G.n_bins_r, BT = G.n_bins_theta;
  int np = (int)pts.size();
  if (np == 0) return boxes;
  const double ht = 2.0 * PI / BT;
  // Step 2: theta bins and runs.
  std::vector<int> tb(np), occT(BT, 0);
  for (int p = 0; p < np; ++p) {
    int t = (int)std::floor((pts[p].thv + PI) / ht);
    if (t > BT - 1) t = BT - 1;
    if (t < 0) t = 0;
    tb[p] = t;
    occT[t] = 1;
  }
  std::vector<int> runT(BT, -1), startT;
  int nT = 0;
  bool full = true;
  for (int t = 0; t < BT; ++t) if (!occT[t]) full = false;
  if (full) {
    for (int t = 0; t < BT; ++t) runT[t] = 0;
    startT.push_back(0);
    nT = 1;
  } else {
    int t0 = 0;
    while (occT[t0]) ++t0;  // an empty bin exists
    for (int k = 1; k <= BT; ++k) {
      int t = (t0 + k) % BT;
      if (!occT[t]) continue;
      int prev = (t + BT - 1) % BT;
      if (occT[prev]) runT[t] = runT[prev];
      else { runT[t] = nT++; startT.push_back(t); }
    }
  }
  bool origin_in = maps_inside(Lv, C(0.0, 0.0), wc, rho);
  for (int T_ = 0; T_ < nT; ++T_) {
    // Step 3: r histogram of this angular interval's points.
    std::vector<int> mine;
    for (int p = 0; p < np; ++p) if (runT[tb[p]] == T_) mine.push_back(p);
    double rlo = pts[mine[0]].rv, rhi = rlo;
    for (int p : mine) { rlo = std::min(rlo, pts[p].rv); rhi = std::max(rhi, pts[p].rv); }
    double hr = (rhi - rlo) / BR;
    std::vector<int> rb(np, 0), occR(BR, 0);
    std::vector<std::vector<char>> tmaskR(BR, std::vector<char>(BT, 0));  // theta bins per r bin
    for (int p : mine) {
      int b = hr > 0 ? (int)std::floor((pts[p].rv - rlo) / hr) : 0;
      if (b > BR - 1) b = BR - 1;
      if (b < 0) b = 0;
      rb[p] = b;
      occR[b] = 1;
      tmaskR[b][tb[p]] = 1;
    }
    // Step 4: fill gaps that an image wraps round.
    std::vector<int> fill(BR, 0);
    for (int b = 1; b < BR; ++b) {
      if (occR[b] || !occR[b - 1]) continue;  // b = first empty bin of a gap
      int e = b;
      while (e < BR && !occR[e]) ++e;       // gap = [b, e); bin BR-1 is occupied
      std::vector<char> below(BT, 0), above(BT, 0);
      for (int k = 0; k < b; ++k) for (int t = 0; t < BT; ++t) below[t] |= tmaskR[k][t];
      for (int k = e; k < BR; ++k) for (int t = 0; t < BT; ++t) above[t] |= tmaskR[k][t];
      double rg = rlo + hr * 0.5 * (double)(b + e);
      bool inside = false;
      for (int t = 0; t < BT && !inside; ++t) {
        if (!(below[t] && above[t])) continue;
        double th = -PI + (t + 0.5) * ht;
        if (maps_inside(Lv, C(rg * std::cos(th), rg * std::sin(th)), wc, rho)) inside = true;
      }
      if (inside) for (int k = b; k < e; ++k) fill[k] = 1;
    }
    for (int b = 0; b < BR; ++b) if (fill[b]) occR[b] = 1;
    std::vector<int> runR(BR, -1);
    int nR = 0;
    for (int b = 0; b < BR; ++b) {
      if (!occR[b]) continue;
      if (b > 0 && occR[b - 1]) runR[b] = runR[b - 1]; else runR[b] = nR++;
    }
    // Step 6: cells of this angular interval.
    std::vector<int> cnt(nR, 0);
    std::vector<T> crlo(nR), crhi(nR), ctlo(nR), cthi(nR);
    double start = -PI + startT[T_] * ht;
    for (int p : mine) {
      int c = runR[rb[p]];
      T thu = pts[p].th;
      if (pts[p].thv < start) thu = thu + 2.0 * PI;  // unwrap within the interval
      if (cnt[c] == 0) { crlo[c] = crhi[c] = pts[p].r; ctlo[c] = cthi[c] = thu; }
      else {
        crlo[c] = tmin(crlo[c], pts[p].r); crhi[c] = tmax(crhi[c], pts[p].r);
        ctlo[c] = tmin(ctlo[c], thu); cthi[c] = tmax(cthi[c], thu);
      }
      cnt[c]++;
    }
    for (int c = 0; c < nR; ++c) {
      if (!cnt[c]) continue;
      Box<T> B;
      T er = crhi[c] - crlo[c];
      B.r_lo = crlo[c] - G.margin * er;
      if (val(B.r_lo) < 0.0) B.r_lo = T(0.0);
      B.r_hi = crhi[c] + G.margin * er;
      if (origin_in && c == 0) B.r_lo = T(0.0);  // step 5
      T et = cthi[c] - ctlo[c];
      T lo = ctlo[c] - G.margin * et, wd = et + 2.0 * G.margin * et;
      if (full || val(wd) >= 2.0 * PI) {
        B.periodic = true; B.th_lo = T(-PI); B.width = T(2.0 * PI);
      } else {
        B.periodic = false;
        double lv = val(lo);
        B.th_lo = lo + (wrap_pi(lv) - lv);
        B.width = wd;
      }
      boxes.push_back(B);
    }
  }
  // Step 7: merge overlapping sectors to a fixpoint; step 8: cap.
  for (;;) {
    bool merged = false;
    for (size_t i = 0; i < boxes.size() && !merged; ++i)
      for (size_t j = i + 1; j < boxes.size() && !merged; ++j)
        if (boxes_overlap(boxes[i], boxes[j])) {
          boxes[i] = box_union(boxes[i], boxes[j]);
          boxes.erase(boxes.begin() + j);
          merged = true;
        }
    if (merged) continue;
    if ((int)boxes.size() <= cap) break;
    *st |= ST_SECTCAP;
    size_t bi = 0, bj = 1;
    double best = 0.0;
    bool have = false;
    for (size_t i = 0; i < boxes.size(); ++i)
      for (size_t j = i + 1; j < boxes.size(); ++j) {
        Box<T> u = box_union(boxes[i], boxes[j]);
        double cost = box_area(u) - box_area(boxes[i]) - box_area(boxes[j]);
        if (!have || cost < best) { best = cost; bi = i; bj = j; have = true; }
      }
    boxes[bi] = box_union(boxes[bi], boxes[bj]);
    boxes.erase(boxes.begin() + bj);
  }
  return boxes;
}

// ----------------------------------------------------------------------------
// Quadrature (Appendix A).
// ----------------------------------------------------------------------------

// Lagrange interpolant through (x_m, y_m), m < npt, and its derivative at x.
template <class T>
void lagrange(const double* xs, const T* ys, int npt, double x, T* f, double* df) {
  T acc(0.0);
  double dacc = 0.0;
  for (int m = 0; m < npt; ++m) {
    double l = 1.0, dl = 0.0;
    for (int k = 0; k < npt; ++k) {
      if (k == m) continue;
      double den = xs[m] - xs[k];
      // derivative of the product by the product rule
      dl = dl * (x - xs[k]) / den + l / den;
      l = l * (x - xs[k]) / den;
    }
    acc = acc + ys[m] * l;
    dacc += val(ys[m]) * dl;
  }
  *f = acc;
  *df = dacc;
}

// Crossing of the interpolated distance with rho on the bracket between the
// inside sample (x_in) and the outside sample (x_out), offsets in grid steps.
// READING: safeguarded Newton from the linear-interpolation guess, bisection
// when a step leaves the bracket; FP64 to 1e-13.  The T version adds the
// implicit derivative dx = -g_T / g'.
template <class T>
T crossing(const double* xs, const T* ys, int npt, double x_in, double x_out, const T& rho) {
  double rv = val(rho);
  double yin = 0, yout = 0;
  for (int m = 0; m < npt; ++m) { if (xs[m] == x_in) yin = val(ys[m]); if (xs[m] == x_out) yout = val(ys[m]); }
  double x = x_in + (x_out - x_in) * (rv - yin) / (yout - yin);
  double lo = x_in, hi = x_out;  // g(lo) < 0 (inside), g(hi) >= 0
  for (int it = 0; it < 60; ++it) {
    T f; double df;
    lagrange(xs, ys, npt, x, &f, &df);
    double g = val(f) - rv;
    if (g < 0) lo = x; else hi = x;
    double xn = (df != 0.0) ? x - g / df : 0.5 * (lo + hi);
    bool in_br = (lo < hi) ? (xn > lo && xn < hi) : (xn > hi && xn < lo);
    if (!in_br) xn = 0.5 * (lo + hi);
    if (std::fabs(xn - x) < 1e-13) { x = xn; break; }
    x = xn;
  }
  T f; double df;
  lagrange(xs, ys, npt, x, &f, &df);
  T xt(x);
  // implicit derivative of g(x) = L(x; y) - rho = 0
  xt = xt - (f - rho - (val(f) - rv)) / df;
  return xt;
}

// f(delta): LD correction (Appendix A.2) or the uniform rule delta + 1/2.
// The paper's gradient rule (Sec. 3.5, G.grad_rule = 1) keeps the value and
// gives the LD correction the fixed derivative of its second-order branch,
// f'(delta) = 2/3, on both branches.
template <class T>
T fdelta(const T& delta, const Grid& G) {
  if (G.uniform) return delta + 0.5;
  if (G.grad_rule) {
    const double dv_ = val(delta);
    const double fv = dv_ >= G.delta_c ? (0.5 + dv_) * ((2.0 / 3.0) * std::sqrt(1.0 + 1.0 / (2.0 * dv_)))
                                       : (2.0 / 3.0) * dv_ + 0.5;
    return T(fv) + (2.0 / 3.0) * (delta - dv_);  // value fv, tangent (2/3) d delta
  }
  if (val(delta) >= G.delta_c) return (0.5 + delta) * ((2.0 / 3.0) * sqrt(1.0 + 1.0 / (2.0 * delta)));
  return (2.0 / 3.0) * delta + 0.5;
}

// Limb darkening (Appendix A.2 gives the linear law; the quadratic law adds
// the next term in (1 - mu), mu = sqrt(1 - rt^2); the paper's "arbitrary
// profiles" are read as the power series in mu^(1/2) of the four-coefficient
// law, each term normalised like the others):
//   I(rt) = I0 [1 - u1 (1 - mu) - u2 (1 - mu)^2 - sum_k a_k (1 - mu^(k/2))],
//   I0 = 1 / (pi (1 - u1/3 - u2/6 - sum_k a_k k/(k+4)))
// (int_0^1 (1 - mu^(k/2)) 2 rt drt = k/(k+4); = 3 / (pi (3 - u1)) for the
// linear law, the normalisation of Appendix A.2: the total flux is 1);
// uniform: 1/pi.
template <class T>
T norm_I0(const T& u1, const Prof& pf) {
  double sa = 0.0;
  for (int k = 1; k <= 4; ++k) sa += pf.a[k - 1] * (double)k / (double)(k + 4);
  return 1.0 / (PI * (1.0 - u1 / 3.0 - pf.u2 / 6.0 - sa));
}
template <class T>
T brightness(const T& rt2, const T& u1, const Prof& pf, const Grid& G) {
  if (G.uniform) return T(1.0 / PI);
  T I0 = norm_I0(u1, pf);
  T one = T(1.0);
  T x = one - rt2;
  if (val(x) < 0) x = T(0.0);
  T mu = sqrt(x);
  T om = one - mu;
  T I = one - u1 * om - pf.u2 * (om * om);
  if (pf.a[0] != 0.0 || pf.a[1] != 0.0 || pf.a[2] != 0.0 || pf.a[3] != 0.0) {
    T sq = sqrt(mu);  // mu^(1/2)
    T pw = one;
    for (int k = 1; k <= 4; ++k) {
      pw = pw * sq;
      I = I - pf.a[k - 1] * (one - pw);
    }
  }
  return I0 * I;
}

// The same law at the limb (mu = 0): the part of I that jumps to zero across
// the source edge.
template <class T>
T brightness_limb(const T& u1, const Prof& pf, const Grid& G) {
  if (G.uniform) return T(1.0 / PI);
  return norm_I0(u1, pf) * (1.0 - u1 - pf.u2 - pf.a[0] - pf.a[1] - pf.a[2] - pf.a[3]);
}

// Integral over one sector: sum_i A_i dr with
//   A_i = r_i dtheta sum_l I_l chi_l W_l   (Appendix A.2 per-point rule).
// Split-profile rule (G.ld_split = 1; a variant, not in the paper): the part
// of I that is constant across the edge, I_limb, takes the uniform-source
// weight W_U (f_U(delta) = delta + 1/2, exact for a step) and the rest,
// which vanishes at the edge like sqrt(distance), the weight W of f(delta):
//   I_l W_l  ->  I_limb W_U,l + (I_l - I_limb) W_l.
// READING (per-point form for both profiles): W = 1 if both neighbours are
// inside; f(delta_L) / f(delta_R) if the left / right neighbour is outside
// with delta_L = (theta_l - theta_cross)/dtheta, delta_R = (theta_cross -
// theta_l)/dtheta; max(0, f(delta_L) + f(delta_R) - 1) if both are outside.
// Neighbours beyond a non-periodic grid edge count as outside with delta = 1/2
// (flag EDGE); a missing stencil point degrades the cubic to a quadratic, then
// linear fit (flag EDGE).
// Gauss-Legendre nodes and weights on [-1, 1] (Newton on the Legendre
// recurrence from the Chebyshev-like first guess).
inline void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-15) {
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        break;
      }
    }
  }
}

// The spot's share of the unspotted flux, F_spot = int_spot I dA in units of
// rho (the disk's flux is 1): polar quadrature about the spot centre, the
// periodic trapezoid rule in the angle (128 nodes) and Gauss-Legendre in the
// radius (16 nodes per panel) on panels graded geometrically toward the
// spot's edge ([0, sr/2], [sr/2, 3 sr/4], ..., 20 halvings, then the rest),
// where a spot that touches the limb meets the square-root profile.
template <class T>
T spot_flux(const T& u1, const Prof& pf, const Grid& G) {
  std::vector<double> gx, gw;
  gauss_legendre(16, gx, gw);
  const int NA = 128;
  std::vector<double> edges{0.0};
  for (int k = 1; k <= 20; ++k) edges.push_back(pf.sr * (1.0 - std::ldexp(1.0, -k)));
  edges.push_back(pf.sr);
  T sum(0.0);
  for (size_t b = 0; b + 1 < edges.size(); ++b) {
    const double lo = edges[b], hi = edges[b + 1];
    for (size_t i = 0; i < gx.size(); ++i) {
      const double rr = 0.5 * (hi - lo) * gx[i] + 0.5 * (hi + lo);
      const double wr = 0.5 * (hi - lo) * gw[i] * rr * (2.0 * PI / NA);
      for (int j = 0; j < NA; ++j) {
        const double ph = 2.0 * PI * j / NA;
        const double x = pf.sx + rr * std::cos(ph), y = pf.sy + rr * std::sin(ph);
        sum = sum + wr * brightness(T(x * x + y * y), u1, pf, G);
      }
    }
  }
  return sum;
}

// Spot (a variant beyond the paper's radial profiles; the paper names
// starspots as a case ICRS handles by sampling): READING: each ray's
// brightness is multiplied by (1 - sc) when its source-plane position lies
// inside the spot, a plain midpoint decision with no sub-pixel rule at the
// spot's edge (the paper gives none).
template <class T>
T sector_integral(const Box<T>& B, const Lens<T>& L, const Cx<T>& wc, const T& rho,
                  const T& u1, const Prof& pf, const Grid& G, uint32_t* st) {
  const int NR = G.n_r, NT = G.n_theta;
  T dr = (B.r_hi - B.r_lo) / (double)NR;
  T dth = B.width / (double)NT;
  std::vector<T> d(NT);
  std::vector<char> chi(NT);
  std::vector<double> fs(NT, 1.0);  // spot factor of each ray
  T total(0.0);
  T rho2 = rho * rho;
  for (int i = 0; i < NR; ++i) {
    T r = B.r_lo + (i + 0.5) * dr;
    for (int l = 0; l < NT; ++l) {
      T th = B.th_lo + (l + 0.5) * dth;
      Cx<T> z(r * cos(th), r * sin(th));
      Cx<T> w = lens_map(L, z);
      Cx<T> dw = w - wc;
      d[l] = sqrt(abs2(dw));
      chi[l] = val(d[l]) < val(rho);  // chi = Theta(rho - d), strict (Sec. 2.2)
      if (pf.sc != 0.0) {
        const double ex = val(dw.re) / val(rho) - pf.sx, ey = val(dw.im) / val(rho) - pf.sy;
        fs[l] = (ex * ex + ey * ey < pf.sr * pf.sr) ? 1.0 - pf.sc : 1.0;
      }
    }
    T row(0.0);
    if constexpr (std::is_same<T, Dual>::value) {
      // The paper's gradient rule (Sec. 3.5): the indicator chi = Theta(x)
      // gets the derivative of a sigmoid of steepness S, dchi/dx =
      // S s (1 - s), s = 1 / (1 + e^{-S x}).  READING: x = (rho - d) / rho
      // (S dimensionless); each ray's term I_l dchi_l (the interior weight),
      // a tangent only -- the primal value is unchanged.
      if (G.grad_rule) {
        for (int l = 0; l < NT; ++l) {
          T x = (rho - d[l]) / rho;
          double sx = G.s_fac * val(x);
          if (std::fabs(sx) > 40.0) continue;
          double sg = 1.0 / (1.0 + std::exp(-sx));
          double dchi = G.s_fac * sg * (1.0 - sg);
          double Iv = val(brightness(d[l] * d[l] / rho2, u1, pf, G)) * fs[l];
          row = row + (Iv * dchi) * (x - val(x));
        }
      }
    }
    for (int l = 0; l < NT; ++l) {
      if (!chi[l]) continue;
      auto idx = [&](int k) -> int {  // -1: beyond a non-periodic edge
        if (B.periodic) return ((k % NT) + NT) % NT;
        return (k < 0 || k >= NT) ? -1 : k;
      };
      int lm = idx(l - 1), lp = idx(l + 1);
      bool Lin = lm >= 0 && chi[lm];
      bool Rin = lp >= 0 && chi[lp];
      T W, WU;
      if (Lin && Rin) {
        W = T(1.0);
        WU = T(1.0);
      } else {
        T fL(0.0), fR(0.0), uL(0.0), uR(0.0);
        if (!Lin) {
          T dl;
          if (lm < 0) { dl = T(0.5); *st |= ST_EDGE; }
          else {
            // entering: stencil offsets -2, -1, 0, +1; bracket (-1, 0)
            double xs[4]; T ys[4]; int npt = 0;
            int cand[4] = {-2, -1, 0, 1};
            for (int c = 0; c < 4; ++c) {
              int k = idx(l + cand[c]);
              if (k < 0) { *st |= ST_EDGE; continue; }
              xs[npt] = cand[c]; ys[npt] = d[k]; ++npt;
            }
            T x = crossing(xs, ys, npt, 0.0, -1.0, rho);
            dl = -x;
          }
          fL = fdelta(dl, G);
          uL = dl + 0.5;
        }
        if (!Rin) {
          T dd;
          if (lp < 0) { dd = T(0.5); *st |= ST_EDGE; }
          else {
            double xs[4]; T ys[4]; int npt = 0;
            int cand[4] = {-1, 0, 1, 2};
            for (int c = 0; c < 4; ++c) {
              int k = idx(l + cand[c]);
              if (k < 0) { *st |= ST_EDGE; continue; }
              xs[npt] = cand[c]; ys[npt] = d[k]; ++npt;
            }
            dd = crossing(xs, ys, npt, 0.0, 1.0, rho);
          }
          fR = fdelta(dd, G);
          uR = dd + 0.5;
        }
        if (Lin) { W = fR; WU = uR; }
        else if (Rin) { W = fL; WU = uL; }
        else {
          W = fL + fR - 1.0; if (val(W) < 0) W = T(0.0);
          WU = uL + uR - 1.0; if (val(WU) < 0) WU = T(0.0);
        }
      }
      T I = brightness(d[l] * d[l] / rho2, u1, pf, G);
      if (G.ld_split && !G.uniform) {
        T Il = brightness_limb(u1, pf, G);
        row = row + (Il * WU + (I - Il) * W) * fs[l];
      } else {
        row = row + I * W * fs[l];
      }
    }
    total = total + r * row;
  }
  return total * dth * dr;
}

// ----------------------------------------------------------------------------
// One epoch: limb roots -> sectors -> rays -> magnification.
// ----------------------------------------------------------------------------
template <class T>
T magnification_epoch(const double* prm, double t, const Grid& G, uint32_t* st,
                      std::vector<Box<T>>* boxes_out) {
  Par<T> P = par_from<T>(prm, true);
  Lens<T> L = make_lens<T>(prm, P.s, P.q);
  Lens<double> Lv = lens_val(L);
  Cx<T> wc = source_centre(P, t);
  C wcv = cval(wc);
  int n_lens = Lv.n;
  int ndeg = n_lens * n_lens + 1;
  // Source-limb points w_k = w_c + rho e^{2 pi i k / N_limb}  (Sec. 3.2).
  // READING: the printed exponent lacks the index k.
  std::vector<Pt<T>> pts;
  pts.reserve(G.n_limb * ndeg);
  for (int k = 0; k < G.n_limb; ++k) {
    double ph = 2.0 * PI * k / G.n_limb;
    Cx<T> w = wc + Cx<T>(P.rho * std::cos(ph), P.rho * std::sin(ph));
    C wv = cval(w);
    Root R[16];
    if (!lens_roots(Lv, wv, G.max_iter, R)) *st |= ST_NONCONV;
    int m = 0;
    for (int j = 0; j < ndeg; ++j) {
      if (!is_image(Lv, R[j], wv, G.img_tol)) continue;
      ++m;
      Cx<T> zt = lift(Lv, R[j], L, Lv.a[R[j].j] + R[j].x, w);
      Pt<T> p;
      p.r = sqrt(abs2(zt));
      p.th = atan2(zt.im, zt.re);
      p.rv = val(p.r); p.thv = val(p.th);
      pts.push_back(p);
    }
    if (!legal_count(n_lens, m)) *st |= ST_IMGCOUNT;
  }
  std::vector<Box<T>> boxes = build_sectors(pts, Lv, wcv, val(P.rho), G, ndeg, st);
  if (boxes_out) *boxes_out = boxes;
  T sum(0.0);
  for (size_t b = 0; b < boxes.size(); ++b)
    sum = sum + sector_integral(boxes[b], L, wc, P.rho, P.u1, P.pf, G, st);
  // A = sum_sectors A_sector / rho^2 (Appendix A.2; with I = 1/pi this is the
  // 1/(pi rho^2) normalisation of Appendix A.1).
  T A = sum / (P.rho * P.rho);
  // a spot: the unlensed flux is 1 - sc F_spot, F_spot the spot's share of
  // the unspotted flux; it must lie inside the disk (else NaN)
  if (P.pf.sc != 0.0) {
    const double off = std::hypot(P.pf.sx, P.pf.sy);
    if (!(P.pf.sr >= 0.0) || !(P.pf.sc < 1.0) || !(off + P.pf.sr <= 1.0)) {
      A = T(std::numeric_limits<double>::quiet_NaN());
    } else {
      A = A / (1.0 - P.pf.sc * spot_flux(P.u1, P.pf, G));
    }
  }
  if (!(val(A) == val(A))) *st |= ST_NAN;
  return A;
}

}  // namespace

// ============================================================================
// C API (ctypes).  All pointers are host pointers owned by the caller.
// ============================================================================
extern "C" {

int orc_version(void) { return 1; }

// Lens positions and masses: eps[3], ax[3], ay[3]; returns the lens count.
int orc_lens(const double* prm, double* eps, double* ax, double* ay) {
  Lens<double> L = make_lens<double>(prm, prm[7], prm[8]);
  for (int i = 0; i < L.n; ++i) { eps[i] = L.eps[i]; ax[i] = L.a[i].re; ay[i] = L.a[i].im; }
  return L.n;
}

// Source centre at times t[n].
void orc_source_centre(const double* prm, const double* t, int n, double* wx, double* wy) {
  Par<double> P = par_from<double>(prm, false);
  for (int i = 0; i < n; ++i) { C w = source_centre(P, t[i]); wx[i] = w.re; wy[i] = w.im; }
}

// Polynomial coefficients (low -> high) in the frame centred at (cx, cy).
int orc_poly(const double* prm, double wx, double wy, double cx, double cy, double* re, double* im) {
  Lens<double> L = make_lens<double>(prm, prm[7], prm[8]);
  Poly b = lens_poly(L, C(wx, wy), C(cx, cy));
  for (size_t i = 0; i < b.size(); ++i) { re[i] = b[i].re; im[i] = b[i].im; }
  return (int)b.size() - 1;
}

// All polynomial roots (original frame).  Returns 1 if EA converged.
int orc_roots(const double* prm, double wx, double wy, int max_iter, double* zr, double* zi) {
  Lens<double> L = make_lens<double>(prm, prm[7], prm[8]);
  C z[16];
  int ok = poly_roots(L, C(wx, wy), max_iter, z);
  for (int k = 0; k < L.n * L.n + 1; ++k) { zr[k] = z[k].re; zi[k] = z[k].im; }
  return ok;
}

// Lens map at n points.
void orc_lens_map(const double* prm, const double* zx, const double* zy, int n, double* wx, double* wy) {
  Lens<double> L = make_lens<double>(prm, prm[7], prm[8]);
  for (int i = 0; i < n; ++i) { C w = lens_map(L, C(zx[i], zy[i])); wx[i] = w.re; wy[i] = w.im; }
}

// Point-source magnification at n source positions; images optional.
void orc_point_source(const double* prm, const double* grid, const double* wx, const double* wy,
                      int n, double* A, int* n_img, double* zr, double* zi, uint32_t* status) {
  Lens<double> L = make_lens<double>(prm, prm[7], prm[8]);
  Grid G = grid_from(grid);
  int nd = L.n * L.n + 1;
  for (int i = 0; i < n; ++i) {
    uint32_t st = 0;
    C imgs[16];
    int m = 0;
    A[i] = point_source(L, C(wx[i], wy[i]), G, &st, imgs, &m);
    if (n_img) n_img[i] = m;
    if (zr && zi)
      for (int j = 0; j < nd; ++j) {
        zr[i * nd + j] = j < m ? imgs[j].re : 0.0;
        zi[i * nd + j] = j < m ? imgs[j].im : 0.0;
      }
    if (status) status[i] = st;
  }
}

// Sectors of one epoch: out[k*5 + {r_lo, r_hi, th_lo, width, periodic}].
int orc_sectors(const double* prm, double t, const double* grid, double* out, int max_out, uint32_t* status) {
  Grid G = grid_from(grid);
  uint32_t st = 0;
  std::vector<Box<double>> boxes;
  magnification_epoch<double>(prm, t, G, &st, &boxes);
  int n = (int)boxes.size();
  for (int k = 0; k < n && k < max_out; ++k) {
    out[k * 5 + 0] = boxes[k].r_lo; out[k * 5 + 1] = boxes[k].r_hi;
    out[k * 5 + 2] = boxes[k].th_lo; out[k * 5 + 3] = boxes[k].width;
    out[k * 5 + 4] = boxes[k].periodic ? 1.0 : 0.0;
  }
  if (status) *status = st;
  return n;
}

// Image-limb points of one epoch: out[(k * ndeg + j) * 3 + {r, theta, valid}]
// for every root j of limb point k (Sec. 3.2).  Returns ndeg.
int orc_limb_points(const double* prm, double t, const double* grid, double* out) {
  Grid G = grid_from(grid);
  Par<double> P = par_from<double>(prm, false);
  Lens<double> L = make_lens<double>(prm, P.s, P.q);
  C wc = source_centre(P, t);
  int ndeg = L.n * L.n + 1;
  for (int k = 0; k < G.n_limb; ++k) {
    double ph = 2.0 * PI * k / G.n_limb;
    C w = wc + C(P.rho * std::cos(ph), P.rho * std::sin(ph));
    Root R[16];
    lens_roots(L, w, G.max_iter, R);
    for (int j = 0; j < ndeg; ++j) {
      C z = L.a[R[j].j] + R[j].x;
      double* o = out + ((size_t)k * ndeg + j) * 3;
      o[0] = cabs(z);
      o[1] = std::atan2(z.im, z.re);
      o[2] = is_image(L, R[j], w, G.img_tol) ? 1.0 : 0.0;
    }
  }
  return ndeg;
}

// Finite-source magnification for S parameter sets x E epochs.
// prm[S][NPRM], t[S][E], A[S][E], status[S][E] (optional).
void orc_magnification(const double* prm, int S, const double* t, int E, const double* grid,
                       double* A, uint32_t* status) {
  Grid G = grid_from(grid);
  // Epochs are independent: the baseline build compiled with OpenMP runs
  // them on all host cores (the default build is single-threaded).
#ifdef _OPENMP
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
#endif
  for (int s = 0; s < S; ++s)
    for (int e = 0; e < E; ++e) {
      uint32_t st = 0;
      A[(size_t)s * E + e] = magnification_epoch<double>(prm + NPRM * s, t[(size_t)s * E + e], G, &st, nullptr);
      if (status) status[(size_t)s * E + e] = st;
    }
}

// Forward-mode derivative: A and dA/d(t0, tE, u0, alpha, s, q, rho, u1).
// Binary lenses only.  dA[S][E][8].
void orc_magnification_fwd(const double* prm, int S, const double* t, int E, const double* grid,
                           double* A, double* dA, uint32_t* status) {
  Grid G = grid_from(grid);
  for (int s = 0; s < S; ++s)
    for (int e = 0; e < E; ++e) {
      uint32_t st = 0;
      Dual a = magnification_epoch<Dual>(prm + NPRM * s, t[(size_t)s * E + e], G, &st, nullptr);
      size_t o = (size_t)s * E + e;
      A[o] = a.v;
      for (int i = 0; i < ND; ++i) dA[o * ND + i] = a.d[i];
      if (status) status[o] = st;
    }
}

}  // extern "C"
