// Device helpers shared by the ICRS kernels: complex arithmetic in FP32 and
// FP64, lens configuration, the lens map and its shear, the lens polynomial
// and the Ehrlich-Aberth iteration.
//
// Method: Miyazaki & Kawahara, arXiv:2510.02639 (microJAX), Sec. 2.1 (lens
// equation, point-source magnification, lens polynomial of degree 5(N-1)) and
// Sec. 3.1 (Ehrlich-Aberth root finding from a Cauchy-bound circle).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "icrs.h"

namespace icrs {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr float kPiF = 3.14159265358979f;

// --------------------------------------------------------------- complex
template <class T> struct cx { T x, y; };
using cf = cx<float>;
using cd = cx<double>;

template <class T> __device__ __forceinline__ cx<T> mk(T a, T b) { cx<T> r; r.x = a; r.y = b; return r; }
template <class T> __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <class T> __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <class T> __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
  return mk(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
template <class T> __device__ __forceinline__ cx<T> scl(cx<T> a, T s) { return mk(a.x * s, a.y * s); }
template <class T> __device__ __forceinline__ cx<T> cj(cx<T> a) { return mk(a.x, -a.y); }
template <class T> __device__ __forceinline__ T abs2(cx<T> a) { return fma(a.x, a.x, a.y * a.y); }
template <class T> __device__ __forceinline__ cx<T> inv(cx<T> a) { T n = T(1) / abs2(a); return mk(a.x * n, -a.y * n); }
template <class T> __device__ __forceinline__ cx<T> dv(cx<T> a, cx<T> b) { return a * inv(b); }
__device__ __forceinline__ float cabsf_(cf a) { return sqrtf(abs2(a)); }
// The hardware approximations themselves (PTX rcp.approx / rsqrt.approx,
// subnormals flushed): reciprocal within 1 ulp, reciprocal square root within
// 2^-22.9 relative, one instruction each.  For the ray stage's normal-range
// operands only.
__device__ __forceinline__ float rcp_fast(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_fast(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double cabs_(cd a) { return sqrt(abs2(a)); }
__device__ __forceinline__ cf tof(cd a) { return mk((float)a.x, (float)a.y); }
__device__ __forceinline__ cd tod(cf a) { return mk((double)a.x, (double)a.y); }

// --------------------------------------------------------------- lens
// Masses (fractions of the total) and positions (Einstein radii) of the
// lenses; `ll` is the lightest lens, the centre of the polynomial's frame.
struct Lens {
  int n, ll;
  double eps[3];
  cd a[3];
};

// Binary: eps = (1/(1+q), q/(1+q)), a1 = -q s/(1+q), a2 = s/(1+q) (origin at
// the centre of mass).  Triple: eps = (1-q2-q3, q2, q3); lenses 1, 2 on the
// real axis s2 apart about their barycentre; lens 3 at their midpoint plus
// s3 e^{i psi} (Fig. 3).
__device__ inline Lens make_lens(const icrs_params& p) {
  Lens L;
  if (p.n_lens == 2) {
    L.n = 2;
    double oq = 1.0 + p.q;
    L.eps[0] = 1.0 / oq;
    L.eps[1] = p.q / oq;
    L.eps[2] = 0.0;
    L.a[0] = mk(-(p.q * p.s) / oq, 0.0);
    L.a[1] = mk(p.s / oq, 0.0);
    L.a[2] = mk(0.0, 0.0);
  } else {
    L.n = 3;
    double e1 = 1.0 - p.q2 - p.q3, e2 = p.q2, e3 = p.q3;
    L.eps[0] = e1; L.eps[1] = e2; L.eps[2] = e3;
    double x1 = -p.s2 * e2 / (e1 + e2), x2 = p.s2 * e1 / (e1 + e2);
    double sp, cp;
    sincos(p.psi, &sp, &cp);
    L.a[0] = mk(x1, 0.0);
    L.a[1] = mk(x2, 0.0);
    L.a[2] = mk(0.5 * (x1 + x2) + p.s3 * cp, p.s3 * sp);
  }
  int k = 0;
  for (int i = 1; i < L.n; ++i) if (L.eps[i] < L.eps[k]) k = i;
  L.ll = k;
  return L;
}

// Source centre on the straight trajectory (Sec. 3.5 parameters):
// w_c = tau (cos a, sin a) + u0 (-sin a, cos a), tau = (t - t0)/tE.
__device__ inline cd source_centre(const icrs_params& p, double t) {
  double tau = (t - p.t0) / p.tE;
  double sa, ca;
  sincos(p.alpha, &sa, &ca);
  return mk(tau * ca - p.u0 * sa, tau * sa + p.u0 * ca);
}

// Lens map w = z - sum_i eps_i / conj(z - a_i) (Eq. lens_eq) in any frame:
// `a` are the lens positions in that frame.
template <int NL, class T>
__device__ __forceinline__ cx<T> lens_map(const T* eps, const cx<T>* a, cx<T> z) {
  cx<T> w = z;
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    cx<T> d = z - a[i];
    T s = eps[i] / abs2(d);
    w = w - scl(d, s);
  }
  return w;
}

// gamma(z) = sum_i eps_i/(z - a_i)^2, det J = 1 - |gamma|^2 (Eq. detJ).
template <int NL, class T>
__device__ __forceinline__ cx<T> shear(const T* eps, const cx<T>* a, cx<T> z) {
  cx<T> g = mk(T(0), T(0));
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    cx<T> id = inv(z - a[i]);
    g = g + scl(id * id, eps[i]);
  }
  return g;
}

// One Newton step on the lens equation f(x) = w in a frame (real 2x2 system,
// df = dz + conj(gamma) conj(dz)): dz = (conj(g) conj(F) - F)/(1 - |g|^2).
template <int NL, class T>
__device__ __forceinline__ cx<T> lens_newton_step(const T* eps, const cx<T>* a, cx<T> x, cx<T> w) {
  cx<T> F = lens_map<NL, T>(eps, a, x) - w;
  cx<T> g = shear<NL, T>(eps, a, x);
  T det = T(1) - abs2(g);
  cx<T> num = cj(g) * cj(F) - F;
  return scl(num, T(1) / det);
}

// --------------------------------------------------------------- polynomial
// Product of polynomials with NA and NB coefficients (low -> high).
template <int NA, int NB, class T>
__device__ __forceinline__ void pmul(const cx<T>* a, const cx<T>* b, cx<T>* out) {
#pragma unroll
  for (int i = 0; i < NA + NB - 1; ++i) out[i] = mk(T(0), T(0));
#pragma unroll
  for (int i = 0; i < NA; ++i)
#pragma unroll
    for (int j = 0; j < NB; ++j) out[i + j] = out[i + j] + a[i] * b[j];
}

// w-independent parts of the lens polynomial in a frame with lens positions a:
// D = prod_i (z - a_i) (NL+1 coefficients), E = sum_i eps_i prod_{j!=i} (z - a_j)
// (NL coefficients).
template <int NL, class T>
__device__ inline void poly_DE(const T* eps, const cx<T>* a, cx<T>* D, cx<T>* E) {
  cx<T> tmp[NL + 1];
  D[0] = mk(T(1), T(0));
  int deg = 0;
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    // D <- D * (z - a_i)
    tmp[0] = mk(T(0), T(0));
#pragma unroll
    for (int k = 0; k <= NL; ++k) tmp[k] = mk(T(0), T(0));
    for (int k = 0; k <= deg; ++k) {
      tmp[k + 1] = tmp[k + 1] + D[k];
      tmp[k] = tmp[k] - D[k] * a[i];
    }
    ++deg;
    for (int k = 0; k <= deg; ++k) D[k] = tmp[k];
  }
#pragma unroll
  for (int k = 0; k < NL; ++k) E[k] = mk(T(0), T(0));
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    cx<T> t[NL];
    t[0] = mk(eps[i], T(0));
    int dg = 0;
#pragma unroll
    for (int k = 1; k < NL; ++k) t[k] = mk(T(0), T(0));
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      if (j == i) continue;
      cx<T> u[NL];
#pragma unroll
      for (int k = 0; k < NL; ++k) u[k] = mk(T(0), T(0));
      for (int k = 0; k <= dg; ++k) {
        if (k + 1 < NL) u[k + 1] = u[k + 1] + t[k];
        u[k] = u[k] - t[k] * a[j];
      }
      ++dg;
#pragma unroll
      for (int k = 0; k < NL; ++k) t[k] = u[k];
    }
#pragma unroll
    for (int k = 0; k < NL; ++k) E[k] = E[k] + t[k];
  }
}

// Lens polynomial P(z) = (z - w) prod_k G_k - D sum_k eps_k prod_{j!=k} G_j
// with G_k = conj(w - a_k) D + E  (derived from Eq. lens_eq; degree NL^2+1).
// All quantities in one frame.  b has NL*NL + 2 coefficients.
template <int NL, class T>
__device__ inline void lens_poly(const T* eps, const cx<T>* a, const cx<T>* D, const cx<T>* E,
                                 cx<T> w, cx<T>* b) {
  constexpr int NG = NL + 1;
  cx<T> G[NL][NG];
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    cx<T> c = cj(w - a[k]);
#pragma unroll
    for (int i = 0; i < NG; ++i) G[k][i] = c * D[i];
#pragma unroll
    for (int i = 0; i < NL; ++i) G[k][i] = G[k][i] + E[i];
  }
  if constexpr (NL == 2) {
    cx<T> PG[5], S[3], DS[5];
    pmul<3, 3, T>(G[0], G[1], PG);
#pragma unroll
    for (int i = 0; i < 3; ++i) S[i] = scl(G[1][i], eps[0]) + scl(G[0][i], eps[1]);
    pmul<3, 3, T>(D, S, DS);
    // (z - w) PG
    b[0] = mk(T(0), T(0)) - w * PG[0];
#pragma unroll
    for (int i = 1; i < 5; ++i) b[i] = PG[i - 1] - w * PG[i];
    b[5] = PG[4];
#pragma unroll
    for (int i = 0; i < 5; ++i) b[i] = b[i] - DS[i];
  } else {
    cx<T> P01[7], P02[7], P12[7], PG[10], S[7], DS[10];
    pmul<4, 4, T>(G[0], G[1], P01);
    pmul<4, 4, T>(G[0], G[2], P02);
    pmul<4, 4, T>(G[1], G[2], P12);
    pmul<7, 4, T>(P01, G[2], PG);
#pragma unroll
    for (int i = 0; i < 7; ++i) S[i] = scl(P12[i], eps[0]) + scl(P02[i], eps[1]) + scl(P01[i], eps[2]);
    pmul<4, 7, T>(D, S, DS);
    b[0] = mk(T(0), T(0)) - w * PG[0];
#pragma unroll
    for (int i = 1; i < 10; ++i) b[i] = PG[i - 1] - w * PG[i];
    b[10] = PG[9];
#pragma unroll
    for (int i = 0; i < 10; ++i) b[i] = b[i] - DS[i];
  }
}

// Horner evaluation of P and P' at z.
template <int N, class T>
__device__ __forceinline__ void horner2(const cx<T>* b, cx<T> z, cx<T>& p, cx<T>& dp) {
  p = b[N];
  dp = mk(T(0), T(0));
#pragma unroll
  for (int l = N - 1; l >= 0; --l) {
    dp = dp * z + p;
    p = p * z + b[l];
  }
}

// Initial roots on the Cauchy-bound circle R = 1 + max_{l<n} |b_l / b_n|,
// phases 2 pi k / n + pi / (2n)  (Sec. 3.1).
template <int N>
__device__ inline void cauchy_start(const cf* b, cf* z) {
  float ibn = 1.0f / sqrtf(abs2(b[N]));
  float R = 0.0f;
#pragma unroll
  for (int l = 0; l < N; ++l) R = fmaxf(R, sqrtf(abs2(b[l])) * ibn);
  R += 1.0f;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    float s, c;
    sincospif(2.0f * k / N + 0.5f / N, &s, &c);
    z[k] = mk(R * c, R * s);
  }
}

// Ehrlich-Aberth iteration in FP32 (Sec. 3.1): all roots updated together,
// z_k <- z_k - W_k / (1 - W_k S_k), W_k = P/P', S_k = sum_{j!=k} 1/(z_k - z_j).
// Stops when every step is below tol * max(1, |z_k|) or below twice the
// rounding level of P at that root (eps32 sum_l |b_l||z|^l / |P'|).  Returns
// the number of iterations, or -1 if the cap was hit; last[k] = |last step|.
template <int N>
__device__ inline int ehrlich_aberth_f32(const cf* b, cf* z, int max_iter, float tol, float* last) {
  float ab[N + 1];
#pragma unroll
  for (int l = 0; l <= N; ++l) ab[l] = sqrtf(abs2(b[l]));
  for (int it = 0; it < max_iter; ++it) {
    cf dz[N];
    float noise[N];
    bool done = true;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      cf p, dp;
      horner2<N, float>(b, z[k], p, dp);
      float az = sqrtf(abs2(z[k])), pa = ab[N];
#pragma unroll
      for (int l = N - 1; l >= 0; --l) pa = fmaf(pa, az, ab[l]);
      noise[k] = 5.9604645e-8f * pa * rsqrtf(fmaxf(abs2(dp), 1e-37f));
      cf W = dv(p, dp);
      cf S = mk(0.0f, 0.0f);
#pragma unroll
      for (int j = 0; j < N; ++j)
        if (j != k) S = S + inv(z[k] - z[j]);
      cf den = mk(1.0f, 0.0f) - W * S;
      dz[k] = dv(W, den);
      if (!(abs2(p) > 0.0f)) dz[k] = mk(0.0f, 0.0f);
    }
#pragma unroll
    for (int k = 0; k < N; ++k) {
      z[k] = z[k] - dz[k];
      float st = sqrtf(abs2(dz[k]));
      last[k] = st;
      float lim = fmaxf(tol * fmaxf(1.0f, sqrtf(abs2(z[k]))), 2.0f * noise[k]);
      if (!(st <= lim)) done = false;
    }
    if (done) return it + 1;
  }
  return -1;
}

// Ehrlich-Aberth iteration in FP64 (Sec. 3.1): the fallback for positions
// whose FP32 roots do not give a trustworthy image set (clusters of close
// roots next to a critical curve, which FP32 cannot separate).  Stops when every step is
// below 1e-14 max(1, |z|) or twice the FP64 rounding level of P at the root.
template <int N>
__device__ inline int ehrlich_aberth_f64(const cd* b, cd* z, int max_iter) {
  double ab[N + 1];
  for (int l = 0; l <= N; ++l) ab[l] = sqrt(abs2(b[l]));
  for (int it = 0; it < max_iter; ++it) {
    cd dz[N];
    double noise[N];
    bool done = true;
    for (int k = 0; k < N; ++k) {
      cd p, dp;
      horner2<N, double>(b, z[k], p, dp);
      double az = sqrt(abs2(z[k])), pa = ab[N];
      for (int l = N - 1; l >= 0; --l) pa = fma(pa, az, ab[l]);
      noise[k] = 1.1102230246251565e-16 * pa / fmax(sqrt(abs2(dp)), 1e-300);
      cd W = dv(p, dp);
      cd S = mk(0.0, 0.0);
      for (int j = 0; j < N; ++j)
        if (j != k) S = S + inv(z[k] - z[j]);
      dz[k] = dv(W, mk(1.0, 0.0) - W * S);
      if (!(abs2(p) > 0.0)) dz[k] = mk(0.0, 0.0);
    }
    for (int k = 0; k < N; ++k) {
      z[k] = z[k] - dz[k];
      double st = sqrt(abs2(dz[k]));
      if (!(st <= fmax(1e-14 * fmax(1.0, sqrt(abs2(z[k]))), 2.0 * noise[k]))) done = false;
    }
    if (done) return it + 1;
  }
  return -1;
}

}  // namespace icrs
