// Point-source images and magnification at one source position (Sec. 2.1:
// Eqs. lens_eq, amp_point, detJ; roots by Ehrlich-Aberth, Sec. 3.1), one
// thread per position.  Used by icrs_point_source's kernel and by the
// surrogate's feature kernel.
#pragma once

#include "icrs_common.cuh"

namespace icrs {

template <int NL>
struct PointSource {
  double A;        // sum_j 1 / |det J(z_j)|
  double min_det;  // min_j |det J(z_j)| over the images (+inf if none)
  int m;           // number of images
  uint32_t st;     // ICRS_ST_* bits
};

// Index of the lens nearest to z (original frame).
template <int NL>
__device__ __forceinline__ int ps_nearest_lens(const Lens& L, cd z) {
  int nj = 0;
  double best = abs2(z - L.a[0]);
  for (int i = 1; i < NL; ++i) { double d = abs2(z - L.a[i]); if (d < best) { best = d; nj = i; } }
  return nj;
}

// FP64 Newton on the polynomial about the nearest lens of z0, then the
// lens-equation residual in that frame against img_tol.  Returns 1 and the
// polished image (original frame) and |det J| if z0 converges to an image.
// *conv is cleared when the Newton steps had not converged (linear
// convergence next to a near-double root, where an iterate can still pass
// the residual test).
template <int NL>
__device__ inline int ps_polish_validate(const Lens& L, const double* epsd, cd w, cd z0, double img_tol, cd* zi,
                                         double* det, int* conv) {
  constexpr int N = NL * NL + 1;
  const int nj = ps_nearest_lens<NL>(L, z0);
  cd aj[NL], Dj[NL + 1], Ej[NL], bj[N + 1];
  for (int i = 0; i < NL; ++i) aj[i] = L.a[i] - L.a[nj];
  poly_DE<NL, double>(epsd, aj, Dj, Ej);
  const cd wj = w - L.a[nj];
  lens_poly<NL, double>(epsd, aj, Dj, Ej, wj, bj);
  cd x = z0 - L.a[nj];
  *conv = 0;
  for (int it = 0; it < 8; ++it) {
    cd p, dp;
    horner2<N, double>(bj, x, p, dp);
    if (!(abs2(dp) > 0.0)) break;
    const cd stp = dv(p, dp);
    x = x - stp;
    if (abs2(stp) <= 1e-30 * fmax(1.0, abs2(x))) { *conv = 1; break; }
  }
  const cd F = lens_map<NL, double>(epsd, aj, x) - wj;
  if (!(sqrt(abs2(F)) <= img_tol)) return 0;
  const cd gm = shear<NL, double>(epsd, aj, x);
  *det = fabs(1.0 - abs2(gm));
  *zi = x + L.a[nj];
  return 1;
}

// Two rejected roots of a binary lens closer than PS_PAIR_TOL max(1, |z|)
// make the image set untrustworthy (the ray stage's root check uses the same
// tolerance).
constexpr double PS_PAIR_TOL = 5e-2;

// Images of the source position w.  FP32 Ehrlich-Aberth on the polynomial
// about the lightest lens (triple: a second one about the second-lightest
// lens for the roots nearest it), then FP64 Newton on the polynomial about
// each root's nearest lens and validation against img_tol in that frame.  If
// that image set is not trustworthy (an illegal count, a Newton polish that
// did not converge, two roots that polish to the same image: FP32
// approximations that met at one root of a close cluster, or, binary lens,
// two close roots that are not images), all roots are
// solved again by FP64 Ehrlich-Aberth from the FP32 ones (their converged
// roots validated the same way).  images (optional): [N_deg][2]
// positions, the first m valid, the rest zero.
template <int NL>
__device__ inline PointSource<NL> point_source_solve(const Lens L, const cd w, const int max_iter,
                                                     const double img_tol, double* images) {
  constexpr int N = NL * NL + 1;
  constexpr float kEps32 = 5.9604645e-8f;
  const int ll = L.ll;
  float eps32[NL];
  cf a32[NL], D[NL + 1], E[NL];
  double epsd[NL];
  cd ad[NL], Dd[NL + 1], Ed[NL];
  for (int i = 0; i < NL; ++i) { epsd[i] = L.eps[i]; ad[i] = L.a[i] - L.a[ll]; eps32[i] = (float)epsd[i]; a32[i] = tof(ad[i]); }
  poly_DE<NL, double>(epsd, ad, Dd, Ed);
  for (int i = 0; i <= NL; ++i) D[i] = tof(Dd[i]);
  for (int i = 0; i < NL; ++i) E[i] = tof(Ed[i]);
  const cd wl = w - L.a[ll];
  cf b[N + 1];
  lens_poly<NL, float>(eps32, a32, D, E, tof(wl), b);
  cf z[N];
  float last[N];
  cauchy_start<N>(b, z);
  PointSource<NL> out;
  out.st = 0;
  if (ehrlich_aberth_f32<N>(b, z, max_iter, 4.0f * kEps32, last) < 0) out.st |= ICRS_ST_NONCONV;
  // candidate roots in the original frame (FP64)
  cd cand[2 * N];
  int nc = 0;
  int l2 = -1;
  if (NL == 3) {
    for (int i = 0; i < NL; ++i) if (i != ll && (l2 < 0 || L.eps[i] < L.eps[l2])) l2 = i;
  }
  for (int j = 0; j < N; ++j) {
    const cd z0 = tod(z[j]) + L.a[ll];
    if (NL == 3 && ps_nearest_lens<NL>(L, z0) == l2) continue;
    cand[nc++] = z0;
  }
  if (NL == 3) {
    cd a2[NL], D2d[NL + 1], E2d[NL];
    cf a2f[NL], D2[NL + 1], E2[NL], b2[N + 1], z2[N];
    for (int i = 0; i < NL; ++i) { a2[i] = L.a[i] - L.a[l2]; a2f[i] = tof(a2[i]); }
    poly_DE<NL, double>(epsd, a2, D2d, E2d);
    for (int i = 0; i <= NL; ++i) D2[i] = tof(D2d[i]);
    for (int i = 0; i < NL; ++i) E2[i] = tof(E2d[i]);
    lens_poly<NL, float>(eps32, a2f, D2, E2, tof(w - L.a[l2]), b2);
    for (int j = 0; j < N; ++j) z2[j] = tof(tod(z[j]) + L.a[ll] - L.a[l2]);
    if (ehrlich_aberth_f32<N>(b2, z2, max_iter, 4.0f * kEps32, last) < 0) out.st |= ICRS_ST_NONCONV;
    for (int j = 0; j < N; ++j) {
      const cd z0 = tod(z2[j]) + L.a[l2];
      if (ps_nearest_lens<NL>(L, z0) != l2) continue;
      if (nc < 2 * N) cand[nc++] = z0;
    }
  }
  cd img[N], rej[2 * N];
  double dets[N];
  int m = 0, nr = 0;
  bool trust = true;
  for (int j = 0; j < nc; ++j) {
    cd zi;
    double det;
    int conv;
    if (!ps_polish_validate<NL>(L, epsd, w, cand[j], img_tol, &zi, &det, &conv)) {
      // binary lens: two rejected roots close together may be a close image
      // pair that the FP32 polynomial rounded into a pair of false roots
      if (NL == 2) {
        for (int i = 0; i < nr; ++i)
          if (abs2(cand[j] - rej[i]) <= PS_PAIR_TOL * PS_PAIR_TOL * fmax(1.0, abs2(cand[j]))) trust = false;
        rej[nr++] = cand[j];
      }
      continue;
    }
    if (!conv) trust = false;
    for (int i = 0; i < m; ++i)
      if (abs2(zi - img[i]) <= 1e-18 * fmax(1.0, abs2(zi))) trust = false;
    if (m >= N) { trust = false; break; }
    img[m] = zi;
    dets[m] = det;
    ++m;
  }
  auto legal = [](int c) { return (NL == 2) ? (c == 3 || c == 5) : (c == 4 || c == 6 || c == 8 || c == 10); };
  if (!trust || !legal(m)) {
    // FP64 Ehrlich-Aberth on all roots (polynomial about the lightest lens),
    // warm-started from the FP32 roots, then the same polish and validation
    cd bd[N + 1], zd[N];
    lens_poly<NL, double>(epsd, ad, Dd, Ed, wl, bd);
    for (int j = 0; j < N; ++j) zd[j] = tod(z[j]);
    for (int j = 1; j < N; ++j)
      for (int i = 0; i < j; ++i)
        if (abs2(zd[j] - zd[i]) < 1e-20) zd[j] = zd[j] + mk(1e-7 * (j + 1), 1e-7 * j);
    if (ehrlich_aberth_f64<N>(bd, zd, max_iter) < 0) out.st |= ICRS_ST_NONCONV;
    m = 0;
    for (int j = 0; j < N; ++j) {
      cd zi;
      double det;
      int conv;
      if (!ps_polish_validate<NL>(L, epsd, w, zd[j] + L.a[ll], img_tol, &zi, &det, &conv)) continue;
      img[m] = zi;
      dets[m] = det;
      ++m;
    }
  }
  if (!legal(m)) out.st |= ICRS_ST_IMGCOUNT;
  double Asum = 0.0, mind = __longlong_as_double(0x7ff0000000000000LL);
  for (int j = 0; j < m; ++j) {
    Asum += 1.0 / dets[j];
    mind = fmin(mind, dets[j]);
    if (images) { images[j * 2] = img[j].x; images[j * 2 + 1] = img[j].y; }
  }
  if (images)
    for (int j = m; j < N; ++j) { images[j * 2] = 0.0; images[j * 2 + 1] = 0.0; }
  out.A = Asum;
  out.min_det = mind;
  out.m = m;
  return out;
}

}  // namespace icrs
