// Point-source images and magnification at one source position (Sec. 2.1:
// Eqs. lens_eq, amp_point, detJ; roots by Ehrlich-Aberth, Sec. 3.1), one
// thread per position, for the surrogate's feature kernel.  The steps are
// those of icrs_point_source's kernel.
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

// FP32 Ehrlich-Aberth on the polynomial about the lightest lens (triple: a
// second one about the second-lightest lens for the roots nearest it), then
// FP64 Newton on the polynomial about each root's nearest lens and validation
// against img_tol in that frame.  images (optional): [N_deg][2] positions,
// the first m valid, the rest zero.
template <int NL>
__device__ __forceinline__ PointSource<NL> point_source_solve(const Lens L, const cd w, const int max_iter,
                                                              const double img_tol, double* images) {
  // binary only (the feature kernel's case).  Everything is passed by value:
  // an earlier form that took the lens and the grid (a kernel parameter) by
  // reference returned wrong image counts on the GPU.
  static_assert(NL == 2, "point_source_solve is validated for binary lenses only");
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
  cd wl = w - L.a[ll];
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
    cd z0 = tod(z[j]) + L.a[ll];
    int nj = 0;
    double best = abs2(z0 - L.a[0]);
    for (int i = 1; i < NL; ++i) { double d = abs2(z0 - L.a[i]); if (d < best) { best = d; nj = i; } }
    if (NL == 3 && nj == l2) continue;
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
      cd z0 = tod(z2[j]) + L.a[l2];
      int nj = 0;
      double best = abs2(z0 - L.a[0]);
      for (int i = 1; i < NL; ++i) { double d = abs2(z0 - L.a[i]); if (d < best) { best = d; nj = i; } }
      if (nj != l2) continue;
      if (nc < 2 * N) cand[nc++] = z0;
    }
  }
  double Asum = 0.0, mind = __longlong_as_double(0x7ff0000000000000LL);
  int m = 0;
  for (int j = 0; j < nc; ++j) {
    cd z0 = cand[j];
    int nj = 0;
    double best = abs2(z0 - L.a[0]);
    for (int i = 1; i < NL; ++i) { double d = abs2(z0 - L.a[i]); if (d < best) { best = d; nj = i; } }
    cd aj[NL], Dj[NL + 1], Ej[NL], bj[N + 1];
    for (int i = 0; i < NL; ++i) aj[i] = L.a[i] - L.a[nj];
    poly_DE<NL, double>(epsd, aj, Dj, Ej);
    cd wj = w - L.a[nj];
    lens_poly<NL, double>(epsd, aj, Dj, Ej, wj, bj);
    cd x = z0 - L.a[nj];
    for (int it = 0; it < 8; ++it) {
      cd p, dp;
      horner2<N, double>(bj, x, p, dp);
      if (!(abs2(dp) > 0.0)) break;
      cd stp = dv(p, dp);
      x = x - stp;
      if (abs2(stp) <= 1e-30 * fmax(1.0, abs2(x))) break;
    }
    cd F = lens_map<NL, double>(epsd, aj, x) - wj;
    if (!(sqrt(abs2(F)) <= img_tol)) continue;
    if (m >= N) { out.st |= ICRS_ST_OVERFLOW; break; }
    cd gm = shear<NL, double>(epsd, aj, x);
    double det = fabs(1.0 - abs2(gm));
    Asum += 1.0 / det;
    mind = fmin(mind, det);
    if (images) {
      cd zz = x + L.a[nj];
      images[m * 2] = zz.x;
      images[m * 2 + 1] = zz.y;
    }
    ++m;
  }
  bool legal = (NL == 2) ? (m == 3 || m == 5) : (m == 4 || m == 6 || m == 8 || m == 10);
  if (!legal) out.st |= ICRS_ST_IMGCOUNT;
  if (images)
    for (int j = m; j < N; ++j) { images[j * 2] = 0.0; images[j * 2 + 1] = 0.0; }
  out.A = Asum;
  out.min_det = mind;
  out.m = m;
  return out;
}

}  // namespace icrs
