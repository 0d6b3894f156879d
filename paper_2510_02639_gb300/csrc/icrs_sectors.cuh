// Sector rules of the image-centred grid (Sec. 3.2), written once over the
// scalar type: double for the magnification, DualD (value + 8 tangents with
// respect to t0, tE, u0, alpha, s, q, rho, u1) for its derivative.  Every
// decision (overlap, which bound is larger, wrap) is taken on values, so both
// instantiations build the same sectors.
#pragma once

#include "icrs_common.cuh"

namespace icrs {

constexpr int NPAR = 8;  // t0, tE, u0, alpha, s, q, rho, u1

struct DualD {
  double v;
  double d[NPAR];
};
__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ double val(const DualD& x) { return x.v; }
__device__ __forceinline__ DualD dconst(double c) { DualD r; r.v = c; for (int i = 0; i < NPAR; ++i) r.d[i] = 0.0; return r; }
__device__ __forceinline__ DualD operator+(const DualD& a, const DualD& b) { DualD r; r.v = a.v + b.v; for (int i = 0; i < NPAR; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
__device__ __forceinline__ DualD operator-(const DualD& a, const DualD& b) { DualD r; r.v = a.v - b.v; for (int i = 0; i < NPAR; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
__device__ __forceinline__ DualD operator+(const DualD& a, double c) { DualD r = a; r.v += c; return r; }
__device__ __forceinline__ DualD operator-(const DualD& a, double c) { DualD r = a; r.v -= c; return r; }
__device__ __forceinline__ DualD operator*(double c, const DualD& a) { DualD r; r.v = c * a.v; for (int i = 0; i < NPAR; ++i) r.d[i] = c * a.d[i]; return r; }

template <class T> __device__ __forceinline__ T sconst(double c);
template <> __device__ __forceinline__ double sconst<double>(double c) { return c; }
template <> __device__ __forceinline__ DualD sconst<DualD>(double c) { return dconst(c); }
template <class T> __device__ __forceinline__ T smin(const T& a, const T& b) { return val(b) < val(a) ? b : a; }
template <class T> __device__ __forceinline__ T smax(const T& a, const T& b) { return val(b) > val(a) ? b : a; }

template <class T> struct BoxT {
  T r_lo, r_hi, th_lo, width;  // theta in [th_lo, th_lo + width)
  int periodic;
};

__device__ __forceinline__ double wrap_pi(double a) {
  double x = fmod(a + kPi, 2.0 * kPi);
  if (x < 0) x += 2.0 * kPi;
  return x - kPi;
}

template <class T>
__device__ inline bool box_overlap(const BoxT<T>& a, const BoxT<T>& b) {
  if (!(val(a.r_lo) < val(b.r_hi) && val(b.r_lo) < val(a.r_hi))) return false;
  if (a.periodic || b.periodic) return true;
  double d = fmod(val(b.th_lo) - val(a.th_lo), 2.0 * kPi);
  if (d < 0) d += 2.0 * kPi;
  return d < val(a.width) || d + val(b.width) > 2.0 * kPi;
}

template <class T>
__device__ inline void box_full(BoxT<T>& u) {
  u.periodic = 1;
  u.th_lo = sconst<T>(-kPi);
  u.width = sconst<T>(2.0 * kPi);
}

// Union of two overlapping sectors: r range min/max; the smallest arc covering
// both theta arcs (full circle if >= 2 pi).
template <class T>
__device__ inline BoxT<T> box_unite(const BoxT<T>& a, const BoxT<T>& b) {
  BoxT<T> u;
  u.r_lo = smin(a.r_lo, b.r_lo);
  u.r_hi = smax(a.r_hi, b.r_hi);
  if (a.periodic || b.periodic) { box_full(u); return u; }
  double raw = val(b.th_lo) - val(a.th_lo);
  double dv_ = fmod(raw, 2.0 * kPi);
  if (dv_ < 0) dv_ += 2.0 * kPi;
  T d = b.th_lo - a.th_lo + (dv_ - raw);  // offset of b from a, carries tangents
  T wdt, start;
  if (dv_ < val(a.width)) {
    start = a.th_lo;
    wdt = smax(a.width, d + b.width);
  } else {
    start = a.th_lo + d - 2.0 * kPi;
    wdt = smax(a.width + 2.0 * kPi - d, b.width);
  }
  if (val(wdt) >= 2.0 * kPi) {
    box_full(u);
  } else {
    u.periodic = 0;
    double sv = val(start);
    u.th_lo = start + (wrap_pi(sv) - sv);
    u.width = wdt;
  }
  return u;
}

template <class T>
__device__ inline double box_area(const BoxT<T>& b) {
  return 0.5 * (val(b.r_hi) * val(b.r_hi) - val(b.r_lo) * val(b.r_lo)) * val(b.width);
}

// Sector of one (angular interval, radial run) cell from the min/max r and
// (unwrapped) theta of its points: widened by margin * extent per side,
// r >= 0, r_lo = 0 for the lowest radial run when the origin maps inside the
// source, full circle for a full angular interval or a width >= 2 pi.
template <class T>
__device__ inline BoxT<T> cell_box(const T& rmin, const T& rmax, const T& tmin, const T& tmax,
                                   double m, bool full, bool origin_lowest) {
  BoxT<T> B;
  T er = rmax - rmin;
  B.r_lo = rmin - m * er;
  if (val(B.r_lo) < 0.0) B.r_lo = sconst<T>(0.0);
  B.r_hi = rmax + m * er;
  if (origin_lowest) B.r_lo = sconst<T>(0.0);
  T et = tmax - tmin;
  T lo = tmin - m * et;
  T wd = et + (2.0 * m) * et;
  if (full || val(wd) >= 2.0 * kPi) {
    box_full(B);
  } else {
    B.periodic = 0;
    double lv = val(lo);
    B.th_lo = lo + (wrap_pi(lv) - lv);
    B.width = wd;
  }
  return B;
}

// Merge overlapping sectors until none overlap, then while there are more
// than cap, merge the pair whose union adds the least area.  Returns the
// count; *capped is set when the cap forced a merge.
template <class T>
__device__ inline int merge_boxes(BoxT<T>* box, int nb, int cap, bool* capped) {
  for (;;) {
    bool merged = false;
    for (int i = 0; i < nb && !merged; ++i)
      for (int j = i + 1; j < nb && !merged; ++j)
        if (box_overlap(box[i], box[j])) {
          box[i] = box_unite(box[i], box[j]);
          for (int k = j; k < nb - 1; ++k) box[k] = box[k + 1];
          --nb;
          merged = true;
        }
    if (merged) continue;
    if (nb <= cap) break;
    *capped = true;
    int bi = 0, bj = 1;
    double best = 0.0;
    bool have = false;
    for (int i = 0; i < nb; ++i)
      for (int j = i + 1; j < nb; ++j) {
        BoxT<T> u = box_unite(box[i], box[j]);
        double cost = box_area(u) - box_area(box[i]) - box_area(box[j]);
        if (!have || cost < best) { best = cost; bi = i; bj = j; have = true; }
      }
    box[bi] = box_unite(box[bi], box[bj]);
    for (int k = bj; k < nb - 1; ++k) box[k] = box[k + 1];
    --nb;
  }
  return nb;
}

}  // namespace icrs
