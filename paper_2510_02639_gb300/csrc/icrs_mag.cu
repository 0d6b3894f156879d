// Fused ICRS magnification kernel (one CUDA thread block per light-curve
// epoch, persistent over a contiguous chunk of epochs) and the C ABI of
// include/icrs.h.
//
// Method: Miyazaki & Kawahara, arXiv:2510.02639.  Per epoch:
//   1. source-limb points w_k = w_c + rho e^{2 pi i k/N_limb}      (Sec. 3.2)
//   2. all roots of the lens polynomial at each limb point by Ehrlich-Aberth
//      iteration, validated against the lens equation     (Secs. 2.1, 3.1)
//   3. image-limb points binned in theta and r into image-centred polar
//      sectors                                                    (Sec. 3.2)
//   4. a fixed N_r x N_theta polar grid per sector, every ray mapped through
//      the lens equation, inclusion flags, cubic boundary crossings and the
//      uniform / limb-darkened per-point rule, radial sum, 1/rho^2
//                                                 (Sec. 3.3, Appendix A)
//
// Precision design (GB300: FP64 issues at ~1/64 of the FP32 rate):
//   * roots are found in FP32 on the polynomial written about the lightest
//     lens, warm-started from the previous epoch of the same light curve;
//   * every discrete decision (is a root an image, which bin holds a point,
//     which point is a sector's extreme, is a ray inside the source, which
//     branch of f(delta)) is taken in FP32 only when the FP32 error bound
//     cannot change it; otherwise the point or ray is recomputed in FP64, so
//     the decisions equal those of an FP64 evaluation of the same method;
//   * rays are mapped in FP32 in a difference form about FP64 anchors placed
//     on the sector, so the FP32 error stays relative to the source size.
#include <type_traits>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "icrs.h"
#include "icrs_common.cuh"
#include "icrs_df64.cuh"
#include "icrs_sectors.cuh"
#include "icrs_ps.cuh"

namespace icrs {

// Threads per block (one block per SM).  The binary forward kernel's ray
// stage evaluates two columns per paired FP32 instruction and is bound by
// dependency latency more than by issue: registers for independent column
// pairs pay more than further warps (at 1024 x 2048 on a 320-epoch sample:
// 512 threads 6.66 ms, 576 6.86, 640 6.93, 768 7.01).  NT_WIDE is the binary
// forward block size (with a 512-thread fallback where its layout does not
// fit in shared memory); the derivative and triple instantiations keep 512
// threads (128 registers): with fewer their FP64 phases spill kilobytes.
constexpr int NT_WIDE = 512, NT_BASE = 512;
__host__ __device__ constexpr int mag_threads(int nl, bool der) { return (nl == 2 && !der) ? NT_WIDE : NT_BASE; }
constexpr int NW_MAX = NT_WIDE / 32;  // warps per block, largest instantiation
constexpr int NW_DER = NT_BASE / 32;  // warps per block, derivative mode
constexpr int QMAX = 2048;       // work queue
constexpr int PMAX_MIN = 512;    // FP64-polished image-limb points per epoch (at least)
constexpr int MAXT = 32;         // theta runs (more: ICRS_ST_OVERFLOW)
constexpr int MAXRB = 32;        // r bins per theta run
constexpr int MAXCELL = 96;      // (theta run, r run) cells
constexpr int MAXBOX = 96;       // candidate sectors before merging
constexpr int MAXANCH = 128;     // FP64 anchors per sector
constexpr int GTH_MAX = 256;     // columns per theta group (at most)
// Deferred boundary points per warp in the forward ray stage: 32 (one per
// lane when the queue is flushed), each a (column, row) pair.
__host__ __device__ constexpr int dq_entries(int) { return 32; }
constexpr int MAXCELL_D = 32;    // cells with tracked derivatives
constexpr int MAXBOX_D = 32;     // candidate sectors with tracked derivatives
constexpr float TINY_EXTENT = 3e-4f;  // images smaller than this x rho skip FP64 decisions
constexpr float EPS32 = 5.9604645e-8f;  // 2^-24
// A refined FP32 image whose error bound exceeds EE_SUSPECT max(1, r), or two
// images of one limb point closer than DUP_TOL max(1, r), send the limb point
// to the FP64 re-solve.
constexpr float EE_SUSPECT = 1e-6f;
constexpr float DUP_TOL = 1e-6f;
// Two roots of a limb point that are not images, closer than PAIR_TOL
// max(1, |z|), send it to the FP64 re-solve as well (binary lens; the
// point-source solver's tolerance).
constexpr float PAIR_TOL = (float)PS_PAIR_TOL;

// Meta bits of an image-limb slot.
constexpr uint8_t M_VALID = 1, M_EXACT = 2, M_UNSURE = 4, M_CAND = 8;

// Anchor of a (theta group, r group) of a sector: the rays' squared distance
// is evaluated about it in FP32 with U = sum_j K_j / Q_j (A_j = e^{-i th_m}
// (z_m - a_j), K_j = eps_j / A_j, Q_j = A_j + dz, dz the ray's offset from the
// anchor z_m in the anchor's rotated frame) as one quotient N / P of
// polynomials in dz, with N = sum_j K_j prod_{k != j} Q_k and P = prod_j Q_j:
//   binary:  N = n0 + n1 dz,             P = p0 + dz (p1 + dz)
//   triple:  N = n0 + dz (n1 + dz n2),   P = p0 + dz (p1 + dz (p2 + dz))
// (coefficients formed in FP64 and rounded once).
struct AnchorF {
  cf ws;        // e^{-i th_m} (f(z_m) - w_c)
  cf n[3];      // numerator coefficients
  cf p[3];      // denominator coefficients (monic)
  float e0;     // error bound constant part
  float pad;
  float lo2;    // below: every ray of the group is inside the source (FP32 certain)
  float hi2;    // above: every ray of the group is outside (FP32 certain)
};

using Box = BoxT<double>;

struct Shared {
  // ---- per parameter set
  Lens L;
  double rho, u1, u2;
  double pa[4];        // a1..a4, the power series in mu^(1/2)
  float c1h, c3h;      // their half-integer-power brightness coefficients (ray stage)
  int half;            // c1h or c3h nonzero
  // spot: centre (rho units), radius^2 and contrast; 1 / (1 - c F_spot) and
  // its u1 derivative over itself times c F_spot' ... (see the chain);
  // spot_new: the set changed and has a spot; generic: half or spot
  double spot_x, spot_y, spot_r, spot_c, spot_norm, spot_gu, spot_acc[2];
  int spot, spot_bad, spot_new, generic;
  float eps32[3];
  cf aj32[3][3];       // [frame j][lens i]: a_i - a_j (FP32)
  cf D32[3][4], E32[3][3];  // polynomial parts in frame j (FP32)
  df adf[3][3][2];     // [frame j][lens i][x/y]: a_i - a_j (double-float)
  df adf_ll[2];        // a_ll (original frame, double-float)
  df epsdf[3];
  df rhodf;
  int cur_set;
  int l2;              // second lightest lens (triple) or -1
  cf anc[32][10];      // roots of the cold-start anchor limb points
  // ---- per epoch
  cd wc;
  cf wcj32[3];         // w_c - a_j (FP32)
  df wcdf[3][2];       // w_c - a_j (double-float)
  uint32_t status;
  int warm;            // roots[] hold the previous epoch of this set
  int qn, pn;
  unsigned long long tocc[2];   // occupied theta bins (up to 128)
  int nT, full;
  signed char runT[128];
  int startT[MAXT];
  unsigned int t_rlo_u[MAXT], t_rhi_l[MAXT];
  unsigned long long t_rlo[MAXT], t_rhi[MAXT];
  double rlo[MAXT], hr[MAXT];
  unsigned int rocc[MAXT];
  unsigned long long tmask[MAXT][MAXRB][2];  // theta bins of each (run, r bin)
  signed char rrun[MAXT][MAXRB];
  int cellbase[MAXT + 1];
  int ncell;
  int origin_in;
  int c_cnt[MAXCELL];
  unsigned int c_u[MAXCELL][4];             // FP32 keys: rmin_hi, rmax_lo, tmin_hi, tmax_lo
  unsigned long long c_x[MAXCELL][4];       // FP64 keys: rmin, rmax, tmin, tmax
  int nbox;
  Box box[MAXBOX];
  int probe_hit;
  int cnt[16];         // diagnostics: FP64 polishes, FP64 validations, FP64 rays, FP64 crossings, phase clocks
  long long clk0;
  // ---- ray stage (current sector)
  int mth, mr, gth, gr;
  double dr64, dth64;
  float dr32, dth32;
  int nanch;
  int chunk;           // columns per theta chunk
  double red[NW_MAX];
};

// Derivative-mode state (binary lens), in the dynamic shared memory of that
// instantiation only.
struct DerShared {
  int cell_arg[MAXCELL_D][4];  // slot of the point that sets each cell extreme
  double Gb[MAXBOX_D][4];   // dS / d(r_lo, r_hi, th_lo, width) of each sector
  double H[8];              // dS / d(w_c.x, w_c.y, rho, u1, a1.x, a2.x, eps1, eps2)
  cd dwc[4];                // d w_c / d(t0, tE, u0, alpha)
  double dadp[2][2];        // d a_j.x / d(s, q)
  double depsq[2];          // d eps_j / d q
  DualD cx[MAXCELL_D * 4];  // cell extremes with tangents
  BoxT<DualD> box[MAXBOX_D];  // sectors with tangents
  double wder[NW_DER][12];      // per-warp sums of the row derivatives
  float2 acs[MAXANCH];      // cos, sin of each anchor angle
  float4 aA[MAXANCH];       // A_0, A_1 of each anchor (FP32)
};

// Order-preserving integer keys for signed FP32 / FP64 values.
__device__ __forceinline__ unsigned int fkey(float v) {
  unsigned int u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned int k) {
  unsigned int u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}
__device__ __forceinline__ unsigned long long dkey(double v) {
  unsigned long long u = (unsigned long long)__double_as_longlong(v);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k) {
  unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)u);
}


// ---------------------------------------------------------------- FP64 paths
// Limb point k in FP64 (Sec. 3.2).
__device__ inline cd limb_point64(const Shared& sh, int k, int n_limb) {
  double s, c;
  sincospi(2.0 * (double)k / (double)n_limb, &s, &c);
  return mk(sh.wc.x + sh.rho * c, sh.wc.y + sh.rho * s);
}

// Index of the lens nearest to z (original frame).
template <int NL>
__device__ inline int nearest_lens64(const Lens& L, cd z) {
  int j = 0;
  double best = abs2(z - L.a[0]);
  for (int i = 1; i < NL; ++i) {
    double d = abs2(z - L.a[i]);
    if (d < best) { best = d; j = i; }
  }
  return j;
}

// FP64 polish of an image-limb root by Newton's method on the lens equation
// in the frame of its nearest lens; returns (r, theta) of the image.
template <int NL>
__device__ inline void polish_image64(const Shared& sh, cd z0, cd w, double* r, double* th) {
  int j = nearest_lens64<NL>(sh.L, z0);
  double eps[NL];
  cd a[NL];
  for (int i = 0; i < NL; ++i) { eps[i] = sh.L.eps[i]; a[i] = sh.L.a[i] - sh.L.a[j]; }
  cd x = z0 - sh.L.a[j];
  cd wj = w - sh.L.a[j];
  for (int it = 0; it < 4; ++it) {
    cd st = lens_newton_step<NL, double>(eps, a, x, wj);
    x = x + st;
    if (abs2(st) <= 1e-32 * fmax(1e-20, abs2(x))) break;
  }
  cd z = x + sh.L.a[j];
  *r = sqrt(z.x * z.x + z.y * z.y);
  *th = atan2(z.y, z.x);
}

// FP64 validation of an ambiguous root: Newton's method on the polynomial
// written about the root's nearest lens, then the lens-equation residual in
// that frame against img_tol.  Returns 1 (image) or 0; (r, theta) if image.
// *conv (if given) is cleared when the Newton steps had not converged: next to
// a near-double root Newton converges only linearly, and an iterate still
// ~1e-4 from the root can pass the residual test there (the lens map is flat
// across the critical curve).
template <int NL>
__device__ inline int validate_root64(const Shared& sh, cd z0, cd w, double img_tol, double* r, double* th,
                                      int* conv = nullptr) {
  constexpr int N = NL * NL + 1;
  int j = nearest_lens64<NL>(sh.L, z0);
  double eps[NL];
  cd a[NL];
  for (int i = 0; i < NL; ++i) { eps[i] = sh.L.eps[i]; a[i] = sh.L.a[i] - sh.L.a[j]; }
  cd D[NL + 1], E[NL], b[N + 1];
  poly_DE<NL, double>(eps, a, D, E);
  cd wj = w - sh.L.a[j];
  lens_poly<NL, double>(eps, a, D, E, wj, b);
  cd x = z0 - sh.L.a[j];
  bool done = false;
  for (int it = 0; it < 8; ++it) {
    cd p, dp;
    horner2<N, double>(b, x, p, dp);
    if (!(abs2(dp) > 0.0)) break;
    cd st = dv(p, dp);
    x = x - st;
    if (abs2(st) <= 1e-30 * fmax(1.0, abs2(x))) { done = true; break; }
  }
  if (conv) *conv = done ? 1 : 0;
  cd F = lens_map<NL, double>(eps, a, x) - wj;
  double res = sqrt(abs2(F));
  if (!(res <= img_tol)) return 0;
  cd z = x + sh.L.a[j];
  *r = sqrt(z.x * z.x + z.y * z.y);
  *th = atan2(z.y, z.x);
  return 1;
}

// FP64 offset of ray (i, l) of a sector from the source centre (and its
// distance below), with the grid of Sec. 3.3: r_i = r_lo + (i + 1/2) dr,
// th_l = th_lo + (l + 1/2) dth.  Out of line: these are the rare fallbacks,
// and inlined they cost the ray sweeps registers.
template <int NL>
__device__ __noinline__ cd ray_offset64(const Shared& sh, const Box& B, int i, int l) {
  double r = B.r_lo + (i + 0.5) * sh.dr64;
  double th = B.th_lo + (l + 0.5) * sh.dth64;
  double s, c;
  sincos(th, &s, &c);
  cd z = mk(r * c, r * s);
  return lens_map<NL, double>(sh.L.eps, sh.L.a, z) - sh.wc;
}
template <int NL>
__device__ __noinline__ double ray_distance64(const Shared& sh, const Box& B, int i, int l) {
  double r = B.r_lo + (i + 0.5) * sh.dr64;
  double th = B.th_lo + (l + 0.5) * sh.dth64;
  double s, c;
  sincos(th, &s, &c);
  cd z = mk(r * c, r * s);
  cd w = lens_map<NL, double>(sh.L.eps, sh.L.a, z);
  return sqrt(abs2(w - sh.wc));
}

// Tangents of an image-limb point z = r e^{i th} (the image of the source-limb
// point w_c + rho u) with respect to (t0, tE, u0, alpha, s, q, rho, u1), binary
// lens: the implicit derivative of the lens equation F(z; p) = f(z; p) - w(p)
// = 0, dz = -J^{-1} dF/dp at fixed z, J the real 2x2 Jacobian of f (the root
// derivative of Sec. 3.5, written for the lens equation rather than the
// polynomial so that it holds in any frame).  Returns d r / dp and d th / dp.
__device__ inline void point_tangents(const Shared& sh, const DerShared& ds, double r, double th, cd u, double* dr,
                                      double* dth) {
  double sn, cs;
  sincos(th, &sn, &cs);
  const cd z = mk(r * cs, r * sn);
  cd gm = mk(0.0, 0.0), cA[2], cE[2];
  for (int j = 0; j < 2; ++j) {
    cd iv = inv(z - sh.L.a[j]);
    cd iv2 = iv * iv;
    gm = gm + scl(iv2, sh.L.eps[j]);
    cA[j] = scl(cj(iv2), -sh.L.eps[j]);  // df/da_j.x = -eps_j / conj(z - a_j)^2
    cE[j] = scl(cj(iv), -1.0);           // df/deps_j = -1 / conj(z - a_j)
  }
  // df = dz + conj(gamma) conj(dz):  J = [[1 + g.x, -g.y], [-g.y, 1 - g.x]]
  const double j11 = 1.0 + gm.x, j12 = -gm.y, j22 = 1.0 - gm.x;
  const double det = j11 * j22 - j12 * j12;
  for (int q = 0; q < NPAR; ++q) {
    cd dF = mk(0.0, 0.0);
    if (q < 4) dF = scl(ds.dwc[q], -1.0);
    else if (q == 4) dF = scl(cA[0], ds.dadp[0][0]) + scl(cA[1], ds.dadp[1][0]);
    else if (q == 5) dF = scl(cA[0], ds.dadp[0][1]) + scl(cA[1], ds.dadp[1][1]) + scl(cE[0], ds.depsq[0]) + scl(cE[1], ds.depsq[1]);
    else if (q == 6) dF = scl(u, -1.0);
    double dx = -(j22 * dF.x - j12 * dF.y) / det;
    double dy = -(-j12 * dF.x + j11 * dF.y) / det;
    dr[q] = (z.x * dx + z.y * dy) / r;
    dth[q] = (z.x * dy - z.y * dx) / (r * r);
  }
}

// Lagrange basis of the nodes 0 .. npt-1 (npt = 2..4) at t, and the slope
// of the interpolant through y there.
template <class T>
__device__ inline T lagrange_basis(const T* y, int npt, T t, T* l) {
  const T d1 = y[1] - y[0];
  const T d2 = npt > 2 ? T(0.5) * (y[2] - T(2) * y[1] + y[0]) : T(0);
  const T d3 = npt > 3 ? (y[3] - T(3) * y[2] + T(3) * y[1] - y[0]) * T(1.0 / 6.0) : T(0);
  const T t1 = t - T(1), t2 = t - T(2), t3 = t - T(3);
  if (npt == 4) {
    l[0] = -t1 * t2 * t3 * T(1.0 / 6.0);
    l[1] = T(0.5) * t * t2 * t3;
    l[2] = T(-0.5) * t * t1 * t3;
    l[3] = t * t1 * t2 * T(1.0 / 6.0);
  } else if (npt == 3) {
    l[0] = T(0.5) * t1 * t2;
    l[1] = -t * t2;
    l[2] = T(0.5) * t * t1;
  } else {
    l[0] = -t1;
    l[1] = t;
  }
  return d1 + (T(2) * t - T(1)) * d2 + ((T(3) * t - T(6)) * t + T(2)) * d3;
}

// FP64 re-solve of limb point k (all roots, FP64 Ehrlich-Aberth warm-started
// from the FP32 roots in the lightest lens's frame, FP64 validation of each
// root); rewrites the point's slots and returns its image count.  Kept out of
// line: it runs only for limb points with an illegal FP32 image count.
template <int NL>
__device__ __noinline__ int resolve_limb_point64(Shared& sh, int k, int K, int max_iter, double img_tol, int PMAX,
                                                 cf* phi, float* r32, float* rl32, float* t32, float* e32, short* pidx,
                                                 uint8_t* meta, double* pr, double* pt) {
  constexpr int N = NL * NL + 1;
  const int ll = sh.L.ll;
  const cd w = limb_point64(sh, k, K);
  double eps[NL];
  cd a[NL], D[NL + 1], Ee[NL], b[N + 1], z[N];
  for (int i2 = 0; i2 < NL; ++i2) { eps[i2] = sh.L.eps[i2]; a[i2] = sh.L.a[i2] - sh.L.a[ll]; }
  poly_DE<NL, double>(eps, a, D, Ee);
  lens_poly<NL, double>(eps, a, D, Ee, w - sh.L.a[ll], b);
  for (int j = 0; j < N; ++j) z[j] = tod(phi[k * N + j]);
  // separate coincident starts
  for (int j = 1; j < N; ++j)
    for (int i2 = 0; i2 < j; ++i2)
      if (abs2(z[j] - z[i2]) < 1e-20) z[j] = z[j] + mk(1e-7 * (j + 1), 1e-7 * j);
  if (ehrlich_aberth_f64<N>(b, z, max_iter) < 0) atomicOr(&sh.status, ICRS_ST_NONCONV);
  int m = 0;
  for (int j = 0; j < N; ++j) {
    const int ps = k * N + j;
    phi[ps] = tof(z[j]);
    pidx[ps] = -1;
    uint8_t mm = 0;
    double r, th;
    if (validate_root64<NL>(sh, z[j] + sh.L.a[ll], w, img_tol, &r, &th)) {
      const int pi = atomicAdd(&sh.pn, 1);
      const float rh = (float)r;
      r32[ps] = rh; rl32[ps] = (float)(r - (double)rh); t32[ps] = (float)th;
      if (pi < PMAX) { pr[pi] = r; pt[pi] = th; pidx[ps] = (short)pi; e32[ps] = 0.f; mm = M_VALID | M_EXACT; }
      else { e32[ps] = 1e-12f; mm = M_VALID; atomicOr(&sh.status, ICRS_ST_OVERFLOW); }
      ++m;
    }
    meta[ps] = mm;
  }
  return m;
}

// ---------------------------------------------------------------- queue
__device__ __forceinline__ void q_push(Shared& sh, int* queue, int v) {
  int i = atomicAdd(&sh.qn, 1);
  if (i < QMAX) queue[i] = v;
  else atomicOr(&sh.status, ICRS_ST_OVERFLOW);
}

// ---------------------------------------------------------------- quadrature
// Crossing of the interpolated distance with rho.  The stencil nodes are
// consecutive integers x0, x0+1, ... (npt = 2..4), so the interpolant is
// written in Newton's forward-difference form (the same polynomial as the
// Lagrange form of Appendix A, without divisions).  The root on the bracket
// between the inside sample (offset 0, p < rho) and the outside sample
// (x_out = +-1, p >= rho) is found by the Illinois variant of regula falsi,
// which keeps the bracket and converges superlinearly.
template <class T>
__device__ inline T crossing_solve(const T* y, T x0, int npt, T yin, T yout, T x_out, T rho, T tol, int iters) {
  const T d1 = y[1] - y[0];
  const T d2 = npt > 2 ? T(0.5) * (y[2] - T(2) * y[1] + y[0]) : T(0);
  const T d3 = npt > 3 ? (y[3] - T(3) * y[2] + T(3) * y[1] - y[0]) * T(1.0 / 6.0) : T(0);
  T a = T(0), ga = yin - rho;      // inside end  (g < 0)
  T b = x_out, gb = yout - rho;    // outside end (g >= 0)
  int side = 0;
  for (int it = 0; it < iters; ++it) {
    T den = gb - ga;
    T c = (den != T(0)) ? b - gb * (b - a) / den : T(0.5) * (a + b);
    T t = c - x0;
    T gc = y[0] + t * (d1 + (t - T(1)) * (d2 + (t - T(2)) * d3)) - rho;
    if (gc == T(0)) return c;
    if ((gc < T(0)) == (gb < T(0))) {
      b = c; gb = gc;
      if (side == -1) ga *= T(0.5);
      side = -1;
    } else {
      a = b; ga = gb;
      b = c; gb = gc;
      side = 1;
    }
    if (fabs(b - a) < tol) break;
  }
  return b;
}

// LD correction f(delta) (Appendix A.2) or the uniform rule delta + 1/2.
template <class T>
__device__ __forceinline__ T fdelta(T d, T delta_c, int uniform) {
  if (uniform) return d + T(0.5);
  if (d >= delta_c) return (T(0.5) + d) * (T(2.0 / 3.0) * sqrt(T(1) + T(1) / (T(2) * d)));
  return T(2.0 / 3.0) * d + T(0.5);
}

// f'(delta) of the rule above.
template <class T>
__device__ __forceinline__ T fdelta_prime(T d, T delta_c, int uniform) {
  if (uniform) return T(1);
  if (d >= delta_c) {
    T h = T(1) + T(1) / (T(2) * d);
    T sq = sqrt(h);
    return T(2.0 / 3.0) * sq - (T(0.5) + d) / (T(6) * d * d * sq);
  }
  return T(2.0 / 3.0);
}

// ---------------------------------------------------------------- kernel
// A set whose law has half-integer powers of mu (a1 or a3, on a limb-darkened
// grid) or a spot: the binary forward launch gives these sets to the kernel's
// generic instantiation and all others to the linear one, which carries none
// of their code.
__device__ inline bool generic_law(const icrs_params& p, const icrs_grid& g) {
  return p.spot_c != 0.0 || (!g.uniform && (p.a1 != 0.0 || p.a3 != 0.0));
}

// LAW = 0: only the sets without a generic law (their code compiled out);
// LAW = 1: only the sets with one; LAW = 2: every set, the law decided at run
// time.
// DER = true: also the derivative of A with respect to (t0, tE, u0, alpha, s,
// q, rho, u1) (binary lens): reverse mode over the rays (adjoint seeds per
// ray, then each seeded ray's gradient), forward mode (8 tangents) over the
// sector bounds via the implicit derivative of the extremal image points.
struct DerOut {
  const double* gA;    // [S][E] upstream dL/dA, or NULL
  const double* yobs;  // [S][E] data for chi^2 (with sig), or NULL
  const double* sig;   // [S][E]
  double* dA;          // [S][E][8] or NULL
  double* grad;        // [S][8] accumulated, or NULL
  double* chi2;        // [S] accumulated, or NULL
};

template <int NL, bool DER, int NTB, int LAW>
__global__ void __launch_bounds__(NTB, 1)
mag_kernel(const icrs_params* __restrict__ P, int S, const double* __restrict__ T_, int E,
           icrs_grid g, int tiles_per_block, double* __restrict__ A_out, uint32_t* __restrict__ st_out,
           double* __restrict__ diag_sect, int32_t* __restrict__ diag_cnt, float* __restrict__ diag_pts, int PMAX,
           int has_plo, DerOut dout, const int32_t* __restrict__ items, int n_items, int defer) {
  constexpr int N = NL * NL + 1;
  constexpr int NT = NTB;
  constexpr int NW = NT / 32;
  static_assert(NT % 32 == 0 && NW <= NW_MAX && (!DER || NW == NW_DER), "per-warp tables are sized for these block sizes");
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ Shared sh;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = g.n_limb, NP = K * N;
  const int BT = g.n_bins_theta, BR = g.n_bins_r;
  const double ht = 2.0 * kPi / BT;

  // dynamic shared memory carve-up
  unsigned char* p = dyn;
  // per image-limb slot: root / refined image position in the lightest
  // lens's frame (also the next epoch's warm start), FP32 (r, theta), FP32
  // error bound, flags, bins, index into the FP64 table
  cf* phi = (cf*)p;              p += sizeof(cf) * NP;
  cf* plo = (cf*)p;              p += has_plo ? sizeof(cf) * NP : 0;   // lo part of refined positions
  float* r32 = (float*)p;        p += sizeof(float) * NP;
  float* rl32 = (float*)p;       p += sizeof(float) * NP;   // r = r32 + rl32 (double-float)
  float* t32 = (float*)p;        p += sizeof(float) * NP;
  float* e32 = (float*)p;        p += sizeof(float) * NP;
  short* pidx = (short*)p;       p += sizeof(short) * ((NP + 7) & ~7);
  uint8_t* meta = (uint8_t*)p;   p += (NP + 15) & ~15;
  uint8_t* tb = (uint8_t*)p;     p += (NP + 15) & ~15;
  uint8_t* rb = (uint8_t*)p;     p += (NP + 15) & ~15;
  double* pr = (double*)p;       p += sizeof(double) * PMAX;
  double* pt = (double*)p;       p += sizeof(double) * PMAX;
  int* queue = (int*)p;          p += sizeof(int) * QMAX;
  p = (unsigned char*)(((uintptr_t)p + 15) & ~(uintptr_t)15);  // 16-byte rows of the offset table
  AnchorF* anch = (AnchorF*)p;   p += sizeof(AnchorF) * MAXANCH;
  float2* spc = (float2*)p;      p += sizeof(float2) * MAXANCH;  // spot centre in each anchor's frame
  cf* tab = (cf*)p;              p += sizeof(cf) * (GTH_MAX + 2);  // group offsets (cos d - 1, sin d)
  cdf* ulimb = (cdf*)p;          p += sizeof(cdf) * K;   // e^{2 pi i k / N_limb} as double-float
  // boundary points: a deferred queue per warp of (column, row) pairs
  (void)defer;
  int* wqueue = (int*)p;         p += sizeof(int) * NW * 2 * dq_entries(NL);
  // derivative mode: its state
  DerShared& ds = *(DerShared*)p;  p += DER ? sizeof(DerShared) : 0;
  DualD* cdual = ds.cx;
  BoxT<DualD>* bdual = ds.box;
  double* wder = &ds.wder[0][0];

  if (tid == 0) { sh.cur_set = -1; sh.warm = 0; }
  for (int k = tid; k < K; k += NT) {
    double sn, cs;
    sincospi(2.0 * (double)k / (double)K, &sn, &cs);
    ulimb[k].x = df_from_double(cs);
    ulimb[k].y = df_from_double(sn);
  }
  __syncthreads();

  // tiles: all (set, epoch) pairs, or the listed indices s * E + e
  const long long ntiles = items ? (long long)n_items : (long long)S * E;
  const long long t_begin = (long long)blockIdx.x * tiles_per_block;
  int law_set = -1;
  bool law_gen = false;
  for (long long tile = t_begin; tile < t_begin + tiles_per_block && tile < ntiles; ++tile) {
    long long q = items ? (long long)items[tile] : tile;
    if (q < 0 || q >= (long long)S * E) continue;  // block-uniform: skips the whole tile
    const int s = (int)(q / E), e = (int)(q % E);
    if constexpr (LAW != 2) {
      // the other instantiation takes this set (block-uniform)
      if (s != law_set) { law_set = s; law_gen = generic_law(P[s], g); }
      if (law_gen != (LAW == 1)) continue;
    }
    // ------------------------------------------------ set and epoch set-up
    if (tid == 0) {
      if (s != sh.cur_set) {
        icrs_params prm = P[s];
        sh.L = make_lens(prm);
        sh.rho = prm.rho;
        sh.u1 = prm.u1;
        sh.u2 = prm.u2;
        sh.pa[0] = prm.a1; sh.pa[1] = prm.a2; sh.pa[2] = prm.a3; sh.pa[3] = prm.a4;
        sh.spot = prm.spot_c != 0.0;
        sh.spot_x = prm.spot_x; sh.spot_y = prm.spot_y; sh.spot_r = prm.spot_r; sh.spot_c = prm.spot_c;
        sh.spot_bad = sh.spot && !(prm.spot_r >= 0.0 && prm.spot_c < 1.0 &&
                                   hypot(prm.spot_x, prm.spot_y) + prm.spot_r <= 1.0);
        sh.spot_new = sh.spot && !sh.spot_bad;
        sh.spot_norm = 1.0;
        sh.spot_gu = 0.0;
        sh.spot_acc[0] = sh.spot_acc[1] = 0.0;
        for (int j = 0; j < NL; ++j) {
          sh.eps32[j] = (float)sh.L.eps[j];
          double eps[NL];
          cd a[NL], D[NL + 1], Ee[NL];
          for (int i = 0; i < NL; ++i) { eps[i] = sh.L.eps[i]; a[i] = sh.L.a[i] - sh.L.a[j]; sh.aj32[j][i] = tof(a[i]); }
          poly_DE<NL, double>(eps, a, D, Ee);
          for (int i = 0; i <= NL; ++i) sh.D32[j][i] = tof(D[i]);
          for (int i = 0; i < NL; ++i) sh.E32[j][i] = tof(Ee[i]);
          for (int i = 0; i < NL; ++i) { sh.adf[j][i][0] = df_from_double(a[i].x); sh.adf[j][i][1] = df_from_double(a[i].y); }
          sh.epsdf[j] = df_from_double(sh.L.eps[j]);
        }
        sh.l2 = -1;
        if (NL == 3) {
          int c2 = -1;
          for (int i = 0; i < 3; ++i) {
            if (i == sh.L.ll) continue;
            if (c2 < 0 || sh.L.eps[i] < sh.L.eps[c2]) c2 = i;
          }
          sh.l2 = c2;
        }
        sh.adf_ll[0] = df_from_double(sh.L.a[sh.L.ll].x);
        sh.adf_ll[1] = df_from_double(sh.L.a[sh.L.ll].y);
        sh.rhodf = df_from_double(prm.rho);
        sh.warm = 0;
        sh.cur_set = s;
      } else {
        sh.warm = 1;  // previous tile of this block was the previous epoch of this set
        sh.spot_new = 0;
      }
      sh.wc = source_centre(P[s], T_[(size_t)s * E + e]);
      if (DER) {
        // d w_c / d(t0, tE, u0, alpha) and d(a_j, eps_j) / d(s, q) (binary):
        // w_c = tau (cos a, sin a) + u0 (-sin a, cos a), tau = (t - t0) / tE;
        // a_1 = -q s / (1 + q), a_2 = s / (1 + q), eps_1 = 1 / (1 + q),
        // eps_2 = q / (1 + q)
        const icrs_params& pp = P[s];
        double tau = (T_[(size_t)s * E + e] - pp.t0) / pp.tE;
        double sa, ca;
        sincos(pp.alpha, &sa, &ca);
        ds.dwc[0] = mk(-ca / pp.tE, -sa / pp.tE);
        ds.dwc[1] = mk(-tau * ca / pp.tE, -tau * sa / pp.tE);
        ds.dwc[2] = mk(-sa, ca);
        ds.dwc[3] = mk(-tau * sa - pp.u0 * ca, tau * ca - pp.u0 * sa);
        double oq = 1.0 + pp.q;
        ds.dadp[0][0] = -pp.q / oq;  ds.dadp[0][1] = -pp.s / (oq * oq);
        ds.dadp[1][0] = 1.0 / oq;    ds.dadp[1][1] = -pp.s / (oq * oq);
        ds.depsq[0] = -1.0 / (oq * oq);
        ds.depsq[1] = 1.0 / (oq * oq);
        for (int b = 0; b < MAXBOX_D; ++b) for (int k = 0; k < 4; ++k) ds.Gb[b][k] = 0.0;
        for (int k = 0; k < 8; ++k) ds.H[k] = 0.0;
      }
      for (int j = 0; j < NL; ++j) {
        cd d = sh.wc - sh.L.a[j];
        sh.wcj32[j] = tof(d);
        sh.wcdf[j][0] = df_from_double(d.x);
        sh.wcdf[j][1] = df_from_double(d.y);
      }
      sh.status = 0u;
      sh.qn = 0;
      sh.pn = 0;
      for (int c = 0; c < 16; ++c) sh.cnt[c] = 0;
      sh.clk0 = clock64();
      sh.tocc[0] = sh.tocc[1] = 0ull;
    }
    __syncthreads();
    const int ll = sh.L.ll;
    const float rho32 = (float)sh.rho;
    if (LAW != 0 && sh.spot_new) {
      // the spot's share of the unspotted flux F_spot = int_spot I dA (rho
      // units, the disk's flux is 1) and dF_spot/du1, once per set: polar
      // quadrature about the spot centre, the periodic trapezoid rule in the
      // angle (64 nodes), 8-point Gauss-Legendre in the radius on 16 panels
      // graded geometrically toward the spot's edge
      double gx[8], gw[8];
      for (int i = 0; i < 8; ++i) {
        double z = cos(kPi * (i + 0.75) / 8.5), dp = 1.0;
        for (int it = 0; it < 60; ++it) {
          double p0 = 1.0, p1 = z;
          for (int k = 2; k <= 8; ++k) { const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
          dp = 8.0 * (z * p1 - p0) / (z * z - 1.0);
          const double dz = p1 / dp;
          z -= dz;
          if (fabs(dz) < 1e-15) break;
        }
        gx[i] = z;
        gw[i] = 2.0 / ((1.0 - z * z) * dp * dp);
      }
      const double sa = sh.pa[0] / 5.0 + sh.pa[1] * (2.0 / 6.0) + sh.pa[2] * (3.0 / 7.0) + sh.pa[3] * 0.5;
      const double I0d = g.uniform ? 1.0 / kPi : 1.0 / (kPi * (1.0 - sh.u1 / 3.0 - sh.u2 / 6.0 - sa));
      double f = 0.0, fu = 0.0;
      for (int idx = tid; idx < 16 * 8 * 64; idx += NT) {
        const int b = idx / 512, i = (idx / 64) & 7, j = idx & 63;
        const double lo = b == 0 ? 0.0 : sh.spot_r * (1.0 - ldexp(1.0, -b));
        const double hi = b == 15 ? sh.spot_r : sh.spot_r * (1.0 - ldexp(1.0, -(b + 1)));
        const double rr = 0.5 * (hi - lo) * gx[i] + 0.5 * (hi + lo);
        const double w_ = 0.5 * (hi - lo) * gw[i] * rr * (2.0 * kPi / 64.0);
        double sn_, cs_;
        sincospi(2.0 * j / 64.0, &sn_, &cs_);
        const double x = sh.spot_x + rr * cs_, y = sh.spot_y + rr * sn_;
        const double mu = sqrt(fmax(1.0 - (x * x + y * y), 0.0));
        double I = 1.0, Iu = 0.0;
        if (!g.uniform) {
          const double om = 1.0 - mu, sq = sqrt(mu);
          I = 1.0 - sh.u1 * om - sh.u2 * om * om - sh.pa[0] * (1.0 - sq) - sh.pa[1] * (1.0 - mu) -
              sh.pa[2] * (1.0 - sq * mu) - sh.pa[3] * (1.0 - mu * mu);
          // dI/du1 = (pi/3) I0 I - I0 (1 - mu), with I = I0 x the bracket
          Iu = (kPi / 3.0) * I0d * I0d * I - I0d * om;
        }
        f += w_ * I0d * I;
        fu += w_ * Iu;
      }
      for (int o = 16; o > 0; o >>= 1) {
        f += __shfl_xor_sync(0xffffffffu, f, o);
        fu += __shfl_xor_sync(0xffffffffu, fu, o);
      }
      if (lane == 0) { atomicAdd(&sh.spot_acc[0], f); atomicAdd(&sh.spot_acc[1], fu); }
      __syncthreads();
      if (tid == 0) {
        // A = N S / rho^2, N = 1 / (1 - c F_spot): dN/du1 = N^2 c dF/du1,
        // so dA/du1 gains A N c dF/du1 (spot_gu)
        sh.spot_norm = 1.0 / (1.0 - sh.spot_c * sh.spot_acc[0]);
        sh.spot_gu = sh.spot_norm * sh.spot_c * sh.spot_acc[1];
      }
      __syncthreads();
    }

    // ------------------------------------------------ 1. limb roots (FP32 EA)
    // Cold start: 32 anchor limb points from the Cauchy circle, then every
    // limb point from its nearest anchor; warm start: from the same limb
    // point of the previous epoch.
    const bool warm = sh.warm;
    const int nanc = K < 32 ? K : 32;
    if (!warm) {
      if (warp == 0 && lane < nanc) {
        int k = (int)(((long long)lane * K) / nanc);
        float sp, cp;
        sincospif(2.0f * (float)k / (float)K, &sp, &cp);
        cf w = mk(sh.wcj32[ll].x + rho32 * cp, sh.wcj32[ll].y + rho32 * sp);
        cf b[N + 1];
        lens_poly<NL, float>(sh.eps32, sh.aj32[ll], sh.D32[ll], sh.E32[ll], w, b);
        cf z[N];
        float last[N];
        cauchy_start<N>(b, z);
        int it = ehrlich_aberth_f32<N>(b, z, g.max_iter, 4.0f * EPS32, last);
        if (it < 0) atomicOr(&sh.status, ICRS_ST_NONCONV);
        for (int j = 0; j < N; ++j) sh.anc[lane][j] = z[j];
      }
      __syncthreads();
    }
    for (int k = tid; k < K; k += NT) {
      float sp = ulimb[k].y.hi, cp = ulimb[k].x.hi;
      cf w = mk(sh.wcj32[ll].x + rho32 * cp, sh.wcj32[ll].y + rho32 * sp);
      cf b[N + 1];
      lens_poly<NL, float>(sh.eps32, sh.aj32[ll], sh.D32[ll], sh.E32[ll], w, b);
      cf z[N];
      if (warm) {
        for (int j = 0; j < N; ++j) z[j] = phi[k * N + j];
      } else {
        int a = (int)(((long long)k * nanc + K / 2) / K);
        if (a >= nanc) a = nanc - 1;
        for (int j = 0; j < N; ++j) z[j] = sh.anc[a][j];
      }
      // separate coincident starts
      for (int j = 1; j < N; ++j)
        for (int i = 0; i < j; ++i)
          if (abs2(z[j] - z[i]) < 1e-24f) z[j] = z[j] + mk(1e-6f * (j + 1), 1e-6f * j);
      float last[N];
      int it = ehrlich_aberth_f32<N>(b, z, g.max_iter, 4.0f * EPS32, last);
      if (it < 0) {
        // fall back to a cold start
        cauchy_start<N>(b, z);
        it = ehrlich_aberth_f32<N>(b, z, g.max_iter, 4.0f * EPS32, last);
        if (it < 0) atomicOr(&sh.status, ICRS_ST_NONCONV);
      }
      // Candidate roots (frame f, position in that frame).  Triple lens: the
      // polynomial about the lightest lens cannot resolve the cluster of
      // roots beside the second light lens in FP32, so a second EA about
      // that lens (warm-started from the first) supplies the roots nearest
      // to it.
      cf cz[2 * N];
      signed char cfm[2 * N];
      int nc = 0;
      const int l2 = sh.l2;
      cf z2[N];
      if (NL == 3) {
        cf w2 = w - sh.aj32[ll][l2];
        cf b2[N + 1];
        lens_poly<NL, float>(sh.eps32, sh.aj32[l2], sh.D32[l2], sh.E32[l2], w2, b2);
        for (int j = 0; j < N; ++j) z2[j] = z[j] - sh.aj32[ll][l2];
        float last2[N];
        if (ehrlich_aberth_f32<N>(b2, z2, g.max_iter, 4.0f * EPS32, last2) < 0) atomicOr(&sh.status, ICRS_ST_NONCONV);
      }
      for (int j = 0; j < N; ++j) {
        int nj = ll;
        float best = abs2(z[j]);
        for (int i = 0; i < NL; ++i) {
          if (i == ll) continue;
          float d = abs2(z[j] - sh.aj32[ll][i]);
          if (d < best) { best = d; nj = i; }
        }
        if (NL == 3 && nj == l2) continue;
        cz[nc] = z[j]; cfm[nc] = (signed char)ll; ++nc;
      }
      int n1 = nc;  // candidates from the first frame
      if (NL == 3) {
        for (int j = 0; j < N; ++j) {
          int nj = l2;
          float best = abs2(z2[j]);
          for (int i = 0; i < NL; ++i) {
            if (i == l2) continue;
            float d = abs2(z2[j] - sh.aj32[l2][i]);
            if (d < best) { best = d; nj = i; }
          }
          if (nj != l2) continue;
          cz[nc] = z2[j]; cfm[nc] = (signed char)l2; ++nc;
        }
      }
      // The two frames can disagree about which roots lie nearest the
      // second light lens (a root by a cell boundary, kept from both): drop
      // the first-frame candidate closest to a second-frame one, which
      // resolves that cluster better, until N remain.
      while (NL == 3 && nc > N && n1 > 0) {
        int bi = 0;
        float bd = __int_as_float(0x7f800000);
        for (int i = 0; i < n1; ++i)
          for (int j = n1; j < nc; ++j) {
            const float d = abs2(cz[i] - (cz[j] + sh.aj32[ll][l2]));
            if (d < bd) { bd = d; bi = i; }
          }
        for (int i = bi; i < nc - 1; ++i) { cz[i] = cz[i + 1]; cfm[i] = cfm[i + 1]; }
        --nc;
        --n1;
      }
      if (nc > N) { atomicOr(&sh.status, ICRS_ST_OVERFLOW); nc = N; }
      const float img_tol = (float)g.img_tol;
      for (int j = 0; j < N; ++j) {
        int pslot = k * N + j;
        meta[pslot] = 0;
        pidx[pslot] = -1;
        e32[pslot] = 0.f;
        if (j >= nc) {
          // unused slot (triple, fewer candidates): keep a warm start
          phi[pslot] = z[j];
          continue;
        }
        const int f = cfm[j];
        const cf zf = cz[j];
        // position in the lightest lens's frame (warm start for the next epoch)
        phi[pslot] = (f == ll) ? zf : zf + sh.aj32[ll][f];
        // nearest lens, offset x in its frame
        int nj = f;
        float best = abs2(zf);
        for (int i = 0; i < NL; ++i) {
          if (i == f) continue;
          float d = abs2(zf - sh.aj32[f][i]);
          if (d < best) { best = d; nj = i; }
        }
        cf x = (nj == f) ? zf : zf - sh.aj32[f][nj];
        cf wj = w - sh.aj32[ll][nj];
        // FP32 screen: roots whose residual is far above img_tol are not images
        cf F32 = lens_map<NL, float>(sh.eps32, sh.aj32[nj], x) - wj;
        float noise = 0.f;
        for (int i = 0; i < NL; ++i) noise += sh.eps32[i] * rsqrtf(fmaxf(abs2(x - sh.aj32[nj][i]), 1e-37f));
        noise = 16.0f * EPS32 * (noise + sqrtf(abs2(x)) + sqrtf(abs2(wj)) + 1.0f);
        float res32 = sqrtf(abs2(F32));
        if (res32 == res32 && res32 - noise > 4.0f * img_tol) continue;
        // compensated residual F = x - sum eps_i (x - a_i)/|x - a_i|^2 - w in
        // double-float (frame of lens nj), then one Newton step in FP32
        df wx = df_add(sh.wcdf[nj][0], df_mul(sh.rhodf, ulimb[k].x));
        df wy = df_add(sh.wcdf[nj][1], df_mul(sh.rhodf, ulimb[k].y));
        df Fx = df_make(x.x, 0.f), Fy = df_make(x.y, 0.f);
        for (int i = 0; i < NL; ++i) {
          df dx = df_sub(df_make(x.x, 0.f), sh.adf[nj][i][0]);
          df dy = df_sub(df_make(x.y, 0.f), sh.adf[nj][i][1]);
          df nn = df_add(df_mul(dx, dx), df_mul(dy, dy));
          df tt = df_div(sh.epsdf[i], nn);
          Fx = df_sub(Fx, df_mul(dx, tt));
          Fy = df_sub(Fy, df_mul(dy, tt));
        }
        Fx = df_sub(Fx, wx);
        Fy = df_sub(Fy, wy);
        cf F = mk(Fx.hi + Fx.lo, Fy.hi + Fy.lo);
        float res = sqrtf(abs2(F));
        // position kept for an FP64 decision if needed
        // position of this root in the lightest lens's frame, double-float:
        // x (exact float) + (a_nj - a_ll) (double-float)
        df px = df_add(df_make(x.x, 0.f), sh.adf[ll][nj][0]);
        df py = df_add(df_make(x.y, 0.f), sh.adf[ll][nj][1]);
        if (!(res == res) || res > 0.25f * img_tol) {
          if (!(res >= 4.0f * img_tol)) {  // FP64 decides
            meta[pslot] = M_UNSURE;
            phi[pslot] = mk(px.hi, py.hi);
          }
          continue;
        }
        cf gm = shear<NL, float>(sh.eps32, sh.aj32[nj], x);
        float ag2 = abs2(gm), ag = sqrtf(ag2);
        float det = 1.0f - ag2;
        float jinv = (1.0f + ag) / fmaxf(fabsf(det), 1e-30f);
        cf dz = scl(cj(gm) * cj(F) - F, 1.0f / det);
        // second-derivative scale |dgamma/dz| = |sum 2 eps_i/(x - a_i)^3|
        cf g3 = mk(0.f, 0.f);
        for (int i = 0; i < NL; ++i) { cf id = inv(x - sh.aj32[nj][i]); g3 = g3 + scl(id * id * id, 2.0f * sh.eps32[i]); }
        float adz2 = abs2(dz);
        // refined position: a_nj + x + dz (lightest frame: aj32[ll][nj] + x + dz)
        px = df_add(px, df_make(dz.x, 0.f));
        py = df_add(py, df_make(dz.y, 0.f));
        df zx = df_add(px, sh.adf_ll[0]);
        df zy = df_add(py, sh.adf_ll[1]);
        float zxf = zx.hi + zx.lo, zyf = zy.hi + zy.lo;
        // r = |z| as a double-float: r^2 in double-float, then one Newton
        // correction of the float square root
        df r2 = df_add(df_mul(zx, zx), df_mul(zy, zy));
        float rr = sqrtf(r2.hi);
        df rsq = two_prod(rr, rr);
        float rlo = ((r2.hi - rsq.hi) - rsq.lo + r2.lo) / (2.0f * rr);
        float th = atan2f(zyf, zxf);
        // error bound of the double-float r after the step: second-order Newton
        // term plus the double-float residual's rounding
        float ee = 4.0f * sqrtf(abs2(g3)) * adz2 * jinv + jinv * 1e-12f * (1.0f + noise / (16.0f * EPS32)) +
                   1e-12f * rr;
        if (!(rr == rr) || !(th == th) || !(ee == ee) || isinf(ee)) {
          meta[pslot] = M_UNSURE;
          phi[pslot] = mk(px.hi, py.hi);
          continue;
        }
        meta[pslot] = M_VALID;
        phi[pslot] = mk(px.hi, py.hi);
        if (has_plo) plo[pslot] = mk(px.lo, py.lo);
        r32[pslot] = rr;
        rl32[pslot] = rlo;
        t32[pslot] = th;
        e32[pslot] = ee;
      }
    }
    __syncthreads();

    if (diag_cnt && tid == 0) { long long c_ = clock64(); sh.cnt[4] = (int)min(c_ - sh.clk0, 2000000000LL); sh.clk0 = c_; }
    // ------------------------------------------------ 1b. ambiguous roots in FP64
    for (int ps = tid; ps < NP; ps += NT)
      if (meta[ps] & M_UNSURE) q_push(sh, queue, ps);
    __syncthreads();
    {
      int qn = min(sh.qn, QMAX);
      for (int qi = tid; qi < qn; qi += NT) {
        int ps = queue[qi];
        int k = ps / N;
        atomicAdd(&sh.cnt[1], 1);
        cd w = limb_point64(sh, k, K);
        cd z0 = tod(phi[ps]) + sh.L.a[ll];
        double r, th;
        int conv = 1;
        int ok = validate_root64<NL>(sh, z0, w, g.img_tol, &r, &th, &conv);
        uint8_t m = 0;
        if (ok && NL == 2 && !conv) {
          // not converged: kept as an image with an infinite error bound, so
          // that the limb point goes to the FP64 re-solve below
          m = M_VALID;
          const float rh = (float)r;
          r32[ps] = rh; rl32[ps] = (float)(r - (double)rh); t32[ps] = (float)th;
          e32[ps] = __int_as_float(0x7f800000);
        } else if (ok) {
          int pi = atomicAdd(&sh.pn, 1);
          float rh = (float)r;
          if (pi < PMAX) { pr[pi] = r; pt[pi] = th; pidx[ps] = (short)pi; m = M_VALID | M_EXACT; r32[ps] = rh; rl32[ps] = (float)(r - (double)rh); t32[ps] = (float)th; e32[ps] = 0.f; }
          else { m = M_VALID; atomicOr(&sh.status, ICRS_ST_OVERFLOW); r32[ps] = rh; rl32[ps] = (float)(r - (double)rh); t32[ps] = (float)th; e32[ps] = 1e-12f; }
        }
        meta[ps] = m;
      }
    }
    __syncthreads();
    if (tid == 0) sh.qn = 0;
    __syncthreads();
    // image counts per limb point; an illegal count sends the limb point to
    // an FP64 root solve (warm-started from its FP32 roots) and FP64
    // validation of every root
    auto legal_count = [&](int m) -> bool {
      return (NL == 2) ? (m == 3 || m == 5) : (m == 4 || m == 6 || m == 8 || m == 10);
    };
    // Binary lens: the same FP64 re-solve takes limb points whose FP32 image
    // set is not trustworthy although its count is legal: an image whose
    // refining Newton step left a large error bound (an approximation next to
    // a critical curve, where det J ~ 0 sends the step far away), two slots
    // holding the same image (two approximations that met at one root while
    // another image was missed), or two non-image roots within PAIR_TOL of
    // each other (a close image pair that the FP32 polynomial rounded into a
    // pair of false roots; seen at separations up to 5.5e-3).  Without this check the image set, and
    // so the sectors, could depend on where the iteration started.  (Triple
    // lens: images beside the small lenses have large second derivatives and
    // so large bounds, and the FP64 re-solve in the lightest lens's frame is
    // less accurate there than the two-frame FP32 solve; only illegal counts
    // are re-solved.)
    for (int k = tid; k < K; k += NT) {
      int m = 0;
      bool suspect = false;
      float zx[N], zy[N];
      if (NL == 2) {
        // two roots that are not images, close together: the FP32
        // coefficients may have turned a close image pair (a limb point just
        // inside a fold caustic) into a pair of false roots
        for (int j = 0; j < N; ++j) {
          if (meta[k * N + j] & M_VALID) continue;
          const cf a_ = phi[k * N + j];
          for (int i2 = 0; i2 < j; ++i2) {
            if (meta[k * N + i2] & M_VALID) continue;
            const float tol = PAIR_TOL * fmaxf(1.0f, sqrtf(abs2(a_) + 1e-30f));
            if (abs2(a_ - phi[k * N + i2]) <= tol * tol) suspect = true;
          }
        }
      }
      for (int j = 0; j < N; ++j) {
        const int ps = k * N + j;
        if (!(meta[ps] & M_VALID)) continue;
        const bool ex = meta[ps] & M_EXACT;
        const float r = ex ? (float)pr[pidx[ps]] : r32[ps];
        const float th = ex ? (float)pt[pidx[ps]] : t32[ps];
        if (!ex && !(e32[ps] <= EE_SUSPECT * fmaxf(1.0f, r))) suspect = true;
        float sn, cs;
        sincosf(th, &sn, &cs);
        const float x = r * cs, y = r * sn;
        for (int i2 = 0; i2 < m; ++i2) {
          const float dx = x - zx[i2], dy = y - zy[i2];
          const float tol = DUP_TOL * fmaxf(1.0f, r);
          if (dx * dx + dy * dy <= tol * tol) suspect = true;
        }
        zx[m] = x; zy[m] = y;
        ++m;
      }
      if (!legal_count(m) || (NL == 2 && suspect)) q_push(sh, queue, k);
    }
    __syncthreads();
    {
      const int qn = min(sh.qn, QMAX);
      for (int qi = tid; qi < qn; qi += NT) {
        const int k = queue[qi];
        atomicAdd(&sh.cnt[1], 1);
        const int m = resolve_limb_point64<NL>(sh, k, K, g.max_iter, g.img_tol, PMAX, phi, r32, rl32, t32, e32, pidx,
                                               meta, pr, pt);
        if (!legal_count(m)) atomicOr(&sh.status, ICRS_ST_IMGCOUNT);
      }
    }
    __syncthreads();
    if (tid == 0) sh.qn = 0;
    __syncthreads();

    // polish helper: process the queue (points not yet exact)
    auto run_polish = [&]() {
      __syncthreads();
      int qn = min(sh.qn, QMAX);
      for (int qi = tid; qi < qn; qi += NT) {
        int ps = queue[qi];
        if (meta[ps] & M_EXACT) continue;
        int k = ps / N;
        atomicAdd(&sh.cnt[0], 1);
        double r, th;
        if (has_plo && e32[ps] <= 1e-11f) {
          // the double-float position is already accurate to ~1e-12
          cd z0 = mk((double)phi[ps].x + (double)plo[ps].x, (double)phi[ps].y + (double)plo[ps].y) + sh.L.a[ll];
          r = sqrt(z0.x * z0.x + z0.y * z0.y);
          th = atan2(z0.y, z0.x);
        } else {
          cd w = limb_point64(sh, k, K);
          cd z0 = tod(phi[ps]) + sh.L.a[ll];
          polish_image64<NL>(sh, z0, w, &r, &th);
        }
        int pi = atomicAdd(&sh.pn, 1);
        if (pi < PMAX) {
          pr[pi] = r; pt[pi] = th; pidx[ps] = (short)pi;
          float rh = (float)r;
          r32[ps] = rh; rl32[ps] = (float)(r - (double)rh); t32[ps] = (float)th; e32[ps] = 0.f;
          meta[ps] |= M_EXACT;
        } else {
          atomicOr(&sh.status, ICRS_ST_OVERFLOW);
        }
      }
      __syncthreads();
      if (tid == 0) sh.qn = 0;
      __syncthreads();
    };
    // r of a slot: FP64 if polished, else the double-float (r32 + rl32)
    auto rv = [&](int ps) -> double { return (meta[ps] & M_EXACT) ? pr[pidx[ps]] : (double)r32[ps] + (double)rl32[ps]; };
    auto tv = [&](int ps) -> double { return (meta[ps] & M_EXACT) ? pt[pidx[ps]] : (double)t32[ps]; };

    if (diag_pts) {
      size_t o = ((size_t)s * E + e) * (size_t)NP;
      for (int ps = tid; ps < NP; ps += NT) {
        float* d = diag_pts + (o + ps) * 4;
        bool ex = meta[ps] & M_EXACT;
        if (meta[ps] & M_VALID) {
          d[0] = ex ? (float)pr[pidx[ps]] : r32[ps];
          d[1] = ex ? (float)pt[pidx[ps]] : t32[ps];
        } else {
          // a root that is not an image: its position (r, theta)
          const cd z_ = tod(phi[ps]) + sh.L.a[ll];
          d[0] = (float)sqrt(abs2(z_));
          d[1] = (float)atan2(z_.y, z_.x);
        }
        d[2] = (float)meta[ps];
        d[3] = e32[ps];
      }
    }
    if (diag_cnt && tid == 0) { long long c_ = clock64(); sh.cnt[5] = (int)min(c_ - sh.clk0, 2000000000LL); sh.clk0 = c_; }
    // ------------------------------------------------ 2. theta bins
    for (int ps = tid; ps < NP; ps += NT) {
      if (!(meta[ps] & M_VALID) || (meta[ps] & M_EXACT)) continue;
      // distance of the FP32 angle from the nearest bin edge, against the
      // error of that FP32 evaluation: the point's own bound e32 / r, atan2f
      // (<= 2 ulp of pi, 4.8e-7), the float pi (8.7e-8), the sum (2.4e-7),
      // and the division by the float bin width (<= 128 bins x 1.2e-7 bin
      // widths, 7.5e-7 rad): 1.6e-6 rad in all; 64 EPS32 = 3.8e-6 leaves a
      // factor of two.  Closer points get an FP64 angle.
      float u = (t32[ps] + kPiF) / (float)ht;
      float fr = u - floorf(u);
      float d = fminf(fr, 1.0f - fr) * (float)ht;
      float eth = e32[ps] / fmaxf(r32[ps], 1e-30f) + 64.0f * EPS32;
      if (d <= eth) q_push(sh, queue, ps);
    }
    run_polish();
    for (int ps = tid; ps < NP; ps += NT) {
      if (!(meta[ps] & M_VALID)) continue;
      int t;
      if (meta[ps] & M_EXACT) t = (int)floor((pt[pidx[ps]] + kPi) / ht);
      else t = (int)floorf((t32[ps] + kPiF) / (float)ht);
      t = min(max(t, 0), BT - 1);
      tb[ps] = (uint8_t)t;
      atomicOr(&sh.tocc[t >> 6], 1ull << (t & 63));
    }
    __syncthreads();

    if (diag_cnt && tid == 0) { long long c_ = clock64(); sh.cnt[6] = (int)min(c_ - sh.clk0, 2000000000LL); sh.clk0 = c_; }
    if (diag_cnt && tid == 0) sh.cnt[13] = sh.cnt[0];
    // ------------------------------------------------ 3. theta runs (cyclic)
    if (tid == 0) {
      auto occb = [&](int t) -> bool { return (sh.tocc[t >> 6] >> (t & 63)) & 1ull; };
      bool full = true;
      for (int t = 0; t < BT; ++t) if (!occb(t)) full = false;
      for (int t = 0; t < 128; ++t) sh.runT[t] = -1;
      int nT = 0;
      if (!(sh.tocc[0] | sh.tocc[1])) {
        nT = 0;
      } else if (full) {
        for (int t = 0; t < BT; ++t) sh.runT[t] = 0;
        sh.startT[0] = 0;
        nT = 1;
      } else {
        int t0 = 0;
        while (occb(t0)) ++t0;
        for (int kk = 1; kk <= BT; ++kk) {
          int t = (t0 + kk) % BT;
          if (!occb(t)) continue;
          int prev = (t + BT - 1) % BT;
          if (occb(prev)) sh.runT[t] = sh.runT[prev];
          else if (nT < MAXT) { sh.runT[t] = (signed char)nT; sh.startT[nT] = t; ++nT; }
          else { sh.runT[t] = (signed char)(MAXT - 1); atomicOr(&sh.status, ICRS_ST_OVERFLOW); }
        }
      }
      sh.nT = nT;
      sh.full = full ? 1 : 0;
      for (int T = 0; T < MAXT; ++T) {
        sh.t_rlo_u[T] = 0xffffffffu; sh.t_rhi_l[T] = 0u;
        sh.t_rlo[T] = ~0ull; sh.t_rhi[T] = 0ull;
        sh.rocc[T] = 0u;
        for (int b = 0; b < MAXRB; ++b) { sh.tmask[T][b][0] = sh.tmask[T][b][1] = 0ull; sh.rrun[T][b] = -1; }
      }
    }
    __syncthreads();
    const int nT = sh.nT;

    // ------------------------------------------------ 4. r range per theta run
    for (int ps = tid; ps < NP; ps += NT) {
      if (!(meta[ps] & M_VALID)) continue;
      int T = sh.runT[tb[ps]];
      float r = r32[ps], er = (meta[ps] & M_EXACT) ? 4.0f * EPS32 * r : e32[ps] + 4.0f * EPS32 * r;
      atomicMin(&sh.t_rlo_u[T], fkey(r + er));
      atomicMax(&sh.t_rhi_l[T], fkey(r - er));
    }
    __syncthreads();
    const float tiny = TINY_EXTENT * rho32;
    for (int ps = tid; ps < NP; ps += NT) {
      if (!(meta[ps] & M_VALID)) continue;
      int T = sh.runT[tb[ps]];
      float r = r32[ps], er = (meta[ps] & M_EXACT) ? 4.0f * EPS32 * r : e32[ps] + 4.0f * EPS32 * r;
      bool cand = fkey(r - er) <= sh.t_rlo_u[T] || fkey(r + er) >= sh.t_rhi_l[T];
      // an image smaller than tiny contributes below the parity tolerance:
      // its decisions stay in FP32
      bool is_tiny = fkey_inv(sh.t_rhi_l[T]) - fkey_inv(sh.t_rlo_u[T]) < tiny;
      // the double-float r (error e32) is exact enough unless e32 is large
      if (cand) { meta[ps] |= M_CAND; if (!(meta[ps] & M_EXACT) && !is_tiny && !(e32[ps] <= 1e-11f)) q_push(sh, queue, ps); }
    }
    run_polish();
    for (int ps = tid; ps < NP; ps += NT) {
      if (!(meta[ps] & M_VALID) || !(meta[ps] & M_CAND)) continue;
      meta[ps] &= (uint8_t)~M_CAND;
      int T = sh.runT[tb[ps]];
      double r = rv(ps);
      atomicMin(&sh.t_rlo[T], dkey(r));
      atomicMax(&sh.t_rhi[T], dkey(r));
    }
    __syncthreads();
    if (tid < nT) {
      double lo = dkey_inv(sh.t_rlo[tid]), hi = dkey_inv(sh.t_rhi[tid]);
      sh.rlo[tid] = lo;
      sh.hr[tid] = (hi - lo) / BR;
    }
    __syncthreads();

    if (diag_cnt && tid == 0) { long long c_ = clock64(); sh.cnt[7] = (int)min(c_ - sh.clk0, 2000000000LL); sh.clk0 = c_; }
    if (diag_cnt && tid == 0) sh.cnt[14] = sh.cnt[0];
    // ------------------------------------------------ 5. r bins per theta run
    // Bin of r within its angular interval, floor((r - r_lo) / h_r): in FP32
    // from the double-float r where the bin edge is farther than the FP32
    // error, else in FP64 (after an FP64 polish if the double-float r itself
    // is uncertain).
    auto rbin_u = [&](int ps, int T, float* err) -> float {
      const float rlh = (float)sh.rlo[T];
      const float rll = (float)(sh.rlo[T] - (double)rlh);
      const float ihr = (float)(1.0 / sh.hr[T]);
      float dr = (r32[ps] - rlh) + (rl32[ps] - rll);
      float u = dr * ihr;
      *err = 4.0f * EPS32 * fabsf(u) + e32[ps] * ihr + 1e-6f;
      return u;
    };
    for (int ps = tid; ps < NP; ps += NT) {
      if (!(meta[ps] & M_VALID) || (meta[ps] & M_EXACT)) continue;
      int T = sh.runT[tb[ps]];
      double hr = sh.hr[T];
      if (!(hr > 0.0) || hr * BR < (double)tiny || e32[ps] <= 1e-11f) continue;
      float eu;
      float u = rbin_u(ps, T, &eu);
      float fr = u - floorf(u);
      if (fminf(fr, 1.0f - fr) <= eu && u > 0.5f && u < (float)BR - 0.5f) q_push(sh, queue, ps);
    }
    run_polish();
    for (int ps = tid; ps < NP; ps += NT) {
      if (!(meta[ps] & M_VALID)) continue;
      int T = sh.runT[tb[ps]];
      double hr = sh.hr[T];
      int b;
      if (!(hr > 0.0)) b = 0;
      else {
        float eu;
        float u = rbin_u(ps, T, &eu);
        float fr = u - floorf(u);
        if (fminf(fr, 1.0f - fr) > eu) b = (int)floorf(u);
        else b = (int)floor((rv(ps) - sh.rlo[T]) / hr);
      }
      b = min(max(b, 0), BR - 1);
      rb[ps] = (uint8_t)b;
      atomicOr(&sh.rocc[T], 1u << b);
      atomicOr(&sh.tmask[T][b][tb[ps] >> 6], 1ull << (tb[ps] & 63));
    }
    __syncthreads();

    if (diag_cnt && tid == 0) { long long c_ = clock64(); sh.cnt[8] = (int)min(c_ - sh.clk0, 2000000000LL); sh.clk0 = c_; }
    if (diag_cnt && tid == 0) sh.cnt[15] = sh.cnt[0];
    // ------------------------------------------------ 6. gap probes, r runs, origin
    // One warp: for every theta run, every empty gap with points of a shared
    // theta bin on both sides is probed at its middle radius (FP32 with a
    // guard band, FP64 when the guard cannot decide).
    if (warp == 0) {
      for (int T = 0; T < nT; ++T) {
        unsigned int occ = sh.rocc[T];
        unsigned int fill = 0u;
        for (int b = 1; b < BR; ++b) {
          if (((occ >> b) & 1u) || !((occ >> (b - 1)) & 1u)) continue;
          int e2 = b;
          while (e2 < BR && !((occ >> e2) & 1u)) ++e2;
          if (e2 >= BR) break;
          unsigned long long shared_[2];
          for (int h = 0; h < 2; ++h) {
            unsigned long long below = 0ull, above = 0ull;
            for (int k = 0; k < b; ++k) below |= sh.tmask[T][k][h];
            for (int k = e2; k < BR; ++k) above |= sh.tmask[T][k][h];
            shared_[h] = below & above;
          }
          double rg = sh.rlo[T] + sh.hr[T] * 0.5 * (double)(b + e2);
          bool hit = false;
          for (int t0 = 0; t0 < BT && !hit; t0 += 32) {
            int t = t0 + lane;
            bool in = false;
            if (t < BT && ((shared_[t >> 6] >> (t & 63)) & 1ull)) {
              double th = -kPi + (t + 0.5) * ht;
              float sth, cth;
              sincosf((float)th, &sth, &cth);
              cf z = mk((float)rg * cth, (float)rg * sth);
              float eps[NL];
              cf a[NL];
              for (int i = 0; i < NL; ++i) { eps[i] = sh.eps32[i]; a[i] = tof(sh.L.a[i]); }
              cf w = lens_map<NL, float>(eps, a, z);
              cf dw = w - tof(sh.wc);
              float d2 = abs2(dw);
              float errb = 64.0f * EPS32 * (sqrtf(abs2(w)) + 2.0f);
              float d = sqrtf(d2);
              if (fabsf(d - rho32) <= errb) {
                double s64, c64;
                sincos(th, &s64, &c64);
                cd z64 = mk(rg * c64, rg * s64);
                cd w64 = lens_map<NL, double>(sh.L.eps, sh.L.a, z64);
                in = sqrt(abs2(w64 - sh.wc)) < sh.rho;
              } else {
                in = d < rho32;
              }
            }
            hit = __any_sync(0xffffffffu, in);
          }
          if (hit) for (int k = b; k < e2; ++k) fill |= 1u << k;
        }
        if (lane == 0) {
          occ |= fill;
          sh.rocc[T] = occ;
          int nR = 0;
          for (int b = 0; b < BR; ++b) {
            if (!((occ >> b) & 1u)) continue;
            if (b > 0 && ((occ >> (b - 1)) & 1u)) sh.rrun[T][b] = sh.rrun[T][b - 1];
            else sh.rrun[T][b] = (signed char)(nR++);
          }
          sh.cellbase[T + 1] = nR;
        }
        __syncwarp();
      }
      if (lane == 0) {
        sh.cellbase[0] = 0;
        int tot = 0;
        for (int T = 0; T < nT; ++T) { int c = sh.cellbase[T + 1]; sh.cellbase[T] = tot; tot += c; }
        sh.cellbase[nT] = tot;
        if (tot > MAXCELL) { tot = MAXCELL; atomicOr(&sh.status, ICRS_ST_OVERFLOW); }
        sh.ncell = tot;
        cd w0 = lens_map<NL, double>(sh.L.eps, sh.L.a, mk(0.0, 0.0));
        sh.origin_in = sqrt(abs2(w0 - sh.wc)) < sh.rho;
        for (int c = 0; c < MAXCELL; ++c) {
          sh.c_cnt[c] = 0;
          sh.c_u[c][0] = 0xffffffffu; sh.c_u[c][1] = 0u; sh.c_u[c][2] = 0xffffffffu; sh.c_u[c][3] = 0u;
          sh.c_x[c][0] = ~0ull; sh.c_x[c][1] = 0ull; sh.c_x[c][2] = ~0ull; sh.c_x[c][3] = 0ull;
        }
        if (DER) {
          for (int c = 0; c < MAXCELL_D; ++c)
            for (int k = 0; k < 4; ++k) ds.cell_arg[c][k] = 0x7fffffff;
          if (tot > MAXCELL_D) atomicOr(&sh.status, ICRS_ST_OVERFLOW);
        }
      }
    }
    __syncthreads();

    if (diag_cnt && tid == 0) { long long c_ = clock64(); sh.cnt[9] = (int)min(c_ - sh.clk0, 2000000000LL); sh.clk0 = c_; }
    // ------------------------------------------------ 7. cell extremes
    auto cell_of = [&](int ps) -> int {
      int T = sh.runT[tb[ps]];
      int c = sh.cellbase[T] + sh.rrun[T][rb[ps]];
      return c < MAXCELL ? c : MAXCELL - 1;
    };
    // A point lies past the wrap of its angular interval when its bin comes
    // before the interval's first bin.  The decision is taken on the bin, not
    // on the angle: a point binned in FP64 next to the interval's first edge
    // can have an FP32 angle on the other side of that edge, and the FP32
    // candidate pass and the FP64 extreme pass must unwrap it alike.
    auto unwrap_t = [&](int ps, double th) -> double {
      int T = sh.runT[tb[ps]];
      return (int)tb[ps] < sh.startT[T] ? th + 2.0 * kPi : th;
    };
    for (int ps = tid; ps < NP; ps += NT) {
      if (!(meta[ps] & M_VALID)) continue;
      int c = cell_of(ps);
      atomicAdd(&sh.c_cnt[c], 1);
      float r = r32[ps];
      float th = (float)unwrap_t(ps, (double)t32[ps]);
      bool ex = meta[ps] & M_EXACT;
      float er = ex ? 4.0f * EPS32 * r : e32[ps] + 4.0f * EPS32 * r;
      float et = ex ? 16.0f * EPS32 : e32[ps] / fmaxf(r, 1e-30f) + 16.0f * EPS32;
      atomicMin(&sh.c_u[c][0], fkey(r + er));
      atomicMax(&sh.c_u[c][1], fkey(r - er));
      atomicMin(&sh.c_u[c][2], fkey(th + et));
      atomicMax(&sh.c_u[c][3], fkey(th - et));
    }
    __syncthreads();
    for (int ps = tid; ps < NP; ps += NT) {
      if (!(meta[ps] & M_VALID)) continue;
      int c = cell_of(ps);
      float r = r32[ps];
      float th = (float)unwrap_t(ps, (double)t32[ps]);
      bool ex = meta[ps] & M_EXACT;
      float er = ex ? 4.0f * EPS32 * r : e32[ps] + 4.0f * EPS32 * r;
      float et = ex ? 16.0f * EPS32 : e32[ps] / fmaxf(r, 1e-30f) + 16.0f * EPS32;
      bool cand_r = fkey(r - er) <= sh.c_u[c][0] || fkey(r + er) >= sh.c_u[c][1];
      bool cand_t = fkey(th - et) <= sh.c_u[c][2] || fkey(th + et) >= sh.c_u[c][3];
      bool cand = cand_r || cand_t;
      float ext_r = fkey_inv(sh.c_u[c][1]) - fkey_inv(sh.c_u[c][0]);
      float ext_t = (fkey_inv(sh.c_u[c][3]) - fkey_inv(sh.c_u[c][2])) * r;
      bool is_tiny = ext_r < tiny && ext_t < tiny;
      // theta extremes need an FP64 angle; r extremes only if the
      // double-float r is uncertain
      bool need = (cand_t && !sh.full) || !(e32[ps] <= 1e-11f);
      if (cand) { meta[ps] |= M_CAND; if (!ex && !is_tiny && need) q_push(sh, queue, ps); }
    }
    run_polish();
    for (int ps = tid; ps < NP; ps += NT) {
      if (!(meta[ps] & M_VALID) || !(meta[ps] & M_CAND)) continue;
      meta[ps] &= (uint8_t)~M_CAND;
      int c = cell_of(ps);
      double r = rv(ps), th = unwrap_t(ps, tv(ps));
      atomicMin(&sh.c_x[c][0], dkey(r));
      atomicMax(&sh.c_x[c][1], dkey(r));
      atomicMin(&sh.c_x[c][2], dkey(th));
      atomicMax(&sh.c_x[c][3], dkey(th));
    }
    __syncthreads();
    if (DER) {
      // the point that sets each cell extreme (lowest slot on ties), then
      // the extremes as dual numbers carrying that point's tangents
      for (int ps = tid; ps < NP; ps += NT) {
        if (!(meta[ps] & M_VALID)) continue;
        int c = cell_of(ps);
        if (c >= MAXCELL_D) continue;
        unsigned long long kr = dkey(rv(ps)), kt = dkey(unwrap_t(ps, tv(ps)));
        if (kr == sh.c_x[c][0]) atomicMin(&ds.cell_arg[c][0], ps);
        if (kr == sh.c_x[c][1]) atomicMin(&ds.cell_arg[c][1], ps);
        if (kt == sh.c_x[c][2]) atomicMin(&ds.cell_arg[c][2], ps);
        if (kt == sh.c_x[c][3]) atomicMin(&ds.cell_arg[c][3], ps);
      }
      __syncthreads();
      const int nd = min(sh.ncell, MAXCELL_D) * 4;
      for (int idx = tid; idx < nd; idx += NT) {
        const int c = idx >> 2, k = idx & 3;
        DualD v = dconst(dkey_inv(sh.c_x[c][k]));
        const int ps = ds.cell_arg[c][k];
        if (sh.c_cnt[c] && ps < NP) {
          const int kl = ps / N;
          cd u = mk((double)ulimb[kl].x.hi + (double)ulimb[kl].x.lo, (double)ulimb[kl].y.hi + (double)ulimb[kl].y.lo);
          // tangents at the FP64 position (the value stays the extreme the
          // sectors were built from)
          double r_ = rv(ps), t_ = tv(ps);
          if (!(meta[ps] & M_EXACT)) {
            cd z0 = tod(phi[ps]);
            if (has_plo) z0 = z0 + tod(plo[ps]);
            polish_image64<NL>(sh, z0 + sh.L.a[ll], limb_point64(sh, kl, K), &r_, &t_);
          }
          double dr_[NPAR], dt_[NPAR];
          point_tangents(sh, ds, r_, t_, u, dr_, dt_);
          for (int q = 0; q < NPAR; ++q) v.d[q] = k < 2 ? dr_[q] : dt_[q];
        }
        cdual[idx] = v;
      }
      __syncthreads();
    }

    if (diag_cnt && tid == 0) { long long c_ = clock64(); sh.cnt[10] = (int)min(c_ - sh.clk0, 2000000000LL); sh.clk0 = c_; }
    // ------------------------------------------------ 8. sectors (FP64, one thread)
    if (tid == 0 && !DER) {
      int nb = 0;
      for (int T = 0; T < nT; ++T) {
        int c0 = sh.cellbase[T], c1 = sh.cellbase[T + 1];
        for (int c = c0; c < c1 && c < MAXCELL; ++c) {
          if (!sh.c_cnt[c]) continue;
          Box B = cell_box<double>(dkey_inv(sh.c_x[c][0]), dkey_inv(sh.c_x[c][1]), dkey_inv(sh.c_x[c][2]),
                                   dkey_inv(sh.c_x[c][3]), g.margin, sh.full != 0, sh.origin_in && c == c0);
          if (nb < MAXBOX) sh.box[nb++] = B;
          else sh.status |= ICRS_ST_OVERFLOW;
        }
      }
      bool capped = false;
      nb = merge_boxes<double>(sh.box, nb, N, &capped);
      if (capped) sh.status |= ICRS_ST_SECTCAP;
      sh.nbox = nb;
    }
    if (tid == 0 && DER) {
      // the same rules on dual numbers: the sector bounds and their tangents
      int nb = 0;
      for (int T = 0; T < nT; ++T) {
        int c0 = sh.cellbase[T], c1 = sh.cellbase[T + 1];
        for (int c = c0; c < c1 && c < MAXCELL; ++c) {
          if (!sh.c_cnt[c]) continue;
          if (c >= MAXCELL_D || nb >= MAXBOX_D) { sh.status |= ICRS_ST_OVERFLOW; continue; }
          bdual[nb++] = cell_box<DualD>(cdual[c * 4 + 0], cdual[c * 4 + 1], cdual[c * 4 + 2], cdual[c * 4 + 3],
                                        g.margin, sh.full != 0, sh.origin_in && c == c0);
        }
      }
      bool capped = false;
      nb = merge_boxes<DualD>(bdual, nb, N, &capped);
      if (capped) sh.status |= ICRS_ST_SECTCAP;
      for (int b = 0; b < nb; ++b) {
        sh.box[b].r_lo = bdual[b].r_lo.v;
        sh.box[b].r_hi = bdual[b].r_hi.v;
        sh.box[b].th_lo = bdual[b].th_lo.v;
        sh.box[b].width = bdual[b].width.v;
        sh.box[b].periodic = bdual[b].periodic;
      }
      sh.nbox = nb;
    }
    if (DER)
      for (int k = tid; k < NW * 12; k += NT) wder[k] = 0.0;
    __syncthreads();

    if (diag_cnt && tid == 0) { long long c_ = clock64(); sh.cnt[11] = (int)min(c_ - sh.clk0, 2000000000LL); sh.clk0 = c_; }
    // ------------------------------------------------ 9. rays
    const int NR = g.n_r, NTH = g.n_theta;
    // limb darkening I = I0 [1 - u1 (1 - mu) - u2 (1 - mu)^2 - sum_k a_k (1 -
    // mu^(k/2))], mu = sqrt(1 - d^2/rho^2), I0 = 1 / (pi (1 - u1/3 - u2/6 -
    // sum_k a_k k/(k+4))) (the linear law of Appendix A.2 when the others are
    // 0); uniform: I = 1/pi.  As a polynomial in s = mu^(1/2):
    //   I = c0f + c1f mu + c2f mu^2 + s (c1h + c3h mu),
    //   c0f = I0 (1 - u1 - u2 - sum a) (the limb value), c1f = I0 (u1 + 2 u2 +
    //   a2), c2f = I0 (a4 - u2), c1h = I0 a1, c3h = I0 a3
    const double sa_ = sh.pa[0] / 5.0 + sh.pa[1] * (2.0 / 6.0) + sh.pa[2] * (3.0 / 7.0) + sh.pa[3] * 0.5;
    const double I0d = 1.0 / (kPi * (1.0 - sh.u1 / 3.0 - sh.u2 / 6.0 - sa_));
    const float I0 = g.uniform ? (float)(1.0 / kPi) : (float)I0d;
    const float irho2 = 1.0f / (rho32 * rho32);
    const float irho = 1.0f / rho32;
    const float dcf = (float)g.delta_c;
    const float c0f = g.uniform ? I0 : (float)(I0d * (1.0 - sh.u1 - sh.u2 - sh.pa[0] - sh.pa[1] - sh.pa[2] - sh.pa[3]));
    const float c1f = g.uniform ? 0.f : (float)(I0d * (sh.u1 + 2.0 * sh.u2 + sh.pa[1]));
    const float c2f = g.uniform ? 0.f : (float)(I0d * (sh.pa[3] - sh.u2));
    // c1h, c3h and their flag live in shared memory: the default sweep
    // never reads them
    if (tid == 0) {
      sh.c1h = g.uniform ? 0.f : (float)(I0d * sh.pa[0]);
      sh.c3h = g.uniform ? 0.f : (float)(I0d * sh.pa[2]);
      sh.half = (sh.c1h != 0.f || sh.c3h != 0.f) ? 1 : 0;
      sh.generic = sh.half || sh.spot;
    }
    __syncthreads();
    const bool split = g.ld_split && !g.uniform;  // split-profile boundary rule
    const float sfac = (float)g.s_fac;            // sigmoid steepness of the paper's gradient rule
    float acc_s = 0.f, acc_c = 0.f;  // Kahan sum of this thread
    uint32_t st_local = 0u;
    for (int bxi = 0; bxi < sh.nbox; ++bxi) {
      const Box B = sh.box[bxi];
      if (tid == 0) {
        sh.dr64 = (B.r_hi - B.r_lo) / NR;
        sh.dth64 = B.width / NTH;
        sh.dr32 = (float)sh.dr64;
        sh.dth32 = (float)sh.dth64;
        // anchors: enough groups that an anchor is within ~0.025 of its rays
        const double LMAX = 0.05;
        int mth = (int)ceil(B.r_hi * B.width / LMAX);
        int mr = (int)ceil((B.r_hi - B.r_lo) / LMAX);
        mth = min(max(mth, 1), min(64, NTH));
        // groups of at most GTH_MAX columns (the offset table's size; for
        // n_theta <= 8192 this needs at most 32 groups)
        mth = max(mth, (NTH + GTH_MAX - 1) / GTH_MAX);
        mr = min(max(mr, 1), min(4, NR));
        mth = min(mth, MAXANCH / mr);  // the anchor table holds MAXANCH entries
        // theta groups of an even width: the forward ray stage evaluates
        // column pairs (l, l + 1), l even, which then share their group
        sh.gth = 2 * ((NTH + 2 * mth - 1) / (2 * mth));
        sh.gr = (NR + mr - 1) / mr;
        sh.mth = (NTH + sh.gth - 1) / sh.gth;
        sh.mr = (NR + sh.gr - 1) / sh.gr;
        sh.nanch = sh.mth * sh.mr;
        // ray stage: tasks of 32 rows (one per lane) x a theta chunk
        // of an even number of columns, about 8 tasks per warp per sector
        const int nrb = (NR + 31) >> 5;
        const int nch = max(1, (8 * NW + nrb - 1) / nrb);
        sh.chunk = min(NTH, max(16, 2 * ((NTH + 2 * nch - 1) / (2 * nch))));
      }
      __syncthreads();
      const int gth = sh.gth, gr = sh.gr, mth = sh.mth;
      // group of ray l: l / gth as a multiply-high by ceil(2^32 / gth), exact
      // for l, gth < 2^16 (here both <= 8192)
      const unsigned int gmagic = (unsigned int)((0xFFFFFFFFull / (unsigned long long)gth) + 1ull);
      // anchors (FP64, one per thread)
      for (int an = tid; an < sh.nanch; an += NT) {
        int gi = an / mth, mi = an % mth;
        double rc = B.r_lo + (gi * gr + 0.5 * gr) * sh.dr64;
        double thc = B.th_lo + (mi * gth + 0.5 * gth) * sh.dth64;
        double sn, cs;
        sincos(thc, &sn, &cs);
        cd R = mk(cs, -sn);  // e^{-i th_c}
        cd zc = mk(rc * cs, rc * sn);
        cd wsd = lens_map<NL, double>(sh.L.eps, sh.L.a, zc) - sh.wc;
        const cf ws = tof(R * wsd);
        if (LAW != 0 && sh.spot) spc[an] = make_float2((float)(sh.rho * (cs * sh.spot_x + sn * sh.spot_y)),
                                           (float)(sh.rho * (cs * sh.spot_y - sn * sh.spot_x)));
        // error bound of |Delta w'|: anchor term plus rounding of the ray's
        // offset (at most the group half-diagonal) and of its image term
        const double half = 0.5 * gr * sh.dr64 + (B.r_hi) * 0.5 * gth * sh.dth64;
        const float e0 = (float)(16.0 * EPS32 * (fabs(ws.x) + fabs(ws.y) + 2.0 * half));
        const double rr = (double)rho32 * (double)rho32;
        float lo2 = -1.0f, hi2 = __int_as_float(0x7f800000);
        {
          // U = N / P (AnchorF), coefficients from the FP64 A_j, K_j
          cd A64[NL], K64[NL];
          for (int j = 0; j < NL; ++j) {
            A64[j] = R * (zc - sh.L.a[j]);
            K64[j] = scl(inv(A64[j]), sh.L.eps[j]);
          }
          cd nc[3], pc[3];
          if constexpr (NL == 2) {
            nc[0] = K64[0] * A64[1] + K64[1] * A64[0];
            nc[1] = K64[0] + K64[1];
            nc[2] = mk(0.0, 0.0);
            pc[0] = A64[0] * A64[1];
            pc[1] = A64[0] + A64[1];
            pc[2] = mk(0.0, 0.0);
          } else {
            nc[0] = K64[0] * (A64[1] * A64[2]) + K64[1] * (A64[0] * A64[2]) + K64[2] * (A64[0] * A64[1]);
            nc[1] = K64[0] * (A64[1] + A64[2]) + K64[1] * (A64[0] + A64[2]) + K64[2] * (A64[0] + A64[1]);
            nc[2] = K64[0] + K64[1] + K64[2];
            pc[0] = A64[0] * A64[1] * A64[2];
            pc[1] = A64[0] * A64[1] + A64[0] * A64[2] + A64[1] * A64[2];
            pc[2] = A64[0] + A64[1] + A64[2];
          }
          AnchorF af;
          af.ws = ws;
          for (int k = 0; k < 3; ++k) { af.n[k] = tof(nc[k]); af.p[k] = tof(pc[k]); }
          af.e0 = e0;
          af.pad = 0.f;
          // the group's band: every ray has |dz| <= half, so |Q_j| >= |A_j| -
          // half, |P| >= prod_j (|A_j| - half) and |U| <= sum_j |K_j| / (|A_j|
          // - half); the rounding error of the FP32 quotient is bounded by
          // u (cN M_N + (cP + 9) |U| M_P) / |P| (M_N, M_P: the polynomials
          // with coefficient moduli, at |dz| = half) and that of dz U by
          // |dz| (that + 3 u |U|), times 2 for the FP32 evaluation of the
          // bound itself (see ray_eval)
          bool bounded = true;
          double um = 0.0, pmin = 1.0;
          for (int j = 0; j < NL; ++j) {
            const double aa = sqrt(abs2(A64[j]));
            if (!(aa > 1.0625 * half)) bounded = false;
            else { um += sqrt(abs2(K64[j])) / (aa - half); pmin *= aa - half; }
          }
          if (bounded) {
            const double mn = sqrt(abs2(nc[0])) + half * (sqrt(abs2(nc[1])) + half * sqrt(abs2(nc[2])));
            const double mp = NL == 2 ? sqrt(abs2(pc[0])) + half * (sqrt(abs2(pc[1])) + half)
                                      : sqrt(abs2(pc[0])) + half * (sqrt(abs2(pc[1])) + half * (sqrt(abs2(pc[2])) + half));
            const double cN = NL == 2 ? 4.0 : 9.0, cP = NL == 2 ? 6.0 : 13.0;
            const double du = EPS32 * (cN * mn + (cP + 9.0) * um * mp) / pmin;
            const double eb = (double)e0 + 2.0 * half * (du + 3.0 * EPS32 * um);
            const double X = 1.01 * (2.0 * (double)rho32 * eb + eb * eb) + 8.0 * EPS32 * rr;
            if (X < 0.5 * rr) {
              lo2 = __double2float_rd(rr - X);
              hi2 = __double2float_ru(rr + X);
            }
          }
          af.lo2 = lo2;
          af.hi2 = hi2;
          anch[an] = af;
          if constexpr (DER) {
            // the adjoint's ray gradients: A_j in FP32 and the anchor angle
            ds.aA[an] = make_float4((float)A64[0].x, (float)A64[0].y, (float)A64[1].x, (float)A64[1].y);
            ds.acs[an] = make_float2((float)cs, (float)sn);
          }
        }
      }
      // offsets within a theta group, (cos d - 1, sin d) with d = (o + 1/2 -
      // gth/2) dth; column pairs (o, o + 1), o even, are stored as 16 bytes
      // (x_o, x_o+1, y_o, y_o+1), so that the forward ray stage loads a pair's
      // x and y as two adjacent float2 (gth is even)
      float* tabf = reinterpret_cast<float*>(tab);
      for (int o = tid; o < gth; o += NT) {
        float d = ((float)o + 0.5f - 0.5f * (float)gth) * sh.dth32;
        float s, c;
        sincosf(d, &s, &c);
        float sh2 = sinf(0.5f * d);
        tabf[4 * (o >> 1) + (o & 1)] = -2.0f * sh2 * sh2;
        tabf[4 * (o >> 1) + 2 + (o & 1)] = s;
        (void)c;
      }
      __syncthreads();
      auto tab_at = [&](int o) -> cf {
        const float* t_ = tabf + 4 * (o >> 1) + (o & 1);
        return mk(t_[0], t_[2]);
      };
      const float dr32 = sh.dr32;
      const float bxw = (float)(sh.dr64 * sh.dth64);
      auto wrapl = [&](int l) -> int { return l < 0 ? l + NTH : (l >= NTH ? l - NTH : l); };
      // per-point weights (Appendix A).  Points with both neighbours
      // inside (W = 1) are summed directly; points next to the image
      // boundary are queued per warp and their crossings solved with one
      // point per lane.
      // I(d) = c0f + c1f mu + c2f mu^2, mu^2 = x = 1 - d^2/rho^2
      auto brightness = [&](float d2) -> float {
        const float x = fmaxf(fmaf(-d2, irho2, 1.0f), 1e-30f);
        const float mu = x * rsqrtf(x);
        float I = fmaf(c2f, x, fmaf(c1f, mu, c0f));
        if (LAW != 0 && sh.half) I = fmaf(sqrtf(mu), fmaf(sh.c3h, mu, sh.c1h), I);
        return I;
      };
      // I and dI/dd, dI/drho, dI/du1 at squared distance d2:
      //   dI/dx = c1/(2 mu) + c2, dx/dd = -2 d/rho^2, dx/drho = 2 d^2/rho^3,
      //   dI/du1 = I (pi/3) I0 - I0 (1 - mu)   (dI0/du1 = (pi/3) I0^2)
      // (hc: std::true_type for the generic law: half-integer powers of mu
      // checked at run time)
      auto brightness_der = [&](float d2, float* Id, float* Ir, float* Iu, auto hc) -> float {
        if (g.uniform) { *Id = 0.f; *Ir = 0.f; *Iu = 0.f; return I0; }
        // (hardware reciprocal square roots: 2^-22.9 relative, far inside
        // the derivative's tolerance)
        float x = fmaxf(0.f, 1.0f - d2 * irho2);
        const float rs = x > 0.f ? rsqrt_fast(x) : 0.f;  // 1 / mu
        float sx = x * rs;
        float I = c0f + c1f * sx + c2f * x;
        float d = d2 * rsqrt_fast(fmaxf(d2, 1e-37f));
        // k = (dI/dmu) / mu / rho^2
        float k = x > 0.f ? (c1f * rs + 2.0f * c2f) * irho2 : 0.f;
        if constexpr (decltype(hc)::value) {
          if (LAW != 0 && sh.half && x > 0.f) {
            // s (c1h + c3h mu): dI/dmu = c1h / (2 s) + 1.5 c3h s, s = mu^(1/2)
            const float c1h = sh.c1h, c3h = sh.c3h;
            const float s_ = sqrtf(sx);
            I += s_ * (c1h + c3h * sx);
            k += (0.5f * c1h / s_ + 1.5f * c3h * s_) * rs * irho2;
          }
        }
        *Id = -k * d;
        *Ir = k * d2 * irho;
        *Iu = I * (float)(kPi / 3.0) * I0 + I0 * (sx - 1.0f);
        return I;
      };
      // derivative mode: per side, d delta / d(stencil distances) and
      // d delta / d rho times f'(delta) (crossing p(x) = rho, dx = (drho -
      // sum_m l_m(x) dy_m) / p'(x); delta = -x on the left, x on the right).
      // p'(x) is a difference of nearly equal distances, so the stencil
      // and the crossing are taken in FP64 in this mode.
      float sd_c[2], sd_l[2][4];
      int sd_b[2], sd_n[2];
      // dist (derivative mode): FP64 distances of rays mi-2 .. mi+2 (inf
      // beyond a non-periodic edge), or NULL to compute them here
      // sv[k] = signed squared distance of ray l - 2 + k (sv[2] is the
      // point), lab = l (absolute index), irow = its row
      // WU (forward mode, optional): the same point's weight under the
      // uniform rule f_U(delta) = delta + 1/2, for the split-profile rule
      auto boundary_weight = [&](int mi, const float* sv, int lab, int irow, const double* dist,
                                 float* WU = nullptr) -> float {
        float d2 = -sv[2];
        float vl = sv[1], vr = sv[3];
        bool Lin = signbit(vl), Rin = signbit(vr);
        float W;
          float fL = 0.f, fR = 0.f, uL = 0.f, uR = 0.f;
          if (DER) { sd_n[0] = sd_n[1] = 0; sd_c[0] = sd_c[1] = 0.f; }
          for (int side = 0; side < 2; ++side) {
            bool isL = side == 0;
            if (isL ? Lin : Rin) continue;
            float vo = isL ? vl : vr;
            float delta;
            if (isinf(vo)) {
              delta = 0.5f;
              st_local |= ICRS_ST_EDGE;
            } else if (DER) {
              // FP64 stencil; FP32 regula falsi, then Newton on the FP64
              // cubic; f, f' and the basis in FP32 at the FP64 crossing
              const int c0 = isL ? -2 : -1;
              double xsd[4], ysd[4];
              float ysf[4];
              int nd = 0;
              double yin = 0, yout = 0;
              for (int c = 0; c < 4; ++c) {
                const int off = c0 + c;
                double v;
                if (dist) {
                  v = dist[off + 2];
                } else {
                  const int l2_ = lab + off;
                  v = (!B.periodic && (l2_ < 0 || l2_ >= NTH)) ? __longlong_as_double(0x7ff0000000000000LL)
                                                               : ray_distance64<NL>(sh, B, irow, wrapl(l2_));
                }
                if (isinf(v)) { st_local |= ICRS_ST_EDGE; continue; }
                xsd[nd] = (double)off;
                ysd[nd] = v;
                ysf[nd] = (float)v;
                if (off == 0) yin = v;
                if (off == (isL ? -1 : 1)) yout = v;
                ++nd;
              }
              const double dd1 = ysd[1] - ysd[0];
              const double dd2 = nd > 2 ? 0.5 * (ysd[2] - 2.0 * ysd[1] + ysd[0]) : 0.0;
              const double dd3 = nd > 3 ? (ysd[3] - 3.0 * ysd[2] + 3.0 * ysd[1] - ysd[0]) * (1.0 / 6.0) : 0.0;
              double xd = crossing_solve<float>(ysf, (float)xsd[0], nd, (float)yin, (float)yout, isL ? -1.0f : 1.0f,
                                                rho32, 1e-5f, 12);
              bool ok = true;
              for (int it = 0; it < 2; ++it) {
                const double tt = xd - xsd[0];
                const double pv = ysd[0] + tt * (dd1 + (tt - 1.0) * (dd2 + (tt - 2.0) * dd3)) - sh.rho;
                const double pd = dd1 + (2.0 * tt - 1.0) * dd2 + ((3.0 * tt - 6.0) * tt + 2.0) * dd3;
                if (!(pd != 0.0)) { ok = false; break; }
                xd -= pv / pd;
              }
              if (!ok || !(isL ? (xd >= -1.0 && xd <= 0.0) : (xd >= 0.0 && xd <= 1.0)))
                xd = crossing_solve<double>(ysd, xsd[0], nd, yin, yout, isL ? -1.0 : 1.0, sh.rho, 1e-14, 60);
              const double dd = isL ? -xd : xd;
              const float dl = (float)dd;
              float fv, fp;
              if (g.uniform) { fv = dl + 0.5f; fp = 1.0f; }
              else if (dd >= g.delta_c) {
                const float sq = sqrtf(1.0f + 0.5f / dl);
                fv = (0.5f + dl) * (2.0f / 3.0f) * sq;
                fp = (2.0f / 3.0f) * sq - (0.5f + dl) / (6.0f * dl * dl * sq);
              } else { fv = (2.0f / 3.0f) * dl + 0.5f; fp = 2.0f / 3.0f; }
              // the paper's gradient rule: the fixed derivative of the
              // second-order branch on both branches
              if (g.grad_rule && !g.uniform) fp = 2.0f / 3.0f;
              if (isL) fL = fv; else fR = fv;
              const double tt = xd - xsd[0];
              const double slope = dd1 + (2.0 * tt - 1.0) * dd2 + ((3.0 * tt - 6.0) * tt + 2.0) * dd3;
              (void)lagrange_basis<float>(ysf, nd, (float)tt, sd_l[side]);
              sd_c[side] = (float)((isL ? -fp : fp) / slope);
              sd_b[side] = mi + (int)xsd[0];
              sd_n[side] = nd;
              continue;
            } else {
              // stencil: entering (-2,-1,0,+1), exiting (-1,0,+1,+2)
              float xs[4], ys[4];
              int np_ = 0;
              const int c0 = isL ? -2 : -1;
              for (int c = 0; c < 4; ++c) {
                float vv = sv[2 + c0 + c];
                if (isinf(vv)) { st_local |= ICRS_ST_EDGE; continue; }
                xs[np_] = (float)(c0 + c);
                ys[np_] = sqrtf(fabsf(vv));
                ++np_;
              }
              float xo = isL ? -1.0f : 1.0f;
              float x = crossing_solve<float>(ys, xs[0], np_, sqrtf(d2), sqrtf(fabsf(vo)), xo, rho32, 1e-5f, 12);
              delta = isL ? -x : x;
              if (!g.uniform && fabsf(delta - dcf) < 2e-3f) {
                // branch of f(delta) too close to call in FP32: redo the
                // crossing from FP64 distances
                int l = lab;
                double xsd[4], ysd[4];
                int nd = 0;
                double yin = 0, yout = 0;
                for (int c = 0; c < 4; ++c) {
                  int ll2 = l + c0 + c;
                  if (!B.periodic && (ll2 < 0 || ll2 >= NTH)) continue;
                  int lw2 = ((ll2 % NTH) + NTH) % NTH;
                  xsd[nd] = (double)(c0 + c);
                  ysd[nd] = ray_distance64<NL>(sh, B, irow, lw2);
                  if (c0 + c == 0) yin = ysd[nd];
                  if (c0 + c == (isL ? -1 : 1)) yout = ysd[nd];
                  ++nd;
                }
                if (diag_cnt) atomicAdd(&sh.cnt[3], 1);
                double xd = crossing_solve<double>(ysd, xsd[0], nd, yin, yout, isL ? -1.0 : 1.0, sh.rho, 1e-14, 60);
                double dd = isL ? -xd : xd;
                delta = (float)dd;
                float fv = (float)fdelta<double>(dd, g.delta_c, 0);
                if (isL) { fL = fv; uL = delta + 0.5f; } else { fR = fv; uR = delta + 0.5f; }
                continue;
              }
            }
            float fv = fdelta<float>(delta, dcf, g.uniform);
            if (isL) { fL = fv; uL = delta + 0.5f; } else { fR = fv; uR = delta + 0.5f; }
          }
          if (WU) *WU = Lin ? uR : (Rin ? uL : fmaxf(0.f, uL + uR - 1.0f));
          if (Lin) W = fR;
          else if (Rin) W = fL;
          else W = fmaxf(0.f, fL + fR - 1.0f);
          if (DER && !(Lin || Rin) && !(fL + fR - 1.0f > 0.f)) sd_n[0] = sd_n[1] = 0, sd_c[0] = sd_c[1] = 0.f;
        return W;
      };
      {
        // ---- ray stage.  A warp takes a task of 32 rows (lane = row i) and
        // a chunk [c0, c1) of theta columns, and sweeps the columns in blocks
        // of KB (all lanes at the same column, so the group offsets and,
        // within an r group, the anchor are shared and held in registers).
        // Each ray's squared distance is classified against the group's FP32
        // band: inside (I(d) added to the row), outside, or undecided.  The
        // inside flags go into a per-lane bit window.  At the end of a block
        // one warp vote covers both rare events: a ray the band left
        // undecided (its own bound, else FP64, decides it) and a boundary
        // point (inside with an outside neighbour), which goes to the
        // per-warp deferred queue as (column, row).  A queue flush
        // re-evaluates each point's five-ray stencil and adds I (W - 1)
        // (Appendix A per-point rule).  The adjoint adds, for every inside
        // ray, its seed dI/dd times the gradient of d, and the queue flush
        // the boundary points' seeds.
        constexpr int DQ = dq_entries(NL);
        constexpr int KB = 8;  // columns per block (even: column pairs load as 16 bytes)
        int2* dq = reinterpret_cast<int2*>(wqueue + warp * 2 * DQ);
        int dq_n = 0;
        const int CH = sh.chunk;
        const int nch = (NTH + CH - 1) / CH;
        const int ntask = ((NR + 31) >> 5) * nch;
        const float rr32 = rho32 * rho32;
        const unsigned lt_mask = (1u << lane) - 1u;
        const AnchorF* anf = reinterpret_cast<const AnchorF*>(anch);
        // c + a b in FP32, each operation rounded as written
        auto cfma = [](const cf a, const cf b, const cf c) -> cf {
          return mk(__fmaf_rn(a.x, b.x, __fmaf_rn(-a.y, b.y, c.x)), __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, c.y)));
        };
        // squared distance |Delta w'|^2 of the ray at group offset (tx, ty)
        // in the row (ri_, dri_) of anchor an: Delta w' = ws + dz + conj(dz
        // N / P), dz = (ri_ tx + dri_, ri_ ty).  Every operation is rounded
        // as written, so each evaluation of a ray gives the same bits.  With
        // eb: the ray's own bound on the error of |Delta w'|, e0 + 2 |dz| u
        // (cN M_N + cU |U| M_P) / |P|, from |dN| <= cN u M_N, |dP| <= cP u
        // M_P (Horner in complex FMAs, plus the rounded coefficients) and cU
        // = 3 cP + 10 (the quotient, |P|^2, the reciprocal and the products),
        // times 2 for the FP32 evaluation of the bound.
        // (dzo, dwo: optionally dz and Delta w' themselves, for the adjoint)
        auto ray_eval = [&](const AnchorF& an, float tx, float ty, float ri_, float dri_, float* eb, cf* dzo = nullptr,
                            cf* dwo = nullptr) -> float {
          const cf dz = mk(__fmaf_rn(ri_, tx, dri_), __fmul_rn(ri_, ty));
          cf Pq, Nq;
          if constexpr (NL == 2) {
            const cf F = mk(__fadd_rn(an.p[1].x, dz.x), __fadd_rn(an.p[1].y, dz.y));
            Pq = cfma(dz, F, an.p[0]);
            Nq = cfma(an.n[1], dz, an.n[0]);
          } else {
            const cf F2 = mk(__fadd_rn(an.p[2].x, dz.x), __fadd_rn(an.p[2].y, dz.y));
            Pq = cfma(dz, cfma(dz, F2, an.p[1]), an.p[0]);
            Nq = cfma(dz, cfma(an.n[2], dz, an.n[1]), an.n[0]);
          }
          const float q = __fmaf_rn(Pq.x, Pq.x, __fmul_rn(Pq.y, Pq.y));
          const float ip = rcp_fast(q);  // <= 1 ulp
          // V = N conj(P), pv = dz V, Delta w' = (ws + dz) + conj(pv) / |P|^2
          const cf V = mk(__fmaf_rn(Nq.x, Pq.x, __fmul_rn(Nq.y, Pq.y)), __fmaf_rn(Nq.y, Pq.x, -__fmul_rn(Nq.x, Pq.y)));
          const cf pv = mk(__fmaf_rn(dz.x, V.x, -__fmul_rn(dz.y, V.y)), __fmaf_rn(dz.x, V.y, __fmul_rn(dz.y, V.x)));
          const cf dw = mk(__fmaf_rn(pv.x, ip, __fadd_rn(an.ws.x, dz.x)), __fmaf_rn(-pv.y, ip, __fadd_rn(an.ws.y, dz.y)));
          if (dzo) *dzo = dz;
          if (dwo) *dwo = dw;
          if (eb) {
            const float md = sqrtf(abs2(dz)), aP = sqrtf(q), aU = sqrtf(abs2(V)) * ip;
            const float mn = sqrtf(abs2(an.n[0])) + md * (sqrtf(abs2(an.n[1])) + md * sqrtf(abs2(an.n[2])));
            const float mp = NL == 2 ? sqrtf(abs2(an.p[0])) + md * (sqrtf(abs2(an.p[1])) + md)
                                     : sqrtf(abs2(an.p[0])) + md * (sqrtf(abs2(an.p[1])) + md * (sqrtf(abs2(an.p[2])) + md));
            constexpr float cN = NL == 2 ? 4.0f : 9.0f, cU = NL == 2 ? 28.0f : 49.0f;
            *eb = an.e0 + 2.0f * md * EPS32 * (cN * mn + cU * aU * mp) / aP;
          }
          return __fmaf_rn(dw.x, dw.x, __fmul_rn(dw.y, dw.y));
        };
        // a ray the group band left open: its own bound decides in FP32 where
        // it can, else the FP64 distance (d2 is then replaced by its square)
        auto decide = [&](float& d2, float eb, int irow, int lw) -> bool {
          const float X = 1.01f * (2.0f * rho32 * eb + eb * eb) + 8.0f * EPS32 * rr32;
          if (fabsf(d2 - rr32) > X) return d2 < rr32;
          const double d64 = ray_distance64<NL>(sh, B, irow, lw);
          if (diag_cnt) atomicAdd(&sh.cnt[2], 1);
          d2 = (float)(d64 * d64);
          return d64 < sh.rho;
        };
        // any column l of row irow (wrapped; beyond a non-periodic edge: outside, +inf)
        // a ray's spot factor: 1 - c inside the spot, else 1.  dw: the ray's
        // offset from the source centre in the frame of anchor ai, with error
        // bound eb; the spot centre's FP32 rounding adds 4 u rho.  Decided in
        // FP32 outside the band, else from the FP64 offset as the oracle
        // decides it.
        const float spot_rr = (float)(sh.rho * sh.spot_r);
        const float spot_r2 = spot_rr * spot_rr;
        const float spot_f = (float)(1.0 - sh.spot_c);
        auto spot_factor = [&](int ai, const cf dw, float eb, int irow, int lw) -> float {
          if (LAW == 0 || !sh.spot) return 1.f;
          const float2 c = spc[ai];
          const float ex = dw.x - c.x, ey = dw.y - c.y;
          const float q = fmaf(ex, ex, ey * ey);
          const float e = eb + 4.0f * EPS32 * rho32;
          const float X = 1.01f * (2.0f * spot_rr * e + e * e) + 8.0f * EPS32 * spot_r2;
          if (fabsf(q - spot_r2) > X) return q < spot_r2 ? spot_f : 1.f;
          const cd d64 = ray_offset64<NL>(sh, B, irow, lw);
          const double fx = d64.x / sh.rho - sh.spot_x, fy = d64.y / sh.rho - sh.spot_y;
          return fx * fx + fy * fy < sh.spot_r * sh.spot_r ? spot_f : 1.f;
        };
        // (fso: optionally the ray's spot factor)
        auto classify = [&](int gi_, float ri_, float dri_, int irow, int l, float* d2o,
                            float* fso = nullptr) -> bool {
          if (!B.periodic && (l < 0 || l >= NTH)) { *d2o = __int_as_float(0x7f800000); if (fso) *fso = 1.f; return false; }
          const int lw = wrapl(l);
          const int mgrp = (int)__umulhi((unsigned int)lw, gmagic);
          const AnchorF& an = anf[gi_ * mth + mgrp];
          const cf t = tab_at(lw - mgrp * gth);
          float eb;
          cf dw;
          float d2 = ray_eval(an, t.x, t.y, ri_, dri_, &eb, nullptr, &dw);
          bool in = d2 < an.lo2;
          if (!in && !(d2 > an.hi2)) in = decide(d2, eb, irow, lw);
          *d2o = d2;
          if (fso) *fso = spot_factor(gi_ * mth + mgrp, dw, eb, irow, lw);
          return in;
        };
        if constexpr (!DER) {
        // the anchor as broadcast pairs for two columns at once (binary)
        struct AnchorP { float2 wsx, wsy, n0x, n0y, n1x, n1y, nn1y, p0x, p0y, p1x, p1y; };
        auto pairs_of = [](const AnchorF& a) -> AnchorP {
          AnchorP r;
          r.wsx = make_float2(a.ws.x, a.ws.x);     r.wsy = make_float2(a.ws.y, a.ws.y);
          r.n0x = make_float2(a.n[0].x, a.n[0].x); r.n0y = make_float2(a.n[0].y, a.n[0].y);
          r.n1x = make_float2(a.n[1].x, a.n[1].x); r.n1y = make_float2(a.n[1].y, a.n[1].y);
          r.nn1y = make_float2(-a.n[1].y, -a.n[1].y);
          r.p0x = make_float2(a.p[0].x, a.p[0].x); r.p0y = make_float2(a.p[0].y, a.p[0].y);
          r.p1x = make_float2(a.p[1].x, a.p[1].x); r.p1y = make_float2(a.p[1].y, a.p[1].y);
          return r;
        };
        // rays of columns (l, l + 1) of one row with paired FP32 operations
        // (binary lens): component k is rounded exactly as ray_eval rounds
        // ray l + k, operation by operation, so both give the same bits
        auto ray_eval2 = [&](const AnchorP& a, float2 tx, float2 ty, float2 ri2, float2 dri2) -> float2 {
          const float2 dzx = __ffma2_rn(ri2, tx, dri2), dzy = __fmul2_rn(ri2, ty);
          const float2 ndzy = make_float2(-dzy.x, -dzy.y);
          const float2 Fx = __fadd2_rn(a.p1x, dzx), Fy = __fadd2_rn(a.p1y, dzy);
          const float2 Px = __ffma2_rn(dzx, Fx, __ffma2_rn(ndzy, Fy, a.p0x));
          const float2 Py = __ffma2_rn(dzx, Fy, __ffma2_rn(dzy, Fx, a.p0y));
          const float2 Nx = __ffma2_rn(a.n1x, dzx, __ffma2_rn(a.nn1y, dzy, a.n0x));
          const float2 Ny = __ffma2_rn(a.n1x, dzy, __ffma2_rn(a.n1y, dzx, a.n0y));
          const float2 q = __ffma2_rn(Px, Px, __fmul2_rn(Py, Py));
          const float2 ip = make_float2(rcp_fast(q.x), rcp_fast(q.y));
          const float2 m1 = __fmul2_rn(Nx, Py);
          const float2 Vx = __ffma2_rn(Nx, Px, __fmul2_rn(Ny, Py));
          const float2 Vy = __ffma2_rn(Ny, Px, make_float2(-m1.x, -m1.y));
          const float2 m2 = __fmul2_rn(dzy, Vy);
          const float2 pvx = __ffma2_rn(dzx, Vx, make_float2(-m2.x, -m2.y));
          const float2 pvy = __ffma2_rn(dzx, Vy, __fmul2_rn(dzy, Vx));
          const float2 dwx = __ffma2_rn(pvx, ip, __fadd2_rn(a.wsx, dzx));
          const float2 dwy = __ffma2_rn(make_float2(-pvy.x, -pvy.y), ip, __fadd2_rn(a.wsy, dzy));
          return __ffma2_rn(dwx, dwx, __fmul2_rn(dwy, dwy));
        };
        const float2 irho22 = make_float2(irho2, irho2), one2 = make_float2(1.0f, 1.0f);
        const float2 c1f2 = make_float2(c1f, c1f), c2f2 = make_float2(c2f, c2f);
        // the half-power coefficients, read only by the generic instantiation
        const float2 c1h2 = LAW == 1 ? make_float2(sh.c1h, sh.c1h) : one2;
        const float2 c3h2 = LAW == 1 ? make_float2(sh.c3h, sh.c3h) : one2;
        // the queued points: one per lane, each re-evaluates its stencil
        // (rays m - 2 .. m + 2, signed squared distances, negative inside)
        auto flush_queue = [&]() {
          __syncwarp();
          if (lane < dq_n) {
            const int2 q_ = dq[lane];
            const int m = q_.x, irow = q_.y;
            const int gi_ = irow / gr;
            const float dri_ = ((float)(irow - gi_ * gr) + 0.5f - 0.5f * (float)gr) * dr32;
            const float ri_ = (float)(B.r_lo + (gi_ * gr + 0.5 * gr) * sh.dr64) + dri_;
            float sv[5], fsc = 1.f;
#pragma unroll
            for (int k = 0; k < 5; ++k) {
              float d2;
              const bool in = classify(gi_, ri_, dri_, irow, m - 2 + k, &d2, k == 2 ? &fsc : nullptr);
              sv[k] = in ? __int_as_float(__float_as_int(d2) | 0x80000000) : d2;
            }
            if (signbit(sv[2])) {
              const float I = brightness(-sv[2]);
              float WU;
              const float W = boundary_weight(0, sv, m, irow, nullptr, &WU);
              const float rw = ri_ * bxw;
              // literal rule: I (W - 1); split-profile rule: the limb value c0f
              // with the uniform weight, the rest with f(delta)
              // (a spot scales the point's whole brightness)
              const float term = fsc * (split ? rw * (c0f * (WU - 1.0f) + (I - c0f) * (W - 1.0f)) : rw * I * (W - 1.0f));
              const float y = term - acc_c;
              const float tt = acc_s + y;
              acc_c = (tt - acc_s) - y;
              acc_s = tt;
            }
          }
          __syncwarp();
          dq_n = 0;
        };
        // static task order (warp, warp + NW, ...): the same sums in the same
        // order on every run (dynamic assignment measured no faster)
        for (int task = warp; task < ntask; task += NW) {
          const int rbk = task / nch, chk = task - rbk * nch;
          const int i = rbk * 32 + lane;
          const bool rowok = i < NR;
          const int ii = rowok ? i : NR - 1;
          const int gi = ii / gr;
          const float dri = ((float)(ii - gi * gr) + 0.5f - 0.5f * (float)gr) * dr32;
          const float ri = (float)(B.r_lo + (gi * gr + 0.5 * gr) * sh.dr64) + dri;
          const int c0 = chk * CH, c1 = min(c0 + CH, NTH);
          // the row's inside rays: their count, and the sums of I - c0f =
          // mu (c1f + c2f mu) of the scalar and of the paired evaluations
          int cnt = 0;
          float sj = 0.f;
          float2 sj2 = make_float2(0.f, 0.f);
          float dh;
          // inside flags: bit k = column l - 1 - k before column l; the left
          // halo column c0 - 1 first
          unsigned win = classify(gi, ri, dri, ii, c0 - 1, &dh) ? 1u : 0u;
          float lo2g = 0.f, hi2g = 0.f;  // the current group's band
          int aidx = 0;                  // and its anchor
          AnchorF ar;     // the anchor in registers (triple)
          AnchorP ap;     // the anchor as broadcast pairs (binary)
          // binary: the scalar evaluations read the anchor from the table
          auto anchor = [&]() -> const AnchorF& {
            if constexpr (NL == 2) return anf[aidx];
            else return ar;
          };
          int gbase = 0;  // first column of the current group
          const float* tpf = tabf;  // offsets of the current group: pair rows by column
          const float2 ri2 = make_float2(ri, ri), dri2 = make_float2(dri, dri);
          // queue the boundary points among bits of bm, bit j = column base - j
          auto push_bits = [&](unsigned bm, int base) {
            while (__any_sync(0xffffffffu, bm != 0u)) {
              const bool has = bm != 0u;
              const int m = base - (has ? __ffs(bm) - 1 : 0);
              bm &= bm - 1u;
              unsigned rem = __ballot_sync(0xffffffffu, has);
              // up to 32 points, the queue holds DQ: take the lowest set
              // lanes that fit, flushing whenever the queue is full
              while (rem) {
                if (dq_n == DQ) flush_queue();
                unsigned take = rem;
                const int room = DQ - dq_n;
                if (__popc(take) > room) {
                  take = 0u;
                  unsigned r = rem;
                  for (int k = 0; k < room; ++k) {
                    const unsigned low = r & (0u - r);
                    take |= low;
                    r ^= low;
                  }
                }
                if (take & (1u << lane)) dq[dq_n + __popc(take & lt_mask)] = make_int2(m, i);
                dq_n += __popc(take);
                rem &= ~take;
              }
            }
          };
          // boundary centres among columns l0 - 1 .. l0 + nb - 2 (bit j =
          // column l0 + nb - 2 - j) after the block [l0, l0 + nb); the first
          // block's column c0 - 1 belongs to the previous chunk
          auto centres = [&](int nb, bool first) -> unsigned {
            unsigned bm = ((win & ~((win << 1) & (win >> 1))) >> 1) & ((1u << nb) - 1u);
            if (first) bm &= ~(1u << (nb - 1));
            return rowok ? bm : 0u;
          };
          // an inside ray's share of the row beyond c0f: mu (c1f + c2f mu),
          // plus s (c1h + c3h mu), s = mu^(1/2), when h (half-integer powers)
          // fs: the spot factor (the count adds c0f, so a spotted ray adds
          // fs (c0f + J) - c0f here)
          auto add_in = [&](bool in, float mu, bool h, float fs) {
            float J = mu * fmaf(c2f, mu, c1f);
            if (h) J = fmaf(mu * rsqrt_fast(mu), fmaf(sh.c3h, mu, sh.c1h), J);
            J = fmaf(fs, J, -c0f * (1.0f - fs));
            sj = __fadd_rn(sj, in ? J : 0.0f);
          };
          auto block_end = [&](int l0, int nb, bool first, bool unc) {
            unsigned bm = centres(nb, first);
            if (__any_sync(0xffffffffu, unc || bm != 0u)) {
              if (unc) {
                for (int k = 0; k < nb; ++k) {
                  const cf t = tab_at(l0 + k - gbase);
                  float eb;
                  cf dw;
                  float d2 = ray_eval(anchor(), t.x, t.y, ri, dri, &eb, nullptr, &dw);
                  if (d2 < lo2g || d2 > hi2g) continue;
                  if (decide(d2, eb, ii, l0 + k)) {
                    win |= 1u << (nb - 1 - k);
                    add_in(true, sqrtf(fmaxf(__fmaf_rn(-d2, irho2, 1.0f), 1e-30f)), LAW != 0 && sh.half != 0,
                           spot_factor(aidx, dw, eb, ii, l0 + k));
                  }
                }
                bm = centres(nb, first);
              }
              push_bits(bm, l0 + nb - 2);
            }
            cnt += __popc(win & ((1u << nb) - 1u));
          };
          // one column: classify against the band, flag, and if inside add
          // its share (x > 5 u there, as d^2 < lo2 <= rho^2 (1 - 8 u)); hc:
          // std::true_type for the generic law (half-integer powers of mu or
          // a spot, checked at run time)
          auto col = [&](int l, float tx, float ty, bool& unc, auto hc) {
            cf dw;
            float eb = 0.f;
            constexpr bool GEN = decltype(hc)::value;
            const float d2 = ray_eval(anchor(), tx, ty, ri, dri, GEN ? &eb : nullptr, nullptr, GEN ? &dw : nullptr);
            const bool in = d2 < lo2g;
            unc = unc || !(in || d2 > hi2g);
            win = (win << 1) | (in ? 1u : 0u);
            const float x = __fmaf_rn(-d2, irho2, 1.0f);
            if constexpr (GEN)
              add_in(in, __fmul_rn(x, rsqrt_fast(x)), sh.half != 0, in ? spot_factor(aidx, dw, eb, ii, l) : 1.0f);
            else
              add_in(in, __fmul_rn(x, rsqrt_fast(x)), false, 1.0f);
            (void)l;
          };
          // two columns (l, l + 1) with paired operations (binary lens); the
          // pair row t4 = (x_l, x_l+1, y_l, y_l+1); hh: std::true_type adds the
          // half-integer powers s (c1h + c3h mu), s = mu^(1/2) (no spot)
          auto col2 = [&](const float4 t4, bool& unc, auto hh) {
            const float2 d2 = ray_eval2(ap, make_float2(t4.x, t4.y), make_float2(t4.z, t4.w), ri2, dri2);
            const bool in0 = d2.x < lo2g, in1 = d2.y < lo2g;
            unc = unc || !(in0 || d2.x > hi2g) || !(in1 || d2.y > hi2g);
            win = (win << 2) | (in0 ? 2u : 0u) | (in1 ? 1u : 0u);
            const float2 x = __ffma2_rn(make_float2(-d2.x, -d2.y), irho22, one2);
            const float2 mu = __fmul2_rn(x, make_float2(rsqrt_fast(x.x), rsqrt_fast(x.y)));
            float2 J = __fmul2_rn(mu, __ffma2_rn(c2f2, mu, c1f2));
            if constexpr (decltype(hh)::value) {
              const float2 sq = __fmul2_rn(mu, make_float2(rsqrt_fast(mu.x), rsqrt_fast(mu.y)));
              J = __ffma2_rn(sq, __ffma2_rn(c3h2, mu, c1h2), J);
            }
            sj2 = __fadd2_rn(sj2, make_float2(in0 ? J.x : 0.0f, in1 ? J.y : 0.0f));
          };
          int l = c0;
          bool first = true;
          while (l < c1) {
            const int mgrp = (int)__umulhi((unsigned int)l, gmagic);
            aidx = gi * mth + mgrp;
            lo2g = anf[aidx].lo2;
            hi2g = anf[aidx].hi2;
            if constexpr (NL == 2) ap = pairs_of(anf[aidx]);
            else ar = anf[aidx];
            gbase = mgrp * gth;
            tpf = tabf - 2 * gbase;
            const int lend = min(gbase + gth, c1);
            while (l < lend) {
              const int nb = min(KB, lend - l);
              bool unc = false;
              // a full block, columns l + k, l + k + 1 from one 16-byte row
              // (l + k - gbase even); hc selects the half-power terms
              auto full_block = [&](auto hc) {
#pragma unroll
                for (int k = 0; k < KB; k += 2) {
                  const float4 t4 = *reinterpret_cast<const float4*>(tpf + 2 * (l + k));
                  if constexpr (NL == 2) {
                    col2(t4, unc, hc);
                  } else {
                    col(l + k, t4.x, t4.z, unc, hc);
                    col(l + k + 1, t4.y, t4.w, unc, hc);
                  }
                }
              };
              // (a spot, or the half-integer powers outside the generic
              // instantiation's paired sweep: the scalar loop)
              if (nb == KB && (LAW == 0 || !sh.generic)) {
                full_block(std::false_type{});
              } else if (LAW == 1 && NL == 2 && nb == KB && !sh.spot) {
                full_block(std::true_type{});
              } else {
#pragma unroll 1
                for (int k = 0; k < nb; ++k) {
                  const cf t = tab_at(l + k - gbase);
                  if (LAW != 0 && sh.generic) col(l + k, t.x, t.y, unc, std::true_type{});
                  else col(l + k, t.x, t.y, unc, std::false_type{});
                }
              }
              block_end(l, nb, first, unc);
              first = false;
              l += nb;
            }
          }
          // right halo column c1: finalizes column c1 - 1
          win = (win << 1) | (classify(gi, ri, dri, ii, c1, &dh) ? 1u : 0u);
          push_bits(rowok ? (((win & ~((win << 1) & (win >> 1))) >> 1) & 1u) : 0u, c1 - 1);
          if (rowok) {
            const float rowacc = c0f * (float)cnt + (sj + (sj2.x + sj2.y));
            const float term = ri * rowacc * bxw;
            const float y = term - acc_c;
            const float tt = acc_s + y;
            acc_c = (tt - acc_s) - y;
            acc_s = tt;
          }
        }
        flush_queue();
        } else {
          // ---- derivative ray stage (binary lens).  Per ray with seed a =
          // dRow/dd (dI/dd inside; the paper's sigmoid rule adds its own),
          // the row's sums pg[k] += a dd/dq_k are taken from the ray's FP32
          // geometry (rotated frame R = e^{-i th_m}: Q_j = A_j + dz, u =
          // Delta w' / d, gamma = sum eps_j / Q_j^2):
          //   dd/dz = J u, J = [[1 + g.x, -g.y], [-g.y, 1 - g.x]]
          //   dd/dr_i = (J u) . e^{i phi},  dd/dth_l = (J u) . (i z)
          //   dd/dw_c = -conj(R) u,  dd/da_j.x = -eps_j Re(conj(u) conj(R) Q_j^2) / |Q_j|^4
          //   dd/deps_j = -(u . Q_j) / |Q_j|^2
          // pg: sum a dd/dr_i, sum a dd/dth_l, sum a dd/dth_l (l + 1/2), then
          // d/d(w_c.x, w_c.y, rho, u1, a1.x, a2.x, eps1, eps2).
          const float eps0 = sh.eps32[0], eps1 = sh.eps32[1];
          const bool gradrule = g.grad_rule != 0;
          auto grad_core = [&](const cf dz, const cf dw, float tx, float ty, float ri_, float lwf, const float4 A01,
                               const float2 cs_, float a, float* pgx) {
            const cf Q0 = mk(A01.x + dz.x, A01.y + dz.y), Q1 = mk(A01.z + dz.x, A01.w + dz.y);
            const float i0 = rcp_fast(abs2(Q0)), i1 = rcp_fast(abs2(Q1));
            const float id = rsqrt_fast(fmaxf(abs2(dw), 1e-37f));
            const float ux = dw.x * id, uy = dw.y * id;
            const cf q0 = Q0 * Q0, q1 = Q1 * Q1;
            const cf gm = scl(cj(q0), eps0 * i0 * i0) + scl(cj(q1), eps1 * i1 * i1);
            const float gzx = (1.0f + gm.x) * ux - gm.y * uy;
            const float gzy = -gm.y * ux + (1.0f - gm.x) * uy;
            const float ex = 1.0f + tx, ey = ty;
            const float gr_ = gzx * ex + gzy * ey;
            const float gt_ = ri_ * (gzy * ex - gzx * ey);
            pgx[0] += a * gr_;
            pgx[1] += a * gt_;
            pgx[2] += a * gt_ * lwf;
            const float ct = cs_.x, st = cs_.y;
            pgx[3] -= a * (ct * ux - st * uy);
            pgx[4] -= a * (st * ux + ct * uy);
            // conj(R) Q_j^2 with conj(R) = (ct, st)
            const cf P0 = mk(ct, st) * q0, P1 = mk(ct, st) * q1;
            pgx[7] -= a * eps0 * (ux * P0.x + uy * P0.y) * i0 * i0;
            pgx[8] -= a * eps1 * (ux * P1.x + uy * P1.y) * i1 * i1;
            pgx[9] -= a * (ux * Q0.x + uy * Q0.y) * i0;
            pgx[10] -= a * (ux * Q1.x + uy * Q1.y) * i1;
          };
          // a ray's seed, its value I (inside) into racc and the brightness
          // derivatives into pgx[5], pgx[6]; the paper's gradient rule (Sec.
          // 3.5) gives the indicator chi = Theta(x), x = (rho - d) / rho, the
          // sigmoid derivative S s (1 - s), s = 1 / (1 + e^{-S x}), with the
          // interior weight: seed -I S s (1 - s) / rho on d and I S s (1 - s)
          // d / rho^2 on rho (tangents only)
          // (fs: the ray's spot factor, which scales its brightness)
          auto seed_of = [&](bool in, float d2, float* pgx, float& racc, auto hc, float fs) -> float {
            float a = 0.f;
            if (in) {
              float Id, Ir, Iu;
              racc += fs * brightness_der(d2, &Id, &Ir, &Iu, hc);
              a = fs * Id;
              pgx[5] += fs * Ir;
              pgx[6] += fs * Iu;
            }
            if (gradrule) {
              const float dd_ = sqrtf(d2);
              const float sx = sfac * (1.0f - dd_ / rho32);
              if (fabsf(sx) < 40.0f) {
                const float sg = 1.0f / (1.0f + __expf(-sx));
                const float c = fs * brightness(d2) * sfac * sg * (1.0f - sg);
                a -= c / rho32;
                pgx[5] += c * dd_ / (rho32 * rho32);
              }
            }
            return a;
          };
          // ray l (any column, wrapped) of row irow: its seed a times the
          // gradient of its distance into pgx (generic: anchor from the table)
          auto grad_at = [&](int gi_, float ri_, float dri_, int l, float a, float* pgx) {
            if (a == 0.f || (!B.periodic && (l < 0 || l >= NTH))) return;
            const int lw = wrapl(l);
            const int mgrp = (int)__umulhi((unsigned int)lw, gmagic);
            const int ai = gi_ * mth + mgrp;
            const cf t = tab_at(lw - mgrp * gth);
            cf dz, dw;
            (void)ray_eval(anf[ai], t.x, t.y, ri_, dri_, nullptr, &dz, &dw);
            grad_core(dz, dw, t.x, t.y, ri_, (float)lw + 0.5f, ds.aA[ai], ds.acs[ai], a, pgx);
          };
          // a row's sums (v[0] = sum of I W, v[1 + k] = pg[k]) as its terms
          // of dS_b / d(r_lo, r_hi, th_lo, width) and of H: S_b = sum_i K_i
          // Row_i, K_i = r_i dr dth, r_i = r_lo + (i + 1/2) dr, dr = (r_hi -
          // r_lo) / N_r, dth = width / N_theta
          auto row_terms = [&](int irow, float ri_, const float* v, double* x) {
            const double Rw = (double)v[0], rid = (double)ri_, drd = sh.dr64, dtd = sh.dth64;
            const double Ki = rid * drd * dtd, fi = (irow + 0.5) / NR;
            x[0] = Ki * v[1] * (1.0 - fi) + Rw * ((1.0 - fi) * drd * dtd - rid * dtd / NR);
            x[1] = Ki * v[1] * fi + Rw * (fi * drd * dtd + rid * dtd / NR);
            x[2] = Ki * v[2];
            x[3] = Ki * v[3] / NTH + Rw * rid * drd / NTH;
#pragma unroll
            for (int k = 4; k < 12; ++k) x[k] = Ki * v[k];
          };
          auto kahan = [&](float term) {
            const float y = term - acc_c;
            const float tt = acc_s + y;
            acc_c = (tt - acc_s) - y;
            acc_s = tt;
          };
          // the queued boundary points: one per lane.  FP32 stencil values
          // (the flags), FP64 stencil distances for the crossing and its
          // derivative; the point's value I (W - 1) beyond the I the sweep
          // added, its seed (W - 1) dI/dd, and the crossing seeds on the
          // stencil rays; its row's terms go to the warp's sums directly
          auto flush_queue = [&]() {
            __syncwarp();
            double xq[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) xq[k] = 0.0;
            if (lane < dq_n) {
              const int2 q_ = dq[lane];
              const int m = q_.x, irow = q_.y;
              const int gi_ = irow / gr;
              const float dri_ = ((float)(irow - gi_ * gr) + 0.5f - 0.5f * (float)gr) * dr32;
              const float ri_ = (float)(B.r_lo + (gi_ * gr + 0.5 * gr) * sh.dr64) + dri_;
              float sv[5], fsc = 1.f;
              double dist[5];
#pragma unroll 1
              for (int k = 0; k < 5; ++k) {
                const int l = m - 2 + k;
                float d2;
                const bool in = classify(gi_, ri_, dri_, irow, l, &d2, k == 2 ? &fsc : nullptr);
                sv[k] = in ? __int_as_float(__float_as_int(d2) | 0x80000000) : d2;
                dist[k] = (!B.periodic && (l < 0 || l >= NTH)) ? __longlong_as_double(0x7ff0000000000000LL)
                                                               : ray_distance64<NL>(sh, B, irow, wrapl(l));
              }
              if (signbit(sv[2])) {
                float Id, Ir, Iu;
                float I = (LAW != 0 && sh.generic) ? brightness_der(-sv[2], &Id, &Ir, &Iu, std::true_type{})
                                     : brightness_der(-sv[2], &Id, &Ir, &Iu, std::false_type{});
                // a spot scales the point's brightness and its derivatives
                I *= fsc; Id *= fsc; Ir *= fsc; Iu *= fsc;
                const float W = boundary_weight(m, sv, m, irow, dist);
                float v[12];
#pragma unroll
                for (int k = 0; k < 12; ++k) v[k] = 0.f;
                v[0] = I * (W - 1.0f);
                v[1 + 5] += (W - 1.0f) * Ir;
                v[1 + 6] += (W - 1.0f) * Iu;
                grad_at(gi_, ri_, dri_, m, (W - 1.0f) * Id, v + 1);
                for (int sd = 0; sd < 2; ++sd) {
                  if (!sd_n[sd]) continue;
                  const float c = I * sd_c[sd];
                  v[1 + 5] += c;
                  for (int k = 0; k < sd_n[sd]; ++k) grad_at(gi_, ri_, dri_, sd_b[sd] + k, -c * sd_l[sd][k], v + 1);
                }
                row_terms(irow, ri_, v, xq);
                kahan(ri_ * v[0] * bxw);
              }
            }
            // the points' row terms summed over the warp in a fixed order
#pragma unroll 1
            for (int k = 0; k < 12; ++k) {
              double xs = xq[k];
              for (int o2 = 16; o2 > 0; o2 >>= 1) xs += __shfl_xor_sync(0xffffffffu, xs, o2);
              if (lane == k) wder[warp * 12 + k] += xs;
            }
            __syncwarp();
            dq_n = 0;
          };
          // static task order (warp, warp + NW, ...): every sum of the
          // adjoint is taken in the same order on every run
          for (int task = warp; task < ntask; task += NW) {
            const int rbk = task / nch, chk = task - rbk * nch;
            const int i = rbk * 32 + lane;
            const bool rowok = i < NR;
            const int ii = rowok ? i : NR - 1;
            const int gi = ii / gr;
            const float dri = ((float)(ii - gi * gr) + 0.5f - 0.5f * (float)gr) * dr32;
            const float ri = (float)(B.r_lo + (gi * gr + 0.5 * gr) * sh.dr64) + dri;
            const int c0 = chk * CH, c1 = min(c0 + CH, NTH);
            float rowacc = 0.f;  // sum of I over the row's inside rays
            float pg[11];
#pragma unroll
            for (int k = 0; k < 11; ++k) pg[k] = 0.f;
            float dh;
            unsigned win = classify(gi, ri, dri, ii, c0 - 1, &dh) ? 1u : 0u;
            AnchorF ar;  // the current group's anchor, A_j and angle
            int aiD = 0;  // its index
            float4 A01 = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 cs = make_float2(1.f, 0.f);
            int gbase = 0;
            auto push_bits = [&](unsigned bm, int base) {
              while (__any_sync(0xffffffffu, bm != 0u)) {
                const bool has = bm != 0u;
                const int m = base - (has ? __ffs(bm) - 1 : 0);
                bm &= bm - 1u;
                unsigned rem = __ballot_sync(0xffffffffu, has);
                while (rem) {
                  if (dq_n == DQ) flush_queue();
                  unsigned take = rem;
                  const int room = DQ - dq_n;
                  if (__popc(take) > room) {
                    take = 0u;
                    unsigned r = rem;
                    for (int k = 0; k < room; ++k) {
                      const unsigned low = r & (0u - r);
                      take |= low;
                      r ^= low;
                    }
                  }
                  if (take & (1u << lane)) dq[dq_n + __popc(take & lt_mask)] = make_int2(m, i);
                  dq_n += __popc(take);
                  rem &= ~take;
                }
              }
            };
            auto centres = [&](int nb, bool first) -> unsigned {
              unsigned bm = ((win & ~((win << 1) & (win >> 1))) >> 1) & ((1u << nb) - 1u);
              if (first) bm &= ~(1u << (nb - 1));
              return rowok ? bm : 0u;
            };
            // one column: value, flag and, for a decided ray, its seed and
            // gradient; an undecided ray waits for the block end
            auto colD = [&](int l, const cf t, bool& unc, auto hc) {
              cf dz, dw;
              float eb = 0.f;
              const float d2 = ray_eval(ar, t.x, t.y, ri, dri, decltype(hc)::value ? &eb : nullptr, &dz, &dw);
              const bool in = d2 < ar.lo2;
              const bool u_ = !(in || d2 > ar.hi2);
              unc = unc || u_;
              win = (win << 1) | (in ? 1u : 0u);
              if (!u_) {
                float fs = 1.f;
                if constexpr (decltype(hc)::value) fs = in ? spot_factor(aiD, dw, eb, ii, l) : 1.f;
                const float a = seed_of(in, d2, pg, rowacc, hc, fs);
                if (a != 0.f) grad_core(dz, dw, t.x, t.y, ri, (float)l + 0.5f, A01, cs, a, pg);
              }
            };
            auto block_end = [&](int l0, int nb, bool first, bool unc) {
              unsigned bm = centres(nb, first);
              if (__any_sync(0xffffffffu, unc || bm != 0u)) {
                if (unc) {
                  for (int k = 0; k < nb; ++k) {
                    const cf t = tab_at(l0 + k - gbase);
                    float eb;
                    cf dz, dw;
                    float d2 = ray_eval(ar, t.x, t.y, ri, dri, &eb, &dz, &dw);
                    if (d2 < ar.lo2 || d2 > ar.hi2) continue;
                    const bool in = decide(d2, eb, ii, l0 + k);
                    if (in) win |= 1u << (nb - 1 - k);
                    const float fs = in ? spot_factor(aiD, dw, eb, ii, l0 + k) : 1.f;
                    const float a = (LAW != 0 && sh.generic) ? seed_of(in, d2, pg, rowacc, std::true_type{}, fs)
                                               : seed_of(in, d2, pg, rowacc, std::false_type{}, fs);
                    if (a != 0.f) grad_core(dz, dw, t.x, t.y, ri, (float)(l0 + k) + 0.5f, A01, cs, a, pg);
                  }
                  bm = centres(nb, first);
                }
                push_bits(bm, l0 + nb - 2);
              }
            };
            int l = c0;
            bool first = true;
            while (l < c1) {
              const int mgrp = (int)__umulhi((unsigned int)l, gmagic);
              const int ai = gi * mth + mgrp;
              aiD = ai;
              ar = anf[ai];
              A01 = ds.aA[ai];
              cs = ds.acs[ai];
              gbase = mgrp * gth;
              const int lend = min(gbase + gth, c1);
              while (l < lend) {
                const int nb = min(KB, lend - l);
                bool unc = false;
                if (LAW != 0 && sh.generic) {
#pragma unroll 1
                  for (int k = 0; k < nb; ++k) colD(l + k, tab_at(l + k - gbase), unc, std::true_type{});
                } else {
#pragma unroll 1
                  for (int k = 0; k < nb; ++k) colD(l + k, tab_at(l + k - gbase), unc, std::false_type{});
                }
                block_end(l, nb, first, unc);
                first = false;
                l += nb;
              }
            }
            win = (win << 1) | (classify(gi, ri, dri, ii, c1, &dh) ? 1u : 0u);
            push_bits(rowok ? (((win & ~((win << 1) & (win >> 1))) >> 1) & 1u) : 0u, c1 - 1);
            // the row's terms, summed over the warp's rows
            double x[12];
            float v[12];
            v[0] = rowacc;
#pragma unroll
            for (int k = 0; k < 11; ++k) v[k + 1] = pg[k];
            row_terms(ii, ri, v, x);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
              double xs = rowok ? x[k] : 0.0;
              for (int o2 = 16; o2 > 0; o2 >>= 1) xs += __shfl_xor_sync(0xffffffffu, xs, o2);
              if (lane == k) wder[warp * 12 + k] += xs;
            }
            if (rowok) kahan(ri * rowacc * bxw);
          }
          flush_queue();
        }
      }
      __syncthreads();
      if (DER && tid < 12) {
        double sum = 0.0;
        for (int w = 0; w < NW; ++w) { sum += wder[w * 12 + tid]; wder[w * 12 + tid] = 0.0; }
        if (tid < 4) ds.Gb[bxi][tid] = sum;
        else ds.H[tid - 4] += sum;
      }
    }
    if (st_local) atomicOr(&sh.status, st_local);
    if (diag_cnt && tid == 0) { long long c_ = clock64(); sh.cnt[12] = (int)min(c_ - sh.clk0, 2000000000LL); sh.clk0 = c_; }
    // ------------------------------------------------ 10. reduction
    double v = (double)acc_s - (double)acc_c;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh.red[warp] = v;
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      for (int w = 0; w < NW; ++w) tot += sh.red[w];
      // unspotted normalisation A0 = S / rho^2; a spot divides by the
      // unlensed flux 1 - c F_spot (N = spot_norm); an invalid spot gives NaN
      const double A0 = tot / (sh.rho * sh.rho);
      double A = A0 * sh.spot_norm;
      if (LAW != 0 && sh.spot_bad) A = __longlong_as_double(0x7ff8000000000000LL);
      if (!(A == A) || isinf(A)) sh.status |= ICRS_ST_NAN;
      size_t o = (size_t)s * E + e;
      if (DER) {
        // dA/dp = (sum_b G_b . d bounds_b/dp + H . d(w_c, rho, u1, a, eps)/dp) / rho^2
        //         - 2 S / rho^3 [p = rho]
        double dS[NPAR];
        for (int q = 0; q < NPAR; ++q) dS[q] = 0.0;
        for (int b = 0; b < sh.nbox; ++b)
          for (int q = 0; q < NPAR; ++q)
            dS[q] += ds.Gb[b][0] * bdual[b].r_lo.d[q] + ds.Gb[b][1] * bdual[b].r_hi.d[q] +
                     ds.Gb[b][2] * bdual[b].th_lo.d[q] + ds.Gb[b][3] * bdual[b].width.d[q];
        for (int q = 0; q < 4; ++q) dS[q] += ds.H[0] * ds.dwc[q].x + ds.H[1] * ds.dwc[q].y;
        dS[4] += ds.H[4] * ds.dadp[0][0] + ds.H[5] * ds.dadp[1][0];
        dS[5] += ds.H[4] * ds.dadp[0][1] + ds.H[5] * ds.dadp[1][1] + ds.H[6] * ds.depsq[0] + ds.H[7] * ds.depsq[1];
        dS[6] += ds.H[2];
        dS[7] += ds.H[3];
        const double ir2 = 1.0 / (sh.rho * sh.rho);
        double dA[NPAR];
        for (int q = 0; q < NPAR; ++q) dA[q] = dS[q] * ir2;
        dA[6] -= 2.0 * A0 / sh.rho;
        // the spot's normalisation: dA = N dA0 + A0 dN, dN/du1 = N^2 c dF/du1
        for (int q = 0; q < NPAR; ++q) dA[q] *= sh.spot_norm;
        dA[7] += A * sh.spot_gu;
        bool bad = false;
        for (int q = 0; q < NPAR; ++q) bad |= !(dA[q] == dA[q]) || isinf(dA[q]);
        if (bad) sh.status |= ICRS_ST_NAN;
        if (dout.dA)
          for (int q = 0; q < NPAR; ++q) dout.dA[o * NPAR + q] = dA[q];
        double wgt = 0.0;
        if (dout.gA) wgt = dout.gA[o];
        if (dout.yobs) {
          // chi^2 = sum_e ((y_e - A_e) / sigma_e)^2 with the flux F = A
          const double r_ = (dout.yobs[o] - A) / dout.sig[o];
          wgt = -2.0 * r_ / dout.sig[o];
          if (dout.chi2) atomicAdd(&dout.chi2[s], r_ * r_);
        }
        if (dout.grad)
          for (int q = 0; q < NPAR; ++q) atomicAdd(&dout.grad[(size_t)s * NPAR + q], wgt * dA[q]);
      }
      if (A_out) A_out[o] = A;
      if (st_out) st_out[o] = (sh.status & 0xffu) | ((uint32_t)min(sh.nbox, 255) << 8);
      if (diag_cnt)
        for (int c = 0; c < 16; ++c) diag_cnt[o * 16 + c] = sh.cnt[c];
      if (diag_sect)
        for (int b = 0; b < 10; ++b) {
          double* d = diag_sect + (o * 10 + b) * 5;
          if (b < sh.nbox) { d[0] = sh.box[b].r_lo; d[1] = sh.box[b].r_hi; d[2] = sh.box[b].th_lo; d[3] = sh.box[b].width; d[4] = sh.box[b].periodic; }
          else { d[0] = d[1] = d[2] = d[3] = d[4] = 0.0; }
        }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- point source
// One thread per source position: images and magnification of a point source
// (point_source_solve, shared with the surrogate's feature kernel).
template <int NL>
__global__ void point_source_kernel(const icrs_params* __restrict__ P, int S, const double* __restrict__ W, int n,
                                    icrs_grid g, double* __restrict__ A, double* __restrict__ images,
                                    int32_t* __restrict__ n_img, uint32_t* __restrict__ status) {
  constexpr int N = NL * NL + 1;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)S * n) return;
  const int s = (int)(idx / n);
  const Lens L = make_lens(P[s]);
  const cd w = mk(W[2 * idx], W[2 * idx + 1]);
  const PointSource<NL> r = point_source_solve<NL>(L, w, g.max_iter, g.img_tol, images ? images + idx * N * 2 : nullptr);
  A[idx] = r.A;
  if (n_img) n_img[idx] = r.m;
  if (status) status[idx] = r.st;
}

// ---------------------------------------------------------------- likelihood
// Linear-flux marginalised NLL of one light curve per block (Appendix B,
// Eq. NLL, Woodbury form), and optionally its gradient sum_e dnll/dA_e dA_e/dp
// from the per-epoch derivatives dA [S][E][8].  Fixed-order FP64 sums.
constexpr int NLL_THREADS = 256;

__device__ inline double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < NLL_THREADS / 32; ++w) s += red[w];
  return s;
}

__global__ void __launch_bounds__(NLL_THREADS)
marginal_nll_kernel(const double* __restrict__ A, const double* __restrict__ F, const double* __restrict__ sig,
                    const double* __restrict__ prior, int E, const double* __restrict__ dA,
                    double* __restrict__ nll, double* __restrict__ grad, double* __restrict__ fluxes) {
  __shared__ double red[NLL_THREADS / 32];
  const int s = blockIdx.x;
  const size_t o = (size_t)s * E;
  const double mu0 = prior[4 * s + 0], mu1 = prior[4 * s + 1];
  const double l0 = prior[4 * s + 2], l1 = prior[4 * s + 3];
  // sums over the epochs: M^T C^-1 M, M^T C^-1 r, r^T C^-1 r, ln|C|
  // (r = F - M mu, m_e = (A_e - 1, 1), c_e = 1 / sigma_e^2)
  double saa = 0, sa1 = 0, s11 = 0, sar = 0, s1r = 0, srr = 0, slc = 0, nbad = 0;
  for (int e = threadIdx.x; e < E; e += NLL_THREADS) {
    const double a = A[o + e] - 1.0, sg = sig[o + e];
    const double c = 1.0 / (sg * sg);
    const double r = F[o + e] - mu0 * a - mu1;
    saa += c * a * a; sa1 += c * a; s11 += c;
    sar += c * a * r; s1r += c * r; srr += c * r * r;
    slc += log(sg * sg);
    if (!(sg > 0.0)) nbad += 1.0;
  }
  saa = block_sum(saa, red); sa1 = block_sum(sa1, red); s11 = block_sum(s11, red);
  sar = block_sum(sar, red); s1r = block_sum(s1r, red); srr = block_sum(srr, red);
  slc = block_sum(slc, red); nbad = block_sum(nbad, red);
  // K = Lambda^-1 + M^T C^-1 M and its inverse
  const double k00 = 1.0 / l0 + saa, k01 = sa1, k11 = 1.0 / l1 + s11;
  const double det = k00 * k11 - k01 * k01;
  const double i00 = k11 / det, i01 = -k01 / det, i11 = k00 / det;
  const double kv0 = i00 * sar + i01 * s1r, kv1 = i01 * sar + i11 * s1r;  // K^-1 v
  const double a0 = mu0 + kv0, a1 = mu1 + kv1;                              // posterior mean
  const bool bad = nbad > 0.0 || !(l0 > 0.0) || !(l1 > 0.0) || !(det > 0.0);
  if (threadIdx.x == 0) {
    const double quad = srr - (sar * kv0 + s1r * kv1);
    const double logdet = slc + log(l0) + log(l1) + log(det);
    nll[s] = bad ? __longlong_as_double(0x7ff8000000000000LL) : 0.5 * (quad + logdet);
    if (fluxes) { fluxes[2 * s] = a0; fluxes[2 * s + 1] = a1; }
  }
  if (!grad) return;
  double gq[NPAR];
  for (int q = 0; q < NPAR; ++q) gq[q] = 0.0;
  for (int e = threadIdx.x; e < E; e += NLL_THREADS) {
    const double a = A[o + e] - 1.0, sg = sig[o + e];
    const double c = 1.0 / (sg * sg);
    const double ge = c * ((i00 * a + i01) - (F[o + e] - a * a0 - a1) * a0);
    const double* d = dA + (o + e) * NPAR;
    for (int q = 0; q < NPAR; ++q) gq[q] += ge * d[q];
  }
  for (int q = 0; q < NPAR; ++q) {
    const double v = block_sum(gq[q], red);
    if (threadIdx.x == 0) grad[(size_t)s * NPAR + q] = v;
  }
}

// ---------------------------------------------------------------- host side
static size_t mag_smem_bytes(int NL, const icrs_grid& g, int pmax, int has_plo, bool der, int defer, int nt) {
  const int N = NL * NL + 1;
  const size_t NP = (size_t)g.n_limb * N;
  size_t b = has_plo ? sizeof(cf) * NP : 0;
  b += sizeof(cf) * NP + 4 * sizeof(float) * NP;
  b += sizeof(short) * ((NP + 7) & ~(size_t)7);
  b += 3 * ((NP + 15) & ~(size_t)15);
  b += 2 * sizeof(double) * pmax + sizeof(int) * QMAX + 16 + (sizeof(AnchorF) + sizeof(float2)) * MAXANCH;
  const int NW = nt / 32;
  (void)defer;
  b += sizeof(int) * NW * 2 * dq_entries(NL);  // per-warp boundary queues
  if (der) b += sizeof(DerShared);               // derivative state
  b += sizeof(cf) * (GTH_MAX + 2);
  b += sizeof(cdf) * g.n_limb;
  return b;
}

static int check_grid(const icrs_grid* g) {
  if (!g) return ICRS_EINVAL;
  if (g->n_r < 1 || g->n_r > 4096) return ICRS_EINVAL;
  if (g->n_theta < 8 || g->n_theta > 8192) return ICRS_EINVAL;
  if (g->n_limb < 16 || g->n_limb > 1024) return ICRS_EINVAL;
  if (g->n_bins_r < 2 || g->n_bins_r > MAXRB) return ICRS_EINVAL;
  if (g->n_bins_theta < 2 || g->n_bins_theta > 128) return ICRS_EINVAL;
  if (!(g->delta_c > 0.0) || !(g->margin >= 0.0) || !(g->img_tol > 0.0)) return ICRS_EINVAL;
  if (g->max_iter < 1 || g->max_iter > 10000) return ICRS_EINVAL;
  if (g->ld_split != 0 && g->ld_split != 1) return ICRS_EINVAL;
  if (g->grad_rule != 0 && g->grad_rule != 1) return ICRS_EINVAL;
  if (g->grad_rule && !(g->s_fac > 0.0)) return ICRS_EINVAL;
  return ICRS_OK;
}

// Reads n_lens of the first parameter set from the device (the ABI requires
// all sets of one call to share it).
static int first_n_lens(const icrs_params* p, cudaStream_t st, int* nl) {
  int32_t v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, (const char*)p + offsetof(icrs_params, n_lens), sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return ICRS_ECUDA;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return ICRS_ECUDA;
  if (v != 2 && v != 3) return ICRS_EINVAL;
  *nl = v;
  return ICRS_OK;
}

// Launch of one instantiation at NTB threads per block, with its shared
// memory, point-table size and flags already chosen: occupancy, contiguous
// chunks of epochs per block (warm starts along the light curve).
template <int NL, bool DER, int NTB, int LAW>
static int launch_nt(const icrs_params* p, int S, const double* t, int E, const icrs_grid* g, double* A,
                     uint32_t* status, double* dsect, int32_t* dcnt, float* dpts, const DerOut& dout,
                     cudaStream_t st, const int32_t* items, int n_items, int nsm, size_t smem, int pmax,
                     int has_plo, int defer) {
  if (cudaFuncSetAttribute(mag_kernel<NL, DER, NTB, LAW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return ICRS_ECUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mag_kernel<NL, DER, NTB, LAW>, NTB, smem) != cudaSuccess)
    return ICRS_ECUDA;
  if (per_sm < 1) return ICRS_EUNSUPPORTED;
  long long tiles = items ? (long long)n_items : (long long)S * E;
  long long slots = (long long)nsm * per_sm;
  long long per_block = (tiles + slots - 1) / slots;
  if (per_block < 1) per_block = 1;
  long long blocks = (tiles + per_block - 1) / per_block;
  mag_kernel<NL, DER, NTB, LAW><<<(unsigned)blocks, NTB, smem, st>>>(p, S, t, E, *g, (int)per_block, A, status,
                                                                      dsect, dcnt, dpts, pmax, has_plo, dout, items,
                                                                      n_items, defer);
  return cudaGetLastError() == cudaSuccess ? ICRS_OK : ICRS_ECUDA;
}

// Shared-memory sizing of one (NL, DER) launch: the block size (the
// preferred one, else 512 threads when the preferred layout does not fit),
// the deferred boundary queue (binary forward) if it fits; then, forward,
// the FP64 point table grows (up to one entry per image-limb slot) before
// the lo parts of image positions are added; derivative mode takes the lo
// parts first (fewer FP64 polishes).
template <int NL, bool DER, int LAW>
static int launch_inst(const icrs_params* p, int S, const double* t, int E, const icrs_grid* g, double* A,
                       uint32_t* status, double* dsect, int32_t* dcnt, float* dpts, const DerOut& dout,
                       cudaStream_t st, const int32_t* items = nullptr, int n_items = 0) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ICRS_ECUDA;
  int optin = 0, nsm = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return ICRS_ECUDA;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ICRS_ECUDA;
  int nt = mag_threads(NL, DER);
  auto fits = [&](int pm, int plo, int df) {
    return mag_smem_bytes(NL, *g, pm, plo, DER, df, nt) + sizeof(Shared) <= (size_t)optin;
  };
  int pmax = PMAX_MIN;
  int defer = (NL == 2 && !DER) ? 1 : 0;
  if (!fits(pmax, 0, defer)) defer = 0;
  if (!fits(pmax, 0, defer) && nt != NT_BASE) {
    nt = NT_BASE;
    defer = (NL == 2 && !DER) ? 1 : 0;
    if (!fits(pmax, 0, defer)) defer = 0;
  }
  if (!fits(pmax, 0, defer)) return ICRS_EUNSUPPORTED;
  int has_plo = (DER && fits(pmax, 1, defer)) ? 1 : 0;
  const int np_all = g->n_limb * (NL * NL + 1);
  // the FP64 point table takes the remaining room (16 bytes per entry), up to
  // one entry per image-limb slot
  {
    const size_t used = mag_smem_bytes(NL, *g, 0, has_plo, DER, defer, nt) + sizeof(Shared);
    const size_t room = used < (size_t)optin ? (size_t)optin - used : 0;
    const size_t cap = room / (2 * sizeof(double));
    pmax = (int)(cap < (size_t)np_all ? cap : (size_t)np_all);
    if (pmax < PMAX_MIN) pmax = PMAX_MIN;
  }
  if (!DER) has_plo = fits(pmax, 1, defer) ? 1 : 0;
  const size_t smem = mag_smem_bytes(NL, *g, pmax, has_plo, DER, defer, nt);
  if constexpr (mag_threads(NL, DER) != NT_BASE) {
    if (nt == mag_threads(NL, DER))
      return launch_nt<NL, DER, mag_threads(NL, DER), LAW>(p, S, t, E, g, A, status, dsect, dcnt, dpts, dout, st,
                                                           items, n_items, nsm, smem, pmax, has_plo, defer);
  }
  return launch_nt<NL, DER, NT_BASE, LAW>(p, S, t, E, g, A, status, dsect, dcnt, dpts, dout, st, items, n_items, nsm,
                                          smem, pmax, has_plo, defer);
}

// Binary forward: the linear instantiation, then the generic one (each takes
// its own sets and skips the others; same stream, so they run in order).
static int launch_binary_fwd(const icrs_params* p, int S, const double* t, int E, const icrs_grid* g, double* A,
                             uint32_t* status, double* dsect, int32_t* dcnt, float* dpts, cudaStream_t st,
                             const int32_t* items = nullptr, int n_items = 0) {
  DerOut none = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int rc = launch_inst<2, false, 0>(p, S, t, E, g, A, status, dsect, dcnt, dpts, none, st, items, n_items);
  if (rc) return rc;
  return launch_inst<2, false, 1>(p, S, t, E, g, A, status, dsect, dcnt, dpts, none, st, items, n_items);
}

static int launch_mag(const icrs_params* p, int S, const double* t, int E, const icrs_grid* g,
                      double* A, uint32_t* status, double* dsect, int32_t* dcnt, float* dpts, void* stream) {
  if (S < 0 || E < 0) return ICRS_EINVAL;
  if (S == 0 || E == 0) return check_grid(g);
  if (!p || !t || !A) return ICRS_EINVAL;
  int rc = check_grid(g);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int nl = g->n_lens;
  if (nl == 0) { rc = first_n_lens(p, st, &nl); if (rc) return rc; }
  if (nl != 2 && nl != 3) return ICRS_EINVAL;
  DerOut none = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if (nl == 2) return launch_binary_fwd(p, S, t, E, g, A, status, dsect, dcnt, dpts, st);
  return launch_inst<3, false, 2>(p, S, t, E, g, A, status, dsect, dcnt, dpts, none, st);
}

// Derivative launch (binary lens only): zeroes the accumulated outputs on the
// stream, then runs the derivative instantiation.
static int launch_der(const icrs_params* p, int S, const double* t, int E, const icrs_grid* g, DerOut d,
                      double* A, uint32_t* status, void* stream) {
  if (S < 0 || E < 0) return ICRS_EINVAL;
  int rc = check_grid(g);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (S > 0) {
    if (d.grad && cudaMemsetAsync(d.grad, 0, sizeof(double) * NPAR * (size_t)S, st) != cudaSuccess) return ICRS_ECUDA;
    if (d.chi2 && cudaMemsetAsync(d.chi2, 0, sizeof(double) * (size_t)S, st) != cudaSuccess) return ICRS_ECUDA;
  }
  if (S == 0 || E == 0) return ICRS_OK;
  if (!p || !t) return ICRS_EINVAL;
  int nl = g->n_lens;
  if (nl == 0) { rc = first_n_lens(p, st, &nl); if (rc) return rc; }
  if (nl == 3 || g->ld_split) return ICRS_EUNSUPPORTED;
  if (nl != 2) return ICRS_EINVAL;
  return launch_inst<2, true, 2>(p, S, t, E, g, A, status, nullptr, nullptr, nullptr, d, st);
}

}  // namespace icrs

using namespace icrs;

extern "C" {

int icrs_abi_version(void) { return 3; }

void icrs_grid_default(icrs_grid* g) {
  if (!g) return;
  memset(g, 0, sizeof(*g));
  g->n_r = 64; g->n_theta = 256; g->n_limb = 500;
  g->n_bins_r = 32; g->n_bins_theta = 128; g->max_iter = 100; g->uniform = 0;
  g->n_lens = 2;
  g->delta_c = 0.02; g->margin = 0.05; g->img_tol = 1e-3;
  g->s_fac = 100.0;
}

const char* icrs_strerror(int code) {
  switch (code) {
    case ICRS_OK: return "ok";
    case ICRS_EINVAL: return "invalid argument";
    case ICRS_ECUDA: return "CUDA runtime error";
    case ICRS_ETIMEOUT: return "device wait timed out";
    case ICRS_EUNSUPPORTED: return "unsupported configuration (shared memory or sizes)";
    default: return "unknown error";
  }
}

int icrs_point_source(const icrs_params* p, int S, const double* w, int n, const icrs_grid* g,
                      double* A, double* images, int32_t* n_img, uint32_t* status, void* stream) {
  if (S < 0 || n < 0) return ICRS_EINVAL;
  if (S == 0 || n == 0) return check_grid(g);
  if (!p || !w || !A) return ICRS_EINVAL;
  int rc = check_grid(g);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int nl = g->n_lens;
  if (nl == 0) { rc = first_n_lens(p, st, &nl); if (rc) return rc; }
  if (nl != 2 && nl != 3) return ICRS_EINVAL;
  long long total = (long long)S * n;
  int threads = 128;
  long long blocks = (total + threads - 1) / threads;
  if (blocks > 2147483647LL) return ICRS_EUNSUPPORTED;
  if (nl == 2) point_source_kernel<2><<<(unsigned)blocks, threads, 0, st>>>(p, S, w, n, *g, A, images, n_img, status);
  else point_source_kernel<3><<<(unsigned)blocks, threads, 0, st>>>(p, S, w, n, *g, A, images, n_img, status);
  return cudaGetLastError() == cudaSuccess ? ICRS_OK : ICRS_ECUDA;
}

int icrs_magnification(const icrs_params* p, int S, const double* t, int E, const icrs_grid* g,
                       double* A, uint32_t* status, void* stream) {
  return launch_mag(p, S, t, E, g, A, status, nullptr, nullptr, nullptr, stream);
}

int icrs_magnification_diag(const icrs_params* p, int S, const double* t, int E, const icrs_grid* g,
                            double* A, uint32_t* status, double* sectors, int32_t* counters,
                            float* points, void* stream) {
  return launch_mag(p, S, t, E, g, A, status, sectors, counters, points, stream);
}

size_t icrs_marginal_nll_workspace_bytes(int S, int E) {
  if (S <= 0 || E <= 0) return 0;
  return sizeof(double) * (size_t)S * (size_t)E * (NPAR + 1);
}

int icrs_marginal_nll_grad(const icrs_params* p, int S, const double* t, int E, const icrs_grid* g, const double* F,
                           const double* sigma, const double* prior, double* nll, double* grad, double* fluxes,
                           double* A, uint32_t* status, void* workspace, size_t workspace_bytes, void* stream) {
  if (S < 0 || E < 0) return ICRS_EINVAL;
  int rc = check_grid(g);
  if (rc) return rc;
  if (S == 0) return ICRS_OK;
  if (!p || !prior || !nll || (E > 0 && (!t || !F || !sigma))) return ICRS_EINVAL;
  const size_t need = icrs_marginal_nll_workspace_bytes(S, E);
  if (E > 0 && (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 7u))) return ICRS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  double* dA = (double*)workspace;
  double* Aw = A ? A : (E > 0 ? dA + (size_t)S * E * NPAR : nullptr);
  if (E > 0) {
    if (grad) {
      DerOut d = {nullptr, nullptr, nullptr, dA, nullptr, nullptr};
      rc = launch_der(p, S, t, E, g, d, Aw, status, stream);
    } else {
      rc = launch_mag(p, S, t, E, g, Aw, status, nullptr, nullptr, nullptr, stream);
    }
    if (rc) return rc;
  }
  marginal_nll_kernel<<<S, NLL_THREADS, 0, st>>>(Aw, F, sigma, prior, E, dA, nll, grad, fluxes);
  return cudaGetLastError() == cudaSuccess ? ICRS_OK : ICRS_ECUDA;
}

int icrs_magnification_indexed(const icrs_params* p, int S, const double* t, int E, const int32_t* items, int n,
                               const icrs_grid* g, double* A, uint32_t* status, void* stream) {
  if (S < 0 || E < 0 || n < 0) return ICRS_EINVAL;
  int rc = check_grid(g);
  if (rc) return rc;
  if (S == 0 || E == 0 || n == 0) return ICRS_OK;
  if (!p || !t || !items || !A) return ICRS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int nl = g->n_lens;
  if (nl == 0) { rc = first_n_lens(p, st, &nl); if (rc) return rc; }
  if (nl != 2 && nl != 3) return ICRS_EINVAL;
  DerOut none = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if (nl == 2) return launch_binary_fwd(p, S, t, E, g, A, status, nullptr, nullptr, nullptr, st, items, n);
  return launch_inst<3, false, 2>(p, S, t, E, g, A, status, nullptr, nullptr, nullptr, none, st, items, n);
}

int icrs_magnification_vjp(const icrs_params* p, int S, const double* t, int E, const icrs_grid* g,
                           const double* gA, double* grad, double* dA, double* A, uint32_t* status, void* stream) {
  if (S > 0 && E > 0 && !gA && grad) return ICRS_EINVAL;
  if (S > 0 && !grad && !dA) return ICRS_EINVAL;
  DerOut d = {gA, nullptr, nullptr, dA, grad, nullptr};
  return launch_der(p, S, t, E, g, d, A, status, stream);
}

int icrs_chi2_grad(const icrs_params* p, int S, const double* t, int E, const icrs_grid* g, const double* y,
                   const double* sigma, double* chi2, double* grad, double* A, uint32_t* status, void* stream) {
  if (S > 0 && E > 0 && (!y || !sigma)) return ICRS_EINVAL;
  if (S > 0 && (!chi2 || !grad)) return ICRS_EINVAL;
  DerOut d = {nullptr, y, sigma, nullptr, grad, chi2};
  return launch_der(p, S, t, E, g, d, A, status, stream);
}

}  // extern "C"
