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
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "icrs.h"
#include "icrs_common.cuh"
#include "icrs_df64.cuh"

namespace icrs {

constexpr int NT = 512;          // threads per block (one block per SM)
constexpr int NW = NT / 32;      // warps per block
constexpr int QMAX = 2048;       // work queue
constexpr int PMAX_MIN = 512;    // FP64-polished image-limb points per epoch (at least)
constexpr int MAXT = 32;         // theta runs (<= n_bins_theta / 2)
constexpr int MAXRB = 32;        // r bins per theta run
constexpr int MAXCELL = 96;      // (theta run, r run) cells
constexpr int MAXBOX = 96;       // candidate sectors before merging
constexpr int MAXANCH = 128;     // FP64 anchors per sector
constexpr float TINY_EXTENT = 3e-4f;  // images smaller than this x rho skip FP64 decisions
constexpr float EPS32 = 5.9604645e-8f;  // 2^-24

// Meta bits of an image-limb slot.
constexpr uint8_t M_VALID = 1, M_EXACT = 2, M_UNSURE = 4, M_CAND = 8;

struct Anchor {
  cf ws;        // e^{-i th_m} (f(z_m) - w_c)
  cf A[3];      // e^{-i th_m} (z_m - a_j)
  cf K[3];      // eps_j / A_j
  float e0;     // error bound constant part
  float e1;     // error bound factor of |U|_1
};

struct Box {
  double r_lo, r_hi, th_lo, width;
  int periodic;
};

struct Shared {
  // ---- per parameter set
  Lens L;
  double rho, u1;
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
  unsigned long long tocc;
  int nT, full;
  signed char runT[64];
  int startT[MAXT];
  unsigned int t_rlo_u[MAXT], t_rhi_l[MAXT];
  unsigned long long t_rlo[MAXT], t_rhi[MAXT];
  double rlo[MAXT], hr[MAXT];
  unsigned int rocc[MAXT];
  unsigned long long tmask[MAXT][MAXRB];
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
  double red[NW];
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

__device__ __forceinline__ double wrap_pi(double a) {
  double x = fmod(a + kPi, 2.0 * kPi);
  if (x < 0) x += 2.0 * kPi;
  return x - kPi;
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
template <int NL>
__device__ inline int validate_root64(const Shared& sh, cd z0, cd w, double img_tol, double* r, double* th) {
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
  for (int it = 0; it < 8; ++it) {
    cd p, dp;
    horner2<N, double>(b, x, p, dp);
    if (!(abs2(dp) > 0.0)) break;
    cd st = dv(p, dp);
    x = x - st;
    if (abs2(st) <= 1e-30 * fmax(1.0, abs2(x))) break;
  }
  cd F = lens_map<NL, double>(eps, a, x) - wj;
  double res = sqrt(abs2(F));
  if (!(res <= img_tol)) return 0;
  cd z = x + sh.L.a[j];
  *r = sqrt(z.x * z.x + z.y * z.y);
  *th = atan2(z.y, z.x);
  return 1;
}

// FP64 distance of ray (i, l) of a sector from the source centre, with the
// grid of Sec. 3.3: r_i = r_lo + (i + 1/2) dr, th_l = th_lo + (l + 1/2) dth.
template <int NL>
__device__ inline double ray_distance64(const Shared& sh, const Box& B, int i, int l) {
  double r = B.r_lo + (i + 0.5) * sh.dr64;
  double th = B.th_lo + (l + 0.5) * sh.dth64;
  double s, c;
  sincos(th, &s, &c);
  cd z = mk(r * c, r * s);
  cd w = lens_map<NL, double>(sh.L.eps, sh.L.a, z);
  return sqrt(abs2(w - sh.wc));
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

// ---------------------------------------------------------------- kernel
template <int NL>
__global__ void __launch_bounds__(NT, 1)
mag_kernel(const icrs_params* __restrict__ P, int S, const double* __restrict__ T_, int E,
           icrs_grid g, int tiles_per_block, double* __restrict__ A_out, uint32_t* __restrict__ st_out,
           double* __restrict__ diag_sect, int32_t* __restrict__ diag_cnt, float* __restrict__ diag_pts, int PMAX) {
  constexpr int N = NL * NL + 1;
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
  Anchor* anch = (Anchor*)p;     p += sizeof(Anchor) * MAXANCH;
  cf* tab = (cf*)p;              p += sizeof(cf) * g.n_theta;
  const int seg = g.n_theta < 1024 ? g.n_theta : 1024;
  float* rowbuf = (float*)p;     p += sizeof(float) * NW * (seg + 4);
  cdf* ulimb = (cdf*)p;          p += sizeof(cdf) * K;   // e^{2 pi i k / N_limb} as double-float
  int* wqueue = (int*)p;         // NW x 64 boundary points of the current row

  if (tid == 0) { sh.cur_set = -1; sh.warm = 0; }
  for (int k = tid; k < K; k += NT) {
    double sn, cs;
    sincospi(2.0 * (double)k / (double)K, &sn, &cs);
    ulimb[k].x = df_from_double(cs);
    ulimb[k].y = df_from_double(sn);
  }
  __syncthreads();

  const long long ntiles = (long long)S * E;
  const long long t_begin = (long long)blockIdx.x * tiles_per_block;
  for (long long tile = t_begin; tile < t_begin + tiles_per_block && tile < ntiles; ++tile) {
    const int s = (int)(tile / E), e = (int)(tile % E);
    // ------------------------------------------------ set and epoch set-up
    if (tid == 0) {
      if (s != sh.cur_set) {
        icrs_params prm = P[s];
        sh.L = make_lens(prm);
        sh.rho = prm.rho;
        sh.u1 = prm.u1;
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
      }
      sh.wc = source_centre(P[s], T_[(size_t)s * E + e]);
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
      sh.tocc = 0ull;
    }
    __syncthreads();
    const int ll = sh.L.ll;
    const float rho32 = (float)sh.rho;

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
        df px = two_sum(x.x, sh.aj32[ll][nj].x);
        df py = two_sum(x.y, sh.aj32[ll][nj].y);
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
        int ok = validate_root64<NL>(sh, z0, w, g.img_tol, &r, &th);
        uint8_t m = 0;
        if (ok) {
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
    // image counts per limb point
    for (int k = tid; k < K; k += NT) {
      int m = 0;
      for (int j = 0; j < N; ++j) m += (meta[k * N + j] & M_VALID) ? 1 : 0;
      bool legal = (NL == 2) ? (m == 3 || m == 5) : (m == 4 || m == 6 || m == 8 || m == 10);
      if (!legal) atomicOr(&sh.status, ICRS_ST_IMGCOUNT);
    }
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
        cd w = limb_point64(sh, k, K);
        cd z0 = tod(phi[ps]) + sh.L.a[ll];
        double r, th;
        polish_image64<NL>(sh, z0, w, &r, &th);
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
        d[0] = ex ? (float)pr[pidx[ps]] : r32[ps];
        d[1] = ex ? (float)pt[pidx[ps]] : t32[ps];
        d[2] = (float)meta[ps];
        d[3] = e32[ps];
      }
    }
    if (diag_cnt && tid == 0) { long long c_ = clock64(); sh.cnt[5] = (int)min(c_ - sh.clk0, 2000000000LL); sh.clk0 = c_; }
    // ------------------------------------------------ 2. theta bins
    for (int ps = tid; ps < NP; ps += NT) {
      if (!(meta[ps] & M_VALID) || (meta[ps] & M_EXACT)) continue;
      float u = (t32[ps] + kPiF) / (float)ht;
      float fr = u - floorf(u);
      float d = fminf(fr, 1.0f - fr) * (float)ht;
      float eth = e32[ps] / fmaxf(r32[ps], 1e-30f) + 4.0f * EPS32 * 4.0f;
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
      atomicOr(&sh.tocc, 1ull << t);
    }
    __syncthreads();

    if (diag_cnt && tid == 0) { long long c_ = clock64(); sh.cnt[6] = (int)min(c_ - sh.clk0, 2000000000LL); sh.clk0 = c_; }
    if (diag_cnt && tid == 0) sh.cnt[13] = sh.cnt[0];
    // ------------------------------------------------ 3. theta runs (cyclic)
    if (tid == 0) {
      unsigned long long occ = sh.tocc;
      bool full = true;
      for (int t = 0; t < BT; ++t) if (!((occ >> t) & 1ull)) full = false;
      for (int t = 0; t < 64; ++t) sh.runT[t] = -1;
      int nT = 0;
      if (occ == 0ull) {
        nT = 0;
      } else if (full) {
        for (int t = 0; t < BT; ++t) sh.runT[t] = 0;
        sh.startT[0] = 0;
        nT = 1;
      } else {
        int t0 = 0;
        while ((occ >> t0) & 1ull) ++t0;
        for (int kk = 1; kk <= BT; ++kk) {
          int t = (t0 + kk) % BT;
          if (!((occ >> t) & 1ull)) continue;
          int prev = (t + BT - 1) % BT;
          if ((occ >> prev) & 1ull) sh.runT[t] = sh.runT[prev];
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
        for (int b = 0; b < MAXRB; ++b) { sh.tmask[T][b] = 0ull; sh.rrun[T][b] = -1; }
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
      atomicOr(&sh.tmask[T][b], 1ull << tb[ps]);
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
          unsigned long long below = 0ull, above = 0ull;
          for (int k = 0; k < b; ++k) below |= sh.tmask[T][k];
          for (int k = e2; k < BR; ++k) above |= sh.tmask[T][k];
          unsigned long long shared_ = below & above;
          double rg = sh.rlo[T] + sh.hr[T] * 0.5 * (double)(b + e2);
          bool hit = false;
          for (int t0 = 0; t0 < BT && !hit; t0 += 32) {
            int t = t0 + lane;
            bool in = false;
            if (t < BT && ((shared_ >> t) & 1ull)) {
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
    auto unwrap_t = [&](int ps, double th) -> double {
      int T = sh.runT[tb[ps]];
      double start = -kPi + sh.startT[T] * ht;
      return th < start ? th + 2.0 * kPi : th;
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

    if (diag_cnt && tid == 0) { long long c_ = clock64(); sh.cnt[10] = (int)min(c_ - sh.clk0, 2000000000LL); sh.clk0 = c_; }
    // ------------------------------------------------ 8. sectors (FP64, one thread)
    if (tid == 0) {
      int nb = 0;
      const double m = g.margin;
      for (int T = 0; T < nT; ++T) {
        int c0 = sh.cellbase[T], c1 = sh.cellbase[T + 1];
        for (int c = c0; c < c1 && c < MAXCELL; ++c) {
          if (!sh.c_cnt[c]) continue;
          double rmin = dkey_inv(sh.c_x[c][0]), rmax = dkey_inv(sh.c_x[c][1]);
          double tmin = dkey_inv(sh.c_x[c][2]), tmax = dkey_inv(sh.c_x[c][3]);
          Box B;
          double er = rmax - rmin;
          B.r_lo = rmin - m * er;
          if (B.r_lo < 0.0) B.r_lo = 0.0;
          B.r_hi = rmax + m * er;
          if (sh.origin_in && c == c0) B.r_lo = 0.0;
          double et = tmax - tmin;
          double lo = tmin - m * et, wd = et + 2.0 * m * et;
          if (sh.full || wd >= 2.0 * kPi) { B.periodic = 1; B.th_lo = -kPi; B.width = 2.0 * kPi; }
          else { B.periodic = 0; B.th_lo = lo + (wrap_pi(lo) - lo); B.width = wd; }
          if (nb < MAXBOX) sh.box[nb++] = B;
          else sh.status |= ICRS_ST_OVERFLOW;
        }
      }
      // merge overlapping sectors until none overlap; then cap at N_deg
      auto overlap = [](const Box& a, const Box& b) -> bool {
        if (!(a.r_lo < b.r_hi && b.r_lo < a.r_hi)) return false;
        if (a.periodic || b.periodic) return true;
        double d = fmod(b.th_lo - a.th_lo, 2.0 * kPi);
        if (d < 0) d += 2.0 * kPi;
        return d < a.width || d + b.width > 2.0 * kPi;
      };
      auto unite = [](const Box& a, const Box& b) -> Box {
        Box u;
        u.r_lo = fmin(a.r_lo, b.r_lo);
        u.r_hi = fmax(a.r_hi, b.r_hi);
        if (a.periodic || b.periodic) { u.periodic = 1; u.th_lo = -kPi; u.width = 2.0 * kPi; return u; }
        double dv_ = fmod(b.th_lo - a.th_lo, 2.0 * kPi);
        if (dv_ < 0) dv_ += 2.0 * kPi;
        double d = b.th_lo - a.th_lo + (dv_ - (b.th_lo - a.th_lo));
        double wdt, start;
        if (dv_ < a.width) { start = a.th_lo; wdt = fmax(a.width, d + b.width); }
        else { start = a.th_lo + d - 2.0 * kPi; wdt = fmax(a.width + 2.0 * kPi - d, b.width); }
        if (wdt >= 2.0 * kPi) { u.periodic = 1; u.th_lo = -kPi; u.width = 2.0 * kPi; }
        else { u.periodic = 0; u.th_lo = start + (wrap_pi(start) - start); u.width = wdt; }
        return u;
      };
      auto area = [](const Box& b) -> double { return 0.5 * (b.r_hi * b.r_hi - b.r_lo * b.r_lo) * b.width; };
      for (;;) {
        bool merged = false;
        for (int i = 0; i < nb && !merged; ++i)
          for (int j = i + 1; j < nb && !merged; ++j)
            if (overlap(sh.box[i], sh.box[j])) {
              sh.box[i] = unite(sh.box[i], sh.box[j]);
              for (int k = j; k < nb - 1; ++k) sh.box[k] = sh.box[k + 1];
              --nb;
              merged = true;
            }
        if (merged) continue;
        if (nb <= N) break;
        sh.status |= ICRS_ST_SECTCAP;
        int bi = 0, bj = 1;
        double best = 0.0;
        bool have = false;
        for (int i = 0; i < nb; ++i)
          for (int j = i + 1; j < nb; ++j) {
            Box u = unite(sh.box[i], sh.box[j]);
            double cost = area(u) - area(sh.box[i]) - area(sh.box[j]);
            if (!have || cost < best) { best = cost; bi = i; bj = j; have = true; }
          }
        sh.box[bi] = unite(sh.box[bi], sh.box[bj]);
        for (int k = bj; k < nb - 1; ++k) sh.box[k] = sh.box[k + 1];
        --nb;
      }
      sh.nbox = nb;
    }
    __syncthreads();

    if (diag_cnt && tid == 0) { long long c_ = clock64(); sh.cnt[11] = (int)min(c_ - sh.clk0, 2000000000LL); sh.clk0 = c_; }
    // ------------------------------------------------ 9. rays
    const int NR = g.n_r, NTH = g.n_theta;
    const float u1f = (float)sh.u1;
    const float I0 = g.uniform ? (float)(1.0 / kPi) : (float)(3.0 / (kPi * (3.0 - sh.u1)));
    const float irho2 = 1.0f / (rho32 * rho32);
    const float dcf = (float)g.delta_c;
    float acc_s = 0.f, acc_c = 0.f;  // Kahan sum of this thread
    uint32_t st_local = 0u;
    float* buf = rowbuf + warp * (seg + 4);
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
        mr = min(max(mr, 1), min(4, NR));
        mth = min(mth, MAXANCH / mr);  // the anchor table holds MAXANCH entries
        sh.gth = (NTH + mth - 1) / mth;
        sh.gr = (NR + mr - 1) / mr;
        sh.mth = (NTH + sh.gth - 1) / sh.gth;
        sh.mr = (NR + sh.gr - 1) / sh.gr;
        sh.nanch = sh.mth * sh.mr;
      }
      __syncthreads();
      const int gth = sh.gth, gr = sh.gr, mth = sh.mth;
      const float igth = 1.0f / (float)gth;
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
        Anchor an_;
        an_.ws = tof(R * wsd);
        for (int j = 0; j < NL; ++j) {
          cd Aj = R * (zc - sh.L.a[j]);
          an_.A[j] = tof(Aj);
          an_.K[j] = tof(scl(inv(Aj), sh.L.eps[j]));
        }
        // error bound of |Delta w'|: anchor term plus rounding of the ray's
        // offset (at most the group half-diagonal) and of its image term
        double half = 0.5 * gr * sh.dr64 + (B.r_hi) * 0.5 * gth * sh.dth64;
        an_.e0 = (float)(16.0 * EPS32 * (fabs(an_.ws.x) + fabs(an_.ws.y) + 2.0 * half));
        an_.e1 = (float)(16.0 * EPS32 * half);
        anch[an] = an_;
      }
      // offsets within a theta group: (cos d - 1, sin d), d = (o + 1/2 - gth/2) dth
      for (int o = tid; o < gth; o += NT) {
        float d = ((float)o + 0.5f - 0.5f * (float)gth) * sh.dth32;
        float s, c;
        sincosf(d, &s, &c);
        float sh2 = sinf(0.5f * d);
        tab[o] = mk(-2.0f * sh2 * sh2, s);
        (void)c;
      }
      __syncthreads();
      const float dr32 = sh.dr32;
      const float bxw = (float)(sh.dr64 * sh.dth64);
      for (int i = warp; i < NR; i += NW) {
        const int gi = i / gr;
        const float dri = ((float)(i - gi * gr) + 0.5f - 0.5f * (float)gr) * dr32;
        const double rc64 = B.r_lo + (gi * gr + 0.5 * gr) * sh.dr64;
        const float ri = (float)(rc64) + dri;
        float rowacc = 0.f;
        for (int s0 = 0; s0 < NTH; s0 += seg) {
          const int s1 = min(s0 + seg, NTH);
          const int lo = s0 - 2, cnt = (s1 + 2) - lo;
          // signed squared distances of the segment's rays and a 2-ray halo
          // (negative: inside the source; +inf: beyond a non-periodic grid
          // edge); two independent rays per lane and iteration
          auto ray_d2 = [&](int lw, float* d2o) -> bool {
            int mgrp = __float2int_rz((float)lw * igth);
            if (mgrp * gth > lw) --mgrp;
            else if ((mgrp + 1) * gth <= lw) ++mgrp;
            int o = lw - mgrp * gth;
            const Anchor& an_ = anch[gi * mth + mgrp];
            cf t = tab[o];
            cf dz = mk(fmaf(ri, t.x, dri), ri * t.y);
            cf U;
            if constexpr (NL == 2) {
              cf Q0 = an_.A[0] + dz, Q1 = an_.A[1] + dz;
              float n0 = abs2(Q0), n1 = abs2(Q1);
              float ip = __frcp_rn(n0 * n1);
              cf t0 = an_.K[0] * cj(Q0), t1 = an_.K[1] * cj(Q1);
              U = scl(scl(t0, n1) + scl(t1, n0), ip);
            } else {
              cf Q0 = an_.A[0] + dz, Q1 = an_.A[1] + dz, Q2 = an_.A[2] + dz;
              float n0 = abs2(Q0), n1 = abs2(Q1), n2 = abs2(Q2);
              float n01 = n0 * n1;
              float ip = __frcp_rn(n01 * n2);
              cf t0 = an_.K[0] * cj(Q0), t1 = an_.K[1] * cj(Q1), t2 = an_.K[2] * cj(Q2);
              U = scl(scl(t0, n1 * n2) + scl(t1, n0 * n2) + scl(t2, n01), ip);
            }
            cf pz = dz * U;
            cf dw = mk(an_.ws.x + dz.x + pz.x, an_.ws.y + dz.y - pz.y);
            float d2 = abs2(dw);
            float eb = fmaf(an_.e1, fabsf(U.x) + fabsf(U.y), an_.e0);
            *d2o = d2;
            return fabsf(d2 - rho32 * rho32) <= 2.0f * rho32 * eb + eb * eb;  // FP32 cannot decide
          };
          auto wrapl = [&](int l) -> int { return l < 0 ? l + NTH : (l >= NTH ? l - NTH : l); };
          for (int m0 = lane; m0 < cnt; m0 += 64) {
            const int m1 = m0 + 32;
            const int l0 = lo + m0, l1 = lo + m1;
            const bool x0 = !B.periodic && (l0 < 0 || l0 >= NTH);
            const bool x1 = m1 >= cnt || (!B.periodic && (l1 < 0 || l1 >= NTH));
            const int lw0 = x0 ? 0 : wrapl(l0), lw1 = x1 ? 0 : wrapl(l1);
            float a0, a1;
            bool u0 = ray_d2(lw0, &a0);
            bool u1 = ray_d2(lw1, &a1);
            float v0 = a0 < rho32 * rho32 ? -a0 : a0;
            float v1 = a1 < rho32 * rho32 ? -a1 : a1;
            if (!x0 && u0) {
              double d64 = ray_distance64<NL>(sh, B, i, lw0);
              if (diag_cnt) atomicAdd(&sh.cnt[2], 1);
              float q = (float)(d64 * d64);
              v0 = d64 < sh.rho ? -q : q;
            }
            if (!x1 && u1) {
              double d64 = ray_distance64<NL>(sh, B, i, lw1);
              if (diag_cnt) atomicAdd(&sh.cnt[2], 1);
              float q = (float)(d64 * d64);
              v1 = d64 < sh.rho ? -q : q;
            }
            if (v0 == 0.f && a0 < rho32 * rho32) v0 = -0.0f;
            if (v1 == 0.f && a1 < rho32 * rho32) v1 = -0.0f;
            buf[m0] = x0 ? __int_as_float(0x7f800000) : v0;
            if (m1 < cnt) buf[m1] = x1 ? __int_as_float(0x7f800000) : v1;
          }
          __syncwarp();
          // per-point weights (Appendix A).  Points with both neighbours
          // inside (W = 1) are summed directly; points next to the image
          // boundary are queued per warp and their crossings solved with one
          // point per lane.
          auto brightness = [&](float d2) -> float {
            if (g.uniform) return I0;
            float x = fmaxf(0.f, 1.0f - d2 * irho2);
            float sx = x > 0.f ? x * rsqrtf(x) : 0.f;
            return I0 * (1.0f - u1f * (1.0f - sx));
          };
          auto boundary_weight = [&](int mi) -> float {
            float d2 = -buf[mi];
            float vl = buf[mi - 1], vr = buf[mi + 1];
            bool Lin = signbit(vl), Rin = signbit(vr);
            float W;
              float fL = 0.f, fR = 0.f;
              for (int side = 0; side < 2; ++side) {
                bool isL = side == 0;
                if (isL ? Lin : Rin) continue;
                float vo = isL ? vl : vr;
                float delta;
                if (isinf(vo)) {
                  delta = 0.5f;
                  st_local |= ICRS_ST_EDGE;
                } else {
                  // stencil: entering (-2,-1,0,+1), exiting (-1,0,+1,+2)
                  float xs[4], ys[4];
                  int np_ = 0;
                  const int c0 = isL ? -2 : -1;
                  for (int c = 0; c < 4; ++c) {
                    float vv = buf[mi + c0 + c];
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
                    int l = lo + mi;
                    double xsd[4], ysd[4];
                    int nd = 0;
                    double yin = 0, yout = 0;
                    for (int c = 0; c < 4; ++c) {
                      int ll2 = l + c0 + c;
                      if (!B.periodic && (ll2 < 0 || ll2 >= NTH)) continue;
                      int lw2 = ((ll2 % NTH) + NTH) % NTH;
                      xsd[nd] = (double)(c0 + c);
                      ysd[nd] = ray_distance64<NL>(sh, B, i, lw2);
                      if (c0 + c == 0) yin = ysd[nd];
                      if (c0 + c == (isL ? -1 : 1)) yout = ysd[nd];
                      ++nd;
                    }
                    if (diag_cnt) atomicAdd(&sh.cnt[3], 1);
                    double xd = crossing_solve<double>(ysd, xsd[0], nd, yin, yout, isL ? -1.0 : 1.0, sh.rho, 1e-14, 60);
                    double dd = isL ? -xd : xd;
                    delta = (float)dd;
                    float fv = (float)fdelta<double>(dd, g.delta_c, 0);
                    if (isL) fL = fv; else fR = fv;
                    continue;
                  }
                }
                float fv = fdelta<float>(delta, dcf, g.uniform);
                if (isL) fL = fv; else fR = fv;
              }
              if (Lin) W = fR;
              else if (Rin) W = fL;
              else W = fmaxf(0.f, fL + fR - 1.0f);
            return W;
          };
          int* wq = wqueue + warp * 64;
          int nq = 0;
          for (int base = 2; base < cnt - 2; base += 32) {
            const int mi = base + lane;
            bool inside = false, edge = false;
            if (mi < cnt - 2) {
              float v = buf[mi];
              inside = signbit(v);
              if (inside) {
                bool Lin = signbit(buf[mi - 1]), Rin = signbit(buf[mi + 1]);
                if (Lin && Rin) rowacc += brightness(-v);
                else edge = true;
              }
            }
            unsigned msk = __ballot_sync(0xffffffffu, edge);
            if (msk) {
              int pos = nq + __popc(msk & ((1u << lane) - 1u));
              if (edge) {
                if (pos < 64) wq[pos] = mi;
                else rowacc = fmaf(brightness(-buf[mi]), boundary_weight(mi), rowacc);
              }
              nq += __popc(msk);
            }
          }
          __syncwarp();
          for (int q = lane; q < min(nq, 64); q += 32) {
            int mi = wq[q];
            rowacc = fmaf(brightness(-buf[mi]), boundary_weight(mi), rowacc);
          }
          __syncwarp();
        }
        // Kahan-compensated accumulation of r_i dtheta dr sum_l I W
        float term = ri * rowacc * bxw;
        float y = term - acc_c;
        float tt = acc_s + y;
        acc_c = (tt - acc_s) - y;
        acc_s = tt;
      }
      __syncthreads();
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
      double A = tot / (sh.rho * sh.rho);
      if (!(A == A) || isinf(A)) sh.status |= ICRS_ST_NAN;
      A_out[(size_t)s * E + e] = A;
      if (st_out) st_out[(size_t)s * E + e] = (sh.status & 0xffu) | ((uint32_t)min(sh.nbox, 255) << 8);
      size_t o = (size_t)s * E + e;
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
template <int NL>
__global__ void point_source_kernel(const icrs_params* __restrict__ P, int S, const double* __restrict__ W, int n,
                                    icrs_grid g, double* __restrict__ A, double* __restrict__ images,
                                    int32_t* __restrict__ n_img, uint32_t* __restrict__ status) {
  constexpr int N = NL * NL + 1;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)S * n) return;
  int s = (int)(idx / n);
  Lens L = make_lens(P[s]);
  cd w = mk(W[2 * idx], W[2 * idx + 1]);
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
  uint32_t st = 0;
  if (ehrlich_aberth_f32<N>(b, z, g.max_iter, 4.0f * EPS32, last) < 0) st |= ICRS_ST_NONCONV;
  // candidate roots in the original frame (FP64); for a triple lens the roots
  // nearest the second light lens come from a second EA about that lens
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
    if (ehrlich_aberth_f32<N>(b2, z2, g.max_iter, 4.0f * EPS32, last) < 0) st |= ICRS_ST_NONCONV;
    for (int j = 0; j < N; ++j) {
      cd z0 = tod(z2[j]) + L.a[l2];
      int nj = 0;
      double best = abs2(z0 - L.a[0]);
      for (int i = 1; i < NL; ++i) { double d = abs2(z0 - L.a[i]); if (d < best) { best = d; nj = i; } }
      if (nj != l2) continue;
      if (nc < 2 * N) cand[nc++] = z0;
    }
  }
  // FP64 polish on the polynomial about each root's nearest lens, then
  // validation against img_tol (the same as the sector path's FP64 checks).
  double Asum = 0.0;
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
    if (!(sqrt(abs2(F)) <= g.img_tol)) continue;
    if (m >= N) { st |= ICRS_ST_OVERFLOW; break; }
    cd gm = shear<NL, double>(epsd, aj, x);
    Asum += 1.0 / fabs(1.0 - abs2(gm));
    if (images) {
      cd zz = x + L.a[nj];
      images[(idx * N + m) * 2] = zz.x;
      images[(idx * N + m) * 2 + 1] = zz.y;
    }
    ++m;
  }
  bool legal = (NL == 2) ? (m == 3 || m == 5) : (m == 4 || m == 6 || m == 8 || m == 10);
  if (!legal) st |= ICRS_ST_IMGCOUNT;
  if (images)
    for (int j = m; j < N; ++j) { images[(idx * N + j) * 2] = 0.0; images[(idx * N + j) * 2 + 1] = 0.0; }
  A[idx] = Asum;
  if (n_img) n_img[idx] = m;
  if (status) status[idx] = st;
}

// ---------------------------------------------------------------- host side
static size_t mag_smem_bytes(int NL, const icrs_grid& g, int pmax) {
  const int N = NL * NL + 1;
  const size_t NP = (size_t)g.n_limb * N;
  size_t b = 0;
  b += sizeof(cf) * NP + 4 * sizeof(float) * NP;
  b += sizeof(short) * ((NP + 7) & ~(size_t)7);
  b += 3 * ((NP + 15) & ~(size_t)15);
  b += 2 * sizeof(double) * pmax + sizeof(int) * QMAX + sizeof(Anchor) * MAXANCH;
  b += sizeof(int) * NW * 64;  // per-warp boundary queues
  b += sizeof(cf) * g.n_theta;
  const int seg = g.n_theta < 1024 ? g.n_theta : 1024;
  b += sizeof(float) * NW * (seg + 4);
  b += sizeof(cdf) * g.n_limb;
  return b;
}

static int check_grid(const icrs_grid* g) {
  if (!g) return ICRS_EINVAL;
  if (g->n_r < 1 || g->n_r > 4096) return ICRS_EINVAL;
  if (g->n_theta < 8 || g->n_theta > 8192) return ICRS_EINVAL;
  if (g->n_limb < 16 || g->n_limb > 1024) return ICRS_EINVAL;
  if (g->n_bins_r < 2 || g->n_bins_r > MAXRB) return ICRS_EINVAL;
  if (g->n_bins_theta < 2 || g->n_bins_theta > 64) return ICRS_EINVAL;
  if (!(g->delta_c > 0.0) || !(g->margin >= 0.0) || !(g->img_tol > 0.0)) return ICRS_EINVAL;
  if (g->max_iter < 1 || g->max_iter > 10000) return ICRS_EINVAL;
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

}  // namespace icrs

using namespace icrs;

extern "C" {

int icrs_abi_version(void) { return 1; }

void icrs_grid_default(icrs_grid* g) {
  if (!g) return;
  memset(g, 0, sizeof(*g));
  g->n_r = 64; g->n_theta = 256; g->n_limb = 500;
  g->n_bins_r = 32; g->n_bins_theta = 64; g->max_iter = 100; g->uniform = 0;
  g->n_lens = 2;
  g->delta_c = 0.02; g->margin = 0.05; g->img_tol = 1e-3;
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
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ICRS_ECUDA;
  int optin = 0, nsm = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // the FP64 table takes whatever shared memory is left (up to 4096 entries)
  int pmax = PMAX_MIN;
  size_t smem = mag_smem_bytes(nl, *g, pmax);
  if (smem + sizeof(Shared) > (size_t)optin) return ICRS_EUNSUPPORTED;
  while (pmax < 4096 && mag_smem_bytes(nl, *g, pmax * 2) + sizeof(Shared) <= (size_t)optin) pmax *= 2;
  smem = mag_smem_bytes(nl, *g, pmax);
  cudaError_t ce;
  if (nl == 2) ce = cudaFuncSetAttribute(mag_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else ce = cudaFuncSetAttribute(mag_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (ce != cudaSuccess) return ICRS_ECUDA;
  int per_sm = 0;
  if (nl == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mag_kernel<2>, NT, smem);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mag_kernel<3>, NT, smem);
  if (per_sm < 1) return ICRS_EUNSUPPORTED;
  long long tiles = (long long)S * E;
  long long slots = (long long)nsm * per_sm;
  // contiguous chunks of epochs per block (warm starts along the light curve)
  long long per_block = (tiles + slots - 1) / slots;
  if (per_block < 1) per_block = 1;
  long long blocks = (tiles + per_block - 1) / per_block;
  if (nl == 2)
    mag_kernel<2><<<(unsigned)blocks, NT, smem, st>>>(p, S, t, E, *g, (int)per_block, A, status, dsect, dcnt, dpts, pmax);
  else
    mag_kernel<3><<<(unsigned)blocks, NT, smem, st>>>(p, S, t, E, *g, (int)per_block, A, status, dsect, dcnt, dpts, pmax);
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

}  // extern "C"
