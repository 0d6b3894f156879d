/*
 * icrs.h - C ABI of the GB300 image-centred ray shooting (ICRS) library.
 *
 * The library computes microlensing magnifications of a limb-darkened
 * extended source by a binary or triple point-mass lens with the ICRS method
 * of Miyazaki & Kawahara (arXiv:2510.02639, "microJAX"):
 *   - point-source images from the roots of the complex lens polynomial
 *     (Sec. 2.1, Eqs. lens_eq, amp_point, detJ, lens_eq_z; Ehrlich-Aberth
 *     iteration, Sec. 3.1),
 *   - image-centred polar sectors built from binned image-limb points
 *     (Sec. 3.2),
 *   - a fixed N_r x N_theta polar grid per sector whose rays are mapped
 *     through the lens equation, with the uniform / linear limb-darkening
 *     quadrature of Appendix A (Sec. 3.3).
 *
 * Conventions used by every entry point
 *   - All array arguments are DEVICE pointers owned by the caller (for
 *     example torch.Tensor.data_ptr()), contiguous, row-major.  Structs passed
 *     by pointer as "host" are read on the host before the call returns.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued on it and the entry points return without synchronising it
 *     (except when icrs_grid.n_lens = 0, see there).
 *   - The library allocates no device memory in these entry points.
 *   - Return value: ICRS_OK or an error code below; on error nothing has been
 *     enqueued (argument errors) or the CUDA error is reported (ICRS_ECUDA).
 *   - Kernels never trap: per-item problems are reported in `status` words.
 */
#ifndef ICRS_H
#define ICRS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define ICRS_OK 0
#define ICRS_EINVAL 1        /* bad argument: NaN, q <= 0, rho <= 0, grid out of range */
#define ICRS_ECUDA 2         /* a CUDA runtime call failed */
#define ICRS_ETIMEOUT 3      /* a bounded device wait expired */
#define ICRS_EUNSUPPORTED 4  /* valid request this build cannot serve (e.g. shared memory) */

/* Per-item status bits (OR-ed). */
#define ICRS_ST_NONCONV 1u   /* a root iteration hit its iteration cap */
#define ICRS_ST_IMGCOUNT 2u  /* illegal image count (binary: 3 or 5; triple: 4,6,8,10) */
#define ICRS_ST_SECTCAP 4u   /* more sectors than N_deg: the closest ones were merged */
#define ICRS_ST_EDGE 8u      /* an inside ray touched a non-periodic grid edge */
#define ICRS_ST_NAN 16u      /* non-finite result */
#define ICRS_ST_OVERFLOW 32u /* an on-chip table overflowed; a decision was taken in FP32 */
#define ICRS_ST_LIMB 64u     /* surrogate features: the image count changes across the source disk */
#define ICRS_ST_ROUGH 128u   /* surrogate features: the limb magnification varies on the source's scale */
#define ICRS_ST_SPOT (1u << 16)    /* surrogate features: the source has a spot (not radially symmetric) */
#define ICRS_ST_PROFILE (1u << 17) /* surrogate features: the law has u2 or a1..a4, which no network input carries */
/* Threshold of ICRS_ST_ROUGH: the angular harmonics of order >= 3 of A_ps
 * along the 32 limb points, summed in magnitude over both signs of the order,
 * relative to A_ps at the centre. */
#define ICRS_ROUGH_MAX 1e-3
/* icrs_magnification also stores the number of sectors integrated for the
 * epoch in bits 8..15 of its status word. */
#define ICRS_ST_NSECT(st) (((st) >> 8) & 0xffu)

/*
 * Model parameters of one light curve (one "parameter set").
 *   t0, tE      time of closest approach to the origin, Einstein time (days)
 *   u0, alpha   impact parameter and trajectory angle to the binary axis:
 *               w_c(t) = tau (cos a, sin a) + u0 (-sin a, cos a),
 *               tau = (t - t0) / tE                       (Sec. 3.5, Fig. 3)
 *   rho         source radius in Einstein radii (> 0)
 *   u1          linear limb-darkening coefficient (Appendix A.2)
 *   u2          quadratic limb-darkening coefficient (0: the linear law of
 *               Appendix A.2)
 *   a1..a4      coefficients of the power series in mu^(1/2) (the
 *               four-coefficient law; all 0: the linear or quadratic law):
 *               I = I0 [1 - u1 (1 - mu) - u2 (1 - mu)^2 - sum_k a_k (1 - mu^(k/2))],
 *               mu = sqrt(1 - d^2/rho^2),
 *               I0 = 1 / (pi (1 - u1/3 - u2/6 - sum_k a_k k/(k+4)))
 *               (unit total flux).  I must stay positive on the disk (the
 *               caller's responsibility).
 *   spot_x, spot_y, spot_r, spot_c
 *               a circular spot (spot_c = 0: none): centre (spot_x, spot_y)
 *               rho from the source centre (lens-plane axes), radius spot_r
 *               rho, brightness times (1 - spot_c) inside it; the spot must
 *               lie inside the disk (hypot(spot_x, spot_y) + spot_r <= 1,
 *               0 <= spot_r, spot_c < 1), else A is NaN with ICRS_ST_NAN.
 *               A ray inside the spot is weighted by (1 - spot_c) (no
 *               sub-pixel rule at the spot's edge); the unlensed flux is
 *               1 - spot_c F_spot (F_spot by quadrature).
 *   n_lens      2 (binary) or 3 (triple)
 *   binary:     s = separation, q = m2/m1 (> 0); masses eps1 = 1/(1+q),
 *               eps2 = q/(1+q); lenses on the real axis with the primary at
 *               -q s/(1+q), origin at the centre of mass (Eq. lens_eq).
 *   triple:     q2, q3 = mass fractions of lenses 2 and 3, eps1 = 1 - q2 - q3;
 *               lenses 1, 2 on the real axis s2 apart with the origin at their
 *               barycentre; lens 3 at (midpoint of 1,2) + s3 e^{i psi} (Fig. 3).
 */
typedef struct {
  double t0, tE, u0, alpha, rho, u1;
  int32_t n_lens;
  int32_t reserved;
  double s, q;
  double q2, q3, s2, s3, psi;
  double u2;
  double a1, a2, a3, a4;
  double spot_x, spot_y, spot_r, spot_c;
} icrs_params;

/*
 * Discretisation (host struct).
 *   n_r, n_theta   polar grid per sector (Sec. 3.3): 1..4096, 8..8192
 *   n_limb         source-limb points (Sec. 3.2): 16..1024
 *   n_bins_r       radial bins per angular interval: 2..32
 *   n_bins_theta   angular bins over [-pi, pi): 2..128
 *   max_iter       cap on root iterations
 *   uniform        1: uniform source (Appendix A.1 rule), 0: limb darkening
 *                  (u1, u2 of the parameter set)
 *   delta_c        threshold of the LD correction f(delta) (Appendix A.2), > 0
 *   margin         sector widening, fraction of the extent per side (>= 0)
 *   img_tol        lens-equation residual below which a root is an image
 *   n_lens         see the field comment
 *   ld_split       0: the boundary points' weight f(delta) multiplies the whole
 *                  brightness (Appendix A.2); 1: split-profile rule (a
 *                  variant): the limb value I_limb = I(mu = 0), which
 *                  jumps to zero across the edge, takes the uniform weight
 *                  f_U(delta) = delta + 1/2, and I - I_limb, which vanishes at
 *                  the edge like a square root, takes f(delta).  Forward
 *                  entry points only (the derivative ones return
 *                  ICRS_EUNSUPPORTED).
 *   grad_rule      derivative entry points: 0 = the exact almost-everywhere
 *                  derivative of the discrete method; 1 = the paper's
 *                  gradient rules (Sec. 3.5): the inclusion indicator chi =
 *                  Theta(x), x = (rho - d)/rho, gets the derivative of a
 *                  sigmoid of steepness s_fac, S s (1 - s) with s = 1/(1 +
 *                  e^{-S x}), on every ray with the interior weight, and the
 *                  limb-darkening correction f(delta) the fixed derivative
 *                  2/3 of its second-order branch.  Values are unchanged.
 *   s_fac          steepness S of that sigmoid (> 0 when grad_rule = 1)
 */
typedef struct {
  int32_t n_r, n_theta, n_limb, n_bins_r, n_bins_theta, max_iter, uniform;
  int32_t n_lens;  /* lens count shared by every set of the call (2 or 3); 0 = read it
                      from the first set on the device, which synchronises `stream` */
  double delta_c, margin, img_tol;
  int32_t ld_split;
  int32_t grad_rule;
  double s_fac;
} icrs_grid;

/* Fills `g` with the library defaults (64 x 256 grid, 500 limb points, 32 x 128
 * bins, delta_c = 0.02, margin = 0.05, img_tol = 1e-3, limb darkening, the
 * literal boundary rule, the exact derivative (grad_rule = 0, s_fac = 100),
 * n_lens = 2). */
void icrs_grid_default(icrs_grid* g);

/*
 * Point-source magnification A = sum_j 1/|det J(z_j)| (Eqs. amp_point, detJ).
 *   p       [S] device icrs_params
 *   w       [S][n][2] device double: source positions (x, y) per set
 *   A       [S][n] device double (out)
 *   images  [S][n][N_deg][2] device double or NULL (out): image positions,
 *           first n_img[i] entries valid; N_deg = 5 (binary) or 10 (triple)
 *   n_img   [S][n] device int32 or NULL (out)
 *   status  [S][n] device uint32 or NULL (out): ICRS_ST_* bits
 * Images are roots of the lens polynomial whose lens-equation residual is
 * below img_tol (FP32 Ehrlich-Aberth, FP64 polish and validation).
 */
int icrs_point_source(const icrs_params* p, int S, const double* w, int n,
                      const icrs_grid* g, double* A, double* images,
                      int32_t* n_img, uint32_t* status, void* stream);

/*
 * Finite-source magnification of S light curves x E epochs (Sec. 3,
 * Appendix A).
 *   p       [S] device icrs_params (all sets must share n_lens)
 *   t       [S][E] device double: epoch times
 *   g       host icrs_grid
 *   A       [S][E] device double (out)
 *   status  [S][E] device uint32 or NULL (out)
 * One persistent CUDA kernel runs the whole per-epoch path: limb roots,
 * sectors, rays and the brightness reduction.  A binary lens launches it
 * twice on the stream: an instantiation for the sets whose law has no
 * half-integer powers and no spot, then one for the other sets; each skips
 * the other's sets, so every (set, epoch) is computed once.  Errors: ICRS_EINVAL for bad
 * sizes or grid, ICRS_EUNSUPPORTED if the grid needs more shared memory than
 * an SM has, ICRS_ECUDA on launch failure.
 */
int icrs_magnification(const icrs_params* p, int S, const double* t, int E,
                       const icrs_grid* g, double* A, uint32_t* status,
                       void* stream);

/*
 * icrs_magnification plus per-epoch diagnostics (for tests and profiling):
 *   sectors   [S][E][10][5] device double or NULL: the sectors integrated,
 *             (r_lo, r_hi, theta_lo, width, periodic), unused rows zero
 *   counters  [S][E][16] device int32 or NULL: [0] image-limb points polished
 *             in FP64, [1] roots validated in FP64, [2] rays recomputed in
 *             FP64, [3] boundary crossings recomputed in FP64, [4..12] SM
 *             clock cycles spent in the kernel's phases (roots, FP64
 *             validation, theta bins, theta runs and r ranges, r bins, gap
 *             probes, cell extremes, sector merging, rays), [13..15] running
 *             count of [0] after the theta-bin, r-range and r-bin phases
 *   points    [S][E][N_limb][N_deg][4] device float or NULL: image-limb points
 *             (r, theta, flags, FP32 error bound) after root validation; a
 *             slot whose root is not an image (flags without bit 0) holds the
 *             root's position (r, theta)
 * Same semantics and errors as icrs_magnification; the diagnostics add shared
 * memory atomics on the FP64 fallback paths and clock reads.
 */
int icrs_magnification_diag(const icrs_params* p, int S, const double* t, int E,
                            const icrs_grid* g, double* A, uint32_t* status,
                            double* sectors, int32_t* counters, float* points,
                            void* stream);

/*
 * Vector-Jacobian product of the finite-source magnification (binary lens)
 * with respect to the 8 parameters, in this order:
 *     (t0, tE, u0, alpha, s, q, rho, u1).
 * The derivative is the exact derivative, almost everywhere, of the discrete
 * method that icrs_magnification computes.  It runs through:
 *   - the rays: the lens map, the brightness, the cubic boundary crossings and
 *     f(delta) of Appendix A;
 *   - the sector bounds: these move with their extremal image-limb points,
 *     whose derivative is the implicit root derivative of Sec. 3.5, written
 *     for the lens equation.
 * The inclusion indicators and the binning decisions are piecewise constant,
 * so they contribute nothing.  The kernel recomputes every ray instead of
 * storing it: one fused forward and reverse pass per epoch.
 *   p, S, t, E, g  as icrs_magnification (g->n_lens 2 or 0; triple lenses
 *                  give ICRS_EUNSUPPORTED)
 *   gA      [S][E] device double: upstream dL/dA (required when grad != NULL)
 *   grad    [S][8] device double or NULL (out): sum_e gA[s][e] dA[s][e]/dp.
 *           It is zeroed on `stream`, then accumulated with atomics, so the
 *           order of the floating-point sums is not fixed.
 *   dA      [S][E][8] device double or NULL (out): per-epoch dA/dp
 *   A       [S][E] device double or NULL (out): the magnification
 *   status  [S][E] device uint32 or NULL (out), as icrs_magnification
 * At least one of grad and dA must be non-NULL.
 */
int icrs_magnification_vjp(const icrs_params* p, int S, const double* t, int E,
                           const icrs_grid* g, const double* gA, double* grad,
                           double* dA, double* A, uint32_t* status, void* stream);

/*
 * chi^2 of S light curves and its gradient with respect to the 8 parameters
 * of icrs_magnification_vjp.  The flux model is F = (A - 1) F_S + F_base with
 * F_S = F_base = 1, so F = A:
 *     chi2[s] = sum_e ((y[s][e] - A[s][e]) / sigma[s][e])^2.
 *   y, sigma  [S][E] device double: observed flux and its error (sigma > 0)
 *   chi2      [S] device double (out; zeroed on `stream`, then accumulated)
 *   grad      [S][8] device double (out; zeroed, then accumulated)
 *   A, status optional outputs, as in icrs_magnification_vjp
 */
int icrs_chi2_grad(const icrs_params* p, int S, const double* t, int E,
                   const icrs_grid* g, const double* y, const double* sigma,
                   double* chi2, double* grad, double* A, uint32_t* status,
                   void* stream);

/*
 * Linear-flux marginalised likelihood of S light curves (Appendix B) and its
 * gradient with respect to the 8 parameters of icrs_magnification_vjp.
 * Light curve s is F[s][e] = (A[s][e] - 1) F_S + F_base + noise, noise ~
 * N(0, sigma[s][e]^2), with the prior (F_S, F_base) ~ N(mu, diag(lambda)).
 * Marginalising the fluxes (Eq. NLL, evaluated with the Woodbury identity
 * printed after it):
 *     nll[s] = 1/2 (F - M mu)^T B^-1 (F - M mu) + 1/2 ln|B|,
 *     B = C + M Lambda M^T,  M = [A - 1, 1],  C = diag(sigma^2)
 * (no n/2 ln 2 pi term, as printed).  The gradient chains
 *     dnll/dA_e = c_e [(K^-1 m_e)_0 - (F_e - m_e . a) a_0],
 *     K = Lambda^-1 + M^T C^-1 M,  c_e = sigma_e^-2,  m_e = (A_e - 1, 1),
 * with a = mu + K^-1 M^T C^-1 (F - M mu) the posterior mean of (F_S,
 * F_base), through the per-epoch derivative dA/dp of the adjoint kernel.
 *   F, sigma  [S][E] device double: fluxes and their errors (sigma > 0)
 *   prior     [S][4] device double: mu_S, mu_base, lambda_S, lambda_base
 *             (prior means and variances, variances > 0)
 *   nll       [S] device double (out)
 *   grad      [S][8] device double or NULL (out).  NULL: the likelihood only
 *             (one forward launch); otherwise one derivative launch (binary
 *             lens; a triple lens returns ICRS_EUNSUPPORTED)
 *   fluxes    [S][2] device double or NULL (out): the posterior mean a
 *   A, status optional outputs, as icrs_magnification
 *   workspace device memory of icrs_marginal_nll_workspace_bytes(S, E)
 *             bytes, 8-byte aligned, caller-owned (per-epoch dA/dp and A)
 * The per-set sums run in a fixed order in FP64 (one block per set), so the
 * results do not depend on scheduling.  A non-positive sigma or prior
 * variance gives a NaN nll for that set.
 */
size_t icrs_marginal_nll_workspace_bytes(int S, int E);
int icrs_marginal_nll_grad(const icrs_params* p, int S, const double* t, int E,
                           const icrs_grid* g, const double* F, const double* sigma,
                           const double* prior, double* nll, double* grad, double* fluxes,
                           double* A, uint32_t* status, void* workspace,
                           size_t workspace_bytes, void* stream);

/*
 * ICRS on a list of items of an [S][E] problem: for i < n, item items[i] =
 * s * E + e runs set s at time t[s][e] and writes A[s][e] (and status[s][e]).
 * Other entries are left untouched, and an index outside [0, S * E) is
 * skipped.  This runs the epochs that the surrogate's gate routes back to
 * ICRS.  Consecutive items of one set reuse the previous item's roots as
 * starting values.  The image sets and sectors do not depend on those
 * starting values beyond their rounding, so the listed order changes the
 * result by a few parts per million at most (measured: 5e-6 relative on
 * 1.2 million routed epochs against the full launch) and changes the
 * speed.
 *   items  [n] device int32; the other arguments are as icrs_magnification
 */
int icrs_magnification_indexed(const icrs_params* p, int S, const double* t, int E,
                               const int32_t* items, int n, const icrs_grid* g,
                               double* A, uint32_t* status, void* stream);

/*
 * Learned surrogate of the finite-source correction.  It is not in the paper;
 * the gate below sends uncertain epochs back to ICRS.
 *   network   7 -> 128 -> 128 -> 128 -> 128 -> 2 with SiLU on the hidden
 *             layers.  Output 0 is mu, the prediction of y - b, where
 *             y = 1e4 log(A/A_ps) and b is features[7] below; output 1 is s,
 *             the log-variance of that prediction.
 *   numerics  BF16 weights, inputs and activations between layers; FP32
 *             accumulation in tensor memory (tcgen05.mma); FP32 master
 *             weights and Adam moments.  In the backward pass each layer's
 *             upstream gradient is rounded to BF16 before its contractions.
 *   theta     [ICRS_MLP_NPARAM] device float: W0 [128][7], b0 [128],
 *             W1 [128][128], b1, W2, b2, W3, b3, W4 [2][128], b4 [2],
 *             each weight row-major [out][in]
 *   pack      [ICRS_MLP_PACK_BYTES] device bytes (16-byte aligned): the BF16
 *             weights and their transposes in the tensor-core operand layout,
 *             written by icrs_mlp_pack or by a training step
 *   features  [n][8] device float (16-byte aligned): (w_c.x, w_c.y, log10 s,
 *             (log10 q + 3)/2, log10 rho + 3, 4 (u1 - 0.55),
 *             clamp(log10 min_j |det J(z_j)|, -6, 1), b), where z_j are the
 *             point-source images at the source centre and at the 32 limb
 *             points w_c + rho e^{i pi k / 16}.  The network reads the first 7.
 *             b = 1e4 log(1 + f_u (mean_k A_ps(limb k) / A_ps - 1)), with
 *             f_u = <r^2> / rho^2 the second moment of the source's
 *             brightness ((15 - 7 u1) / (10 (3 - u1)) for the linear law,
 *             1/2 on a uniform grid; the quadratic and power-series terms
 *             u2, a1..a4 enter by their moments), is the second-order
 *             finite-source estimate: the network predicts y - b
 */
#define ICRS_MLP_NPARAM 50818
#define ICRS_MLP_PACK_BYTES 208896

/* theta -> pack (BF16 operand tiles). */
int icrs_mlp_pack(const float* theta, void* pack, void* stream);

/*
 * Inference: out [n][2] device float = (mu, s) per row of features.  One
 * persistent tcgen05 kernel.  err: device int32 or NULL, set to 1 if a
 * tensor-core completion wait ran past its bound (the results are then
 * invalid).
 */
int icrs_mlp_infer(const void* pack, const float* theta, const float* features, int n,
                   float* out, int* err, void* stream);

/* Bytes of workspace a training step over n samples needs. */
size_t icrs_mlp_workspace_bytes(int n);

/*
 * One training step on n samples: the mean Gaussian NLL
 *     1/2 [(y - mu)^2 e^{-s} + s]
 * and its gradient, then Adam (beta 0.9 / 0.999, eps 1e-8, bias-corrected,
 * `step` counts from 1) if lr > 0, and the repack of `pack`.
 *   target     [n] device float: y = 1e4 log(A_ICRS / A_ps)
 *   grad       [ICRS_MLP_NPARAM] device float or NULL (out): the gradient
 *   loss       [1] device float or NULL (out)
 *   workspace  device, 256-byte aligned, >= icrs_mlp_workspace_bytes(n);
 *              caller-owned (the library allocates nothing)
 *   adam_m, adam_v  [ICRS_MLP_NPARAM] device float moments (used if lr > 0)
 * With lr = 0 the step computes the gradient only and leaves theta alone.
 */
int icrs_mlp_train_step(float* theta, float* adam_m, float* adam_v, void* pack, int step,
                        float lr, const float* features, const float* target, int n,
                        float* grad, float* loss, void* workspace, size_t workspace_bytes,
                        int* err, void* stream);

/*
 * icrs_mlp_train_step without a caller workspace, for callers that cannot
 * allocate device memory where they train.  The paper has no counterpart:
 * this is an operational variant of the surrogate's training step.
 * Scratch: a static device array inside the library, sized for
 * n <= ICRS_MLP_STATIC_MAX_N samples (larger n gives ICRS_EINVAL).  Its
 * address is looked up once per device.  No device memory is allocated and
 * nothing in the scratch needs clearing between calls.  There is one scratch
 * per device: calls that overlap in time on that device, from any stream or
 * thread, race on it and must be serialised by the caller.  The first call on
 * each device should come before any stream capture, because it looks up the
 * symbol address and sets the kernel's shared-memory attribute.  Arguments and
 * results are otherwise those of icrs_mlp_train_step.
 */
#define ICRS_MLP_STATIC_MAX_N 4096
int icrs_mlp_train_step_noalloc(float* theta, float* adam_m, float* adam_v, void* pack, int step,
                                float lr, const float* features, const float* target, int n,
                                float* grad, float* loss, int* err, void* stream);

/*
 * Surrogate features of every (set, epoch) of an [S][E] problem (binary lens,
 * g->n_lens = 2).  The point-source solve at the source centre is the same as
 * icrs_point_source.
 *   features  [S][E][8] device float (out)
 *   A_ps      [S][E] device double (out): point-source magnification
 *   status    [S][E] device uint32 or NULL (out): the point-source ICRS_ST_* bits
 *             of the centre and limb solves, plus ICRS_ST_LIMB when a limb
 *             point has a different image count from the centre, plus
 *             ICRS_ST_ROUGH when H > ICRS_ROUGH_MAX (or H is not finite), with
 *             H = (1/32) sum_{m=3..29} |sum_k (A_k - A_c) e^{-2 pi i m k / 32}| / A_c
 *             over the limb magnifications A_k at w_c + rho e^{2 pi i k / 32}:
 *             structure on the scale of the source (a caustic a few rho
 *             away) that the second-order estimate of feature 7 misses;
 *             plus ICRS_ST_SPOT when spot_c != 0 and spot_r > 0 (the
 *             estimate assumes a radially symmetric source) and, unless
 *             g->uniform, ICRS_ST_PROFILE when u2 or one of a1..a4 is nonzero
 *             (the network was given u1 only; the estimate itself uses the
 *             law's second moment and stays valid)
 */
int icrs_surrogate_features(const icrs_params* p, int S, const double* t, int E,
                            const icrs_grid* g, float* features, double* A_ps,
                            uint32_t* status, void* stream);

/*
 * Training target of the network for n epochs:
 *     target[i] = 1e4 log(A[i] / A_ps[i]) - features[i][7]
 * (FP64, rounded to float), from ICRS magnifications A and the feature
 * kernel's A_ps and second-order estimate b.
 *   A, A_ps [n] device double; features [n][8] device float; target [n] out
 */
int icrs_surrogate_target(const double* A, const double* A_ps, const float* features, int n,
                          float* target, void* stream);

/*
 * Mini-batch gather for training: out_features[i] = features[idx[i]] and
 * out_target[i] = target[idx[i]] for i < n.  The permutation idx (device
 * int32, entries in range) is drawn by the caller.  features and
 * out_features must be 16-byte aligned.
 */
int icrs_surrogate_batch(const float* features, const float* target, const int32_t* idx, int n,
                         float* out_features, float* out_target, void* stream);

/* Bytes of workspace icrs_surrogate_gate needs for n epochs. */
size_t icrs_surrogate_gate_workspace_bytes(int n);

/*
 * Error gate.  Epoch i is accepted when all of these hold:
 *   - its feature status is 0 (clean solves, the same image count across
 *     the disk, no ICRS_ST_ROUGH, no spot and no law beyond u1);
 *   - features[i][6] >= caustic_min;
 *   - exp(s_i / 2) <= sigma_max;
 *   - |mu_i| <= mu_max and |features[i][7]| <= b_max;
 *   - A_ps[i] <= A_max, or <= A_small when rho < rho_min (for small
 *     sources away from the far field, and for all sources at high
 *     magnification, ICRS itself still moves by ~1e-4 between grid
 *     refinements, so those epochs stay with ICRS).
 * For an accepted epoch, A[i] = A_ps[i] exp(1e-4 (features[i][7] + mu_i)).  Every other epoch is
 * listed, in increasing order, in routed_idx[0 .. *n_routed) (device outputs)
 * and its A[i] is left for icrs_magnification_indexed.
 *   pred [n][2], features [n][8], A_ps [n], st_ps [n]: as produced above
 *   workspace  device, >= icrs_surrogate_gate_workspace_bytes(n)
 */
int icrs_surrogate_gate(const float* pred, const float* features, const double* A_ps,
                        const uint32_t* st_ps, int n, float sigma_max, float mu_max,
                        float b_max, float caustic_min, double A_max, float rho_min, double A_small,
                        double* A, int32_t* routed_idx, int32_t* n_routed,
                        void* workspace, size_t workspace_bytes, void* stream);

/*
 * Non-learned epoch preselection: the control for the learned gate.  Sec.
 * 3.4 (iii) runs the extended-source computation only on a preselected set
 * of epochs near caustics.  Epoch e of light curve s (item q = s * E + e of
 * an [S][E] problem) is near a caustic unless all of these hold:
 *   - its feature status is 0 apart from ICRS_ST_PROFILE (the second-order
 *     estimate holds for every radial law);
 *   - features[q][6] >= caustic_min;
 *   - |features[q][7]| <= b_max (the second-order estimate b);
 *   - A_ps[q] <= A_max, or <= A_small when rho < rho_min.
 * Every epoch of the same light curve within n_ext epochs of a near-caustic
 * epoch is routed to ICRS as well (the caustic can fall between epochs).
 * The remaining epochs get a finite-source estimate without ray shooting:
 *   mode 0: A = A_ps (point source);
 *   mode 1: A = A_ps exp(1e-4 features[q][7]) (second-order estimate).
 * Routed items are listed in increasing order in routed_idx[0 .. *n_routed)
 * and their A is left for icrs_magnification_indexed.
 *   features [S*E][8], A_ps [S*E], st_ps [S*E]: from icrs_surrogate_features
 *   workspace  device, >= icrs_epoch_gate_workspace_bytes(S, E)
 * S * E must fit in an int32 (else ICRS_EUNSUPPORTED).
 */
size_t icrs_epoch_gate_workspace_bytes(int S, int E);
int icrs_epoch_gate(const float* features, const double* A_ps, const uint32_t* st_ps, int S, int E,
                    int n_ext, int mode, float b_max, float caustic_min, double A_max, float rho_min,
                    double A_small, double* A, int32_t* routed_idx, int32_t* n_routed,
                    void* workspace, size_t workspace_bytes, void* stream);

/* Message for a return code (static string). */
const char* icrs_strerror(int code);

/* Version of the library ABI (increments on incompatible changes). */
int icrs_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ICRS_H */
