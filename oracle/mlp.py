"""FP64 oracle of the learned surrogate (test infrastructure only; the product
never imports it).

The surrogate is not in the paper.  It is the gated MLP of the build's scope:
7 features -> 4 x 128 SiLU -> 2 outputs (mu, log-variance s), trained with the
Gaussian negative log-likelihood 1/2 [(y - mu)^2 e^{-s} + s] and Adam.

Precision convention, mirrored from the CUDA kernels:
  - weights and inputs are rounded to BF16 (round to nearest even);
  - every contraction accumulates exactly (here FP64; FP32 on the GPU);
  - the activations between layers are rounded to BF16;
  - in the backward pass, the upstream gradient dZ of each layer is rounded
    to BF16 before it enters its three contractions: dW = dZ^T X,
    db = sum dZ, dX = dZ W.
With bf16=False every rounding is skipped, which gives the plain FP64 network
that the finite-difference pins check.

Parameter vector theta (float32, 50,818 entries), row-major [out][in]:
  W0 [128][7], b0 [128], W1 [128][128], b1, W2, b2, W3, b3, W4 [2][128], b4 [2].
"""
from __future__ import annotations

import numpy as np

NIN, H, NOUT = 7, 128, 2
SHAPES = [("W0", (H, NIN)), ("b0", (H,)), ("W1", (H, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
          ("W3", (H, H)), ("b3", (H,)), ("W4", (NOUT, H)), ("b4", (NOUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16_round(x):
    """Round to the nearest BF16 value, ties to even (via float32: values are
    first rounded to float32, then the low 16 bits of the float32 pattern are
    rounded off).  Returns float64."""
    x32 = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = x32.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(x32)
    if np.any(nan):
        out = np.where(nan, np.nan, out)
    return out


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == N_PARAMS
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_prime(z):
    sg = 1.0 / (1.0 + np.exp(-z))
    return sg * (1.0 + z * (1.0 - sg))


def init_theta(seed=0):
    """He-style uniform initialisation; the last layer starts small."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shp in SHAPES:
        if name.startswith("b"):
            d[name] = np.zeros(shp)
        else:
            fan_in = shp[1]
            lim = np.sqrt(6.0 / fan_in) * (0.1 if name == "W4" else 1.0)
            d[name] = rng.uniform(-lim, lim, shp)
    return pack(d).astype(np.float32)


def forward(theta, X, bf16=True):
    """X [n, 7] -> Y [n, 2] and the cache for backward."""
    p = unpack(theta)
    rnd = bf16_round if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    xs = [rnd(X)]
    zs = []
    for l in range(4):
        z = xs[-1] @ rnd(p[f"W{l}"]).T + p[f"b{l}"]
        zs.append(z)
        xs.append(rnd(silu(z)))
    Y = xs[-1] @ rnd(p["W4"]).T + p["b4"]
    return Y, {"x": xs, "z": zs, "p": p, "bf16": bf16}


U_BF16 = 2.0 ** -8   # unit roundoff of BF16 round-to-nearest (8 significant bits)
U_FP32 = 2.0 ** -24


def reference_forward(theta, X):
    """The network with BF16-rounded weights and inputs and no other rounding
    (every contraction and activation exact in FP64): the reference the
    tensor-core kernels are compared with, element by element."""
    p = unpack(theta)
    xs = [bf16_round(X)]
    zs = []
    for l in range(4):
        zs.append(xs[-1] @ bf16_round(p[f"W{l}"]).T + p[f"b{l}"])
        xs.append(silu(zs[-1]))
    Y = xs[-1] @ bf16_round(p["W4"]).T + p["b4"]
    return Y, {"x": xs, "z": zs, "p": p, "bf16": False, "wr": True}


def inference_bound(theta, X):
    """Per-element first-order bound on |Y_kernel - Y_ref| for a kernel that,
    beyond the reference's rounding of weights and inputs, rounds each hidden
    activation X_l (l = 1..4) to BF16 (|r_l| <= 2^-8 |X_l| elementwise) and
    accumulates every contraction of K terms in FP32 (error <= K 2^-24 of
    the sum of the terms' magnitudes).  Linearised about the reference:
        delta Y_j = sum_l (dY_j/dX_l) . r_l + sum_l (dY_j/dZ_l) . a_l,
    so |delta Y_j| <= sum_l |dY_j/dX_l| . 2^-8 |X_l| + sum_l |dY_j/dZ_l| . |a_l|,
    with dY_j/dX_l from back-propagation through the reference network.
    Returns (Y_ref [n, 2], bound [n, 2])."""
    Y, c = reference_forward(theta, X)
    p, xs, zs = c["p"], c["x"], c["z"]
    W = [bf16_round(p[f"W{l}"]) for l in range(5)]
    b = [p[f"b{l}"] for l in range(5)]
    acc = []   # |a_l|: FP32 accumulation bound of each pre-activation (and of Y)
    for l in range(5):
        K = W[l].shape[1] + 1
        acc.append(K * U_FP32 * (np.abs(xs[l]) @ np.abs(W[l]).T + np.abs(b[l])))
    bound = np.zeros_like(Y)
    for j in range(Y.shape[1]):
        gX = np.tile(W[4][j], (X.shape[0], 1))            # dY_j / dX_4
        bj = acc[4][:, j] + U_BF16 * np.sum(np.abs(gX) * np.abs(xs[4]), axis=1)
        for l in range(3, -1, -1):
            gZ = gX * silu_prime(zs[l])                   # dY_j / dZ_l
            bj += np.sum(np.abs(gZ) * acc[l], axis=1)
            gX = gZ @ W[l]                                # dY_j / dX_l
            if l > 0:
                bj += U_BF16 * np.sum(np.abs(gX) * np.abs(xs[l]), axis=1)
        bound[:, j] = bj
    return Y, bound


def gradient_term_scale(theta, X, y):
    """Sum over the batch of the magnitudes of the terms of every gradient
    entry of the reference network: for W_l[j, i], sum_n |dZ_l[n, j] X_l[n, i]|;
    for b_l[j], sum_n |dZ_l[n, j]| (dZ_l = dL/dZ_l of the mean Gaussian NLL).
    Returns (gradient of the reference network, the scales), both flat in the
    theta layout."""
    Y, c = reference_forward(theta, X)
    L, dY = nll(Y, y)
    p, xs, zs = c["p"], c["x"], c["z"]
    W = [bf16_round(p[f"W{l}"]) for l in range(5)]
    g, sc = {}, {}
    dz = dY
    g["W4"], sc["W4"] = dz.T @ xs[4], np.abs(dz).T @ np.abs(xs[4])
    g["b4"], sc["b4"] = dz.sum(axis=0), np.abs(dz).sum(axis=0)
    dx = dz @ W[4]
    for l in range(3, -1, -1):
        dz = dx * silu_prime(zs[l])
        g[f"W{l}"], sc[f"W{l}"] = dz.T @ xs[l], np.abs(dz).T @ np.abs(xs[l])
        g[f"b{l}"], sc[f"b{l}"] = dz.sum(axis=0), np.abs(dz).sum(axis=0)
        if l > 0:
            dx = dz @ W[l]
    return pack(g), pack(sc), L


def nll(Y, y):
    """Mean Gaussian NLL over the batch and its gradient with respect to Y."""
    n = Y.shape[0]
    mu, s = Y[:, 0], Y[:, 1]
    r = y - mu
    e = np.exp(-s)
    L = 0.5 * np.mean(r * r * e + s)
    dY = np.stack([-r * e, 0.5 * (1.0 - r * r * e)], axis=1) / n
    return L, dY


def backward(cache, dY):
    """Gradient of the loss with respect to theta (float64 vector)."""
    p, xs, zs = cache["p"], cache["x"], cache["z"]
    rnd = bf16_round if cache["bf16"] else (lambda v: np.asarray(v, dtype=np.float64))
    g = {}
    dz = rnd(dY)
    g["W4"] = dz.T @ xs[4]
    g["b4"] = dz.sum(axis=0)
    dx = dz @ rnd(p["W4"])
    for l in range(3, -1, -1):
        dz = rnd(dx * silu_prime(zs[l]))
        g[f"W{l}"] = dz.T @ xs[l]
        g[f"b{l}"] = dz.sum(axis=0)
        if l > 0:
            dx = dz @ rnd(p[f"W{l}"])
    return pack(g)


def adam(theta, m, v, grad, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (bias-corrected); step counts from 1.  Returns new
    (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


ST_LIMB = 64  # the image count changes between the source centre and a limb point
ST_ROUGH = 128  # the limb magnification varies on the scale of the source (limb_roughness > ROUGH_MAX)
ST_SPOT = 1 << 16  # the source carries a spot: its brightness is not radially symmetric
ST_PROFILE = 1 << 17  # the law has terms beyond the linear one (u2, a1..a4), which no network input carries
ROUGH_MAX = 1e-3


def limb_roughness(A_c, A_limb):
    """H = (1/32) sum_{m=3..29} |sum_k (A_k - A_c) e^{-2 pi i m k / 32}| / A_c:
    the angular harmonics of order >= 3 (both signs) of the limb
    magnifications A_limb [n, 32] relative to the centre's A_c [n].  A
    magnification field that is smooth on the source's scale has harmonics
    that fall off like (rho / L)^m; a caustic a few rho away raises them."""
    d = A_limb - A_c[:, None]
    c = np.fft.fft(d, axis=1)
    return np.sum(np.abs(c[:, 3:30]), axis=1) / 32.0 / A_c


def profile_r2(p: dict) -> float:
    """<r^2> / rho^2 of the source's brightness over its disk, for the
    law the oracle integrates (Appendix A.2's linear law plus the quadratic
    and mu^(k/2) terms that stand for the abstract's arbitrary profiles):
    with mu = sqrt(1 - x), x = r^2 / rho^2, the law is a sum of powers
    c_p mu^p (c_0 = 1 - u1 - u2 - sum a_k, c_1 = u1 + 2 u2, c_2 = -u2, and
    a_k at p = k / 2), and over the disk (dA = pi rho^2 dx)
        int_0^1 mu^p dx = 2 / (p + 2),   int_0^1 mu^p x dx = 2 / (p + 2) - 2 / (p + 4),
    so <r^2> / rho^2 = sum c_p (2/(p+2) - 2/(p+4)) / sum c_p 2/(p+2).  The
    linear law gives (15 - 7 u) / (10 (3 - u))."""
    u1, u2 = p["u1"], p.get("u2", 0.0)
    a = [p.get("a%d" % k, 0.0) for k in range(1, 5)]
    terms = [(0.0, 1.0 - u1 - u2 - sum(a)), (1.0, u1 + 2.0 * u2), (2.0, -u2)]
    terms += [(k / 2.0, a[k - 1]) for k in range(1, 5)]
    m0 = sum(c * 2.0 / (q + 2.0) for q, c in terms)
    m1 = sum(c * (2.0 / (q + 2.0) - 2.0 / (q + 4.0)) for q, c in terms)
    return m1 / m0


def features(p: dict, t, grid: dict, return_roughness: bool = False):
    """Surrogate features of one parameter set at times t, from the oracle's
    point-source images at the source centre and at the 32 limb points
    w_c + rho e^{i pi k / 16}: returns (features [n, 8], A_ps [n], status [n]),
    and H of limb_roughness when return_roughness is set.
    Feature 6 is log10 of the smallest |det J| over all those images, with
    det J = 1 - |sum_i eps_i / (z - a_i)^2|^2 (Eq. detJ), clamped to [-6, 1];
    status gains ST_LIMB when a limb point's image count differs from the
    centre's, ST_ROUGH when H > ROUGH_MAX or H is not finite, ST_SPOT for a
    spotted source (spot_c != 0 and spot_r > 0, dark or bright) and, unless
    the grid is uniform, ST_PROFILE for a law with u2 or a1..a4 nonzero."""
    import oracle
    w = oracle.source_centre(p, t)
    A, nimg, z, st = oracle.point_source(p, grid, w)
    eps, a = oracle.lens(p)
    st = st.astype(np.uint32).copy()

    def min_det(zi):
        if len(zi) == 0:
            return 0.0
        gam = np.sum(eps[None, :] / (zi[:, None] - a[None, :]) ** 2, axis=1)
        return float(np.min(np.abs(1.0 - np.abs(gam) ** 2)))

    md = np.array([min_det(z[i, : nimg[i]]) for i in range(len(w))])
    Alimb = np.zeros(len(w))
    Ak = np.zeros((len(w), 32))
    for k in range(32):
        wl = w + p["rho"] * np.exp(1j * np.pi * k / 16.0)
        Al, nl, zl, sl = oracle.point_source(p, grid, wl)
        Alimb += Al / 32.0
        Ak[:, k] = Al
        for i in range(len(w)):
            md[i] = min(md[i], min_det(zl[i, : nl[i]]))
            if nl[i] != nimg[i] or sl[i]:
                st[i] |= np.uint32(ST_LIMB)
    # second-order estimate of the disk average: A + (<r^2>/4) lap A, with the
    # limb mean minus the centre = (rho^2/4) lap A and <r^2> the brightness's
    # second moment (profile_r2; 1/2 for the uniform disk of a uniform grid,
    # whose brightness carries no law)
    uniform = bool(grid.get("uniform", 0))
    fu = 0.5 if uniform else profile_r2(p)
    base = 1e4 * np.log1p(fu * (Alimb / A - 1.0))
    if p.get("spot_c", 0.0) != 0.0 and p.get("spot_r", 0.0) > 0.0:
        st |= np.uint32(ST_SPOT)
    if not uniform and (p.get("u2", 0.0) != 0.0 or any(p.get("a%d" % k, 0.0) != 0.0 for k in range(1, 5))):
        st |= np.uint32(ST_PROFILE)
    with np.errstate(divide="ignore", invalid="ignore"):
        rough = limb_roughness(A, Ak)
    st[~(rough <= ROUGH_MAX)] |= np.uint32(ST_ROUGH)
    out = np.zeros((len(w), 8))
    for i in range(len(w)):
        lg = np.log10(md[i]) if md[i] > 0 else -np.inf
        out[i] = [w[i].real, w[i].imag, np.log10(p["s"]), (np.log10(p["q"]) + 3.0) / 2.0,
                  np.log10(p["rho"]) + 3.0, 4.0 * (p["u1"] - 0.55), min(1.0, max(-6.0, lg)),
                  min(1e4, max(-1e4, base[i]))]
    if return_roughness:
        return out, A, st, rough
    return out, A, st
