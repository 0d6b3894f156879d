"""Independent closed forms and brute-force references used to pin the oracle.

Nothing here imports the oracle or the CUDA library.  Each function states the
mathematics it evaluates.
"""
from __future__ import annotations

import numpy as np


def single_lens_point(u):
    """Point-source, point-lens magnification A = (u^2 + 2) / (u sqrt(u^2 + 4))."""
    u = np.asarray(u, dtype=float)
    return (u * u + 2.0) / (u * np.sqrt(u * u + 4.0))


def single_lens_uniform_disk(u: float, rho: float, n: int = 20000) -> float:
    """Uniform disk magnified by a unit point mass at the origin, from the exact
    image areas (Green's theorem, area = 1/2 closed integral of x dy - y dx).
    The images of a limb point w are z_+- = (w/2)(1 +- sqrt(1 + 4/|w|^2)).
    For u > rho the two image boundaries are separate closed curves; for u < rho
    they are the outer and inner edges of a ring.  The trapezoid rule on the
    periodic limb parametrisation is spectrally accurate."""
    phi = 2.0 * np.pi * np.arange(n) / n
    w = u + rho * np.exp(1j * phi)
    root = np.sqrt(1.0 + 4.0 / np.abs(w) ** 2)
    zp = 0.5 * w * (1.0 + root)
    zm = 0.5 * w * (1.0 - root)

    def area(z):
        # spectral derivative of the periodic curve
        k = np.fft.fftfreq(n, d=1.0 / n)
        dzdphi = np.fft.ifft(1j * k * np.fft.fft(z))
        x, y = z.real, z.imag
        return 0.5 * np.sum(x * dzdphi.imag - y * dzdphi.real) * (2.0 * np.pi / n)

    ap, am = abs(area(zp)), abs(area(zm))
    if u > rho:
        return (ap + am) / (np.pi * rho * rho)
    return (ap - am) / (np.pi * rho * rho)


def single_lens_ld_disk(u: float, rho: float, u1: float, n_phi: int = 200, n_limb: int = 4000) -> float:
    """Linearly limb-darkened disk, I(r~) = I0 [1 - u1 (1 - sqrt(1 - r~^2))],
    I0 = 3 / (pi (3 - u1)), as a superposition of uniform disks:
      A_LD = I(1) pi A_U(u, rho) + I0 u1 int_0^{pi/2} sin(phi) pi sin^2(phi) A_U(u, rho sin phi) dphi,
    (integration by parts of int I dM with r = rho sin phi, which removes the
    square-root singularity of I' at the limb).  Gauss-Legendre in phi, split
    where the sub-disk boundary passes the lens (rho sin phi = u)."""
    I0 = 3.0 / (np.pi * (3.0 - u1))
    val = I0 * (1.0 - u1) * np.pi * single_lens_uniform_disk(u, rho, n_limb)
    edges = [0.0, np.pi / 2]
    if u < rho:
        edges = [0.0, np.arcsin(u / rho), np.pi / 2]
    x, wts = np.polynomial.legendre.leggauss(n_phi)
    tot = 0.0
    for a, b in zip(edges[:-1], edges[1:]):
        ph = 0.5 * (b - a) * x + 0.5 * (b + a)
        ww = 0.5 * (b - a) * wts
        for p, wgt in zip(ph, ww):
            r = rho * np.sin(p)
            if r <= 0:
                continue
            tot += wgt * np.sin(p) * np.pi * np.sin(p) ** 2 * single_lens_uniform_disk(u, r, n_limb)
    return val + I0 * u1 * tot


def single_lens_quadratic_ld_disk(u: float, rho: float, u1: float, u2: float, n_phi: int = 200,
                                  n_limb: int = 4000) -> float:
    """Quadratically limb-darkened disk, I = I0 [1 - u1 (1 - mu) - u2 (1 - mu)^2],
    mu = sqrt(1 - r~^2), I0 = 1 / (pi (1 - u1/3 - u2/6)), by the same
    superposition of uniform disks (r~ = sin phi, mu = cos phi, dI/dmu =
    I0 [u1 + 2 u2 (1 - mu)]):
      A = I(1) pi A_U(u, rho) + int_0^{pi/2} I0 [u1 + 2 u2 (1 - cos phi)] sin(phi) pi sin^2(phi)
                                 A_U(u, rho sin phi) dphi."""
    I0 = 1.0 / (np.pi * (1.0 - u1 / 3.0 - u2 / 6.0))
    val = I0 * (1.0 - u1 - u2) * np.pi * single_lens_uniform_disk(u, rho, n_limb)
    edges = [0.0, np.pi / 2]
    if u < rho:
        edges = [0.0, np.arcsin(u / rho), np.pi / 2]
    x, wts = np.polynomial.legendre.leggauss(n_phi)
    tot = 0.0
    for a, b in zip(edges[:-1], edges[1:]):
        ph = 0.5 * (b - a) * x + 0.5 * (b + a)
        ww = 0.5 * (b - a) * wts
        for p, wgt in zip(ph, ww):
            r = rho * np.sin(p)
            if r <= 0:
                continue
            dIdmu = I0 * (u1 + 2.0 * u2 * (1.0 - np.cos(p)))
            tot += wgt * dIdmu * np.sin(p) * np.pi * np.sin(p) ** 2 * single_lens_uniform_disk(u, r, n_limb)
    return val + tot


def single_lens_profile_disk(u: float, rho: float, u1: float, u2: float, a, n_v: int = 200,
                             n_limb: int = 4000) -> float:
    """Disk with the power-series law I = I0 [1 - u1 (1 - mu) - u2 (1 - mu)^2 -
    sum_k a_k (1 - mu^(k/2))], mu = sqrt(1 - r~^2), normalised to unit flux
    (I0 = 1 / (pi (1 - u1/3 - u2/6 - sum_k a_k k/(k+4))), since
    int_0^1 (1 - mu^(k/2)) 2 r~ dr~ = k/(k+4)), as a superposition of uniform
    disks over mu:
      A = I(mu=0) pi A_U(u, rho) + int_0^1 dI/dmu pi (1 - mu^2) A_U(u, rho sqrt(1 - mu^2)) dmu,
    integrated in v = sqrt(mu), where dI/dmu dmu/dv = I0 [2 u1 v + 4 u2 v (1 - v^2)
    + sum_k k a_k v^(k-1)] is smooth (the mu^(1/2) term's dI/dmu is not).
    Gauss-Legendre in v, split where the sub-disk boundary passes the lens."""
    a = list(a) + [0.0] * (4 - len(a))
    sa = sum(a[k - 1] * k / (k + 4.0) for k in range(1, 5))
    I0 = 1.0 / (np.pi * (1.0 - u1 / 3.0 - u2 / 6.0 - sa))
    val = I0 * (1.0 - u1 - u2 - sum(a)) * np.pi * single_lens_uniform_disk(u, rho, n_limb)
    edges = [0.0, 1.0]
    if u < rho:
        mu_c = np.sqrt(1.0 - (u / rho) ** 2)
        edges = [0.0, np.sqrt(mu_c), 1.0]
    x, wts = np.polynomial.legendre.leggauss(n_v)
    tot = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        vs = 0.5 * (hi - lo) * x + 0.5 * (hi + lo)
        ww = 0.5 * (hi - lo) * wts
        for v, wgt in zip(vs, ww):
            mu = v * v
            r = rho * np.sqrt(max(1.0 - mu * mu, 0.0))
            if r <= 0:
                continue
            dI = I0 * (2.0 * u1 * v + 4.0 * u2 * v * (1.0 - mu) + sum(k * a[k - 1] * v ** (k - 1) for k in range(1, 5)))
            tot += wgt * dI * np.pi * (1.0 - mu * mu) * single_lens_uniform_disk(u, r, n_limb)
    return val + tot


def lens_map(eps, a, z):
    """w = z - sum_i eps_i / conj(z - a_i)."""
    z = np.asarray(z, dtype=complex)
    w = z.copy()
    for e, ai in zip(eps, a):
        w = w - e / np.conj(z - ai)
    return w


def newton_images(eps, a, w, n_start: int = 4000, seed: int = 0, box: float = 3.0):
    """All solutions of the lens equation near the lenses by damped 2-D Newton
    iteration from many random starts (independent of any polynomial)."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(-box, box, n_start) + 1j * rng.uniform(-box, box, n_start)
    # also start near every lens
    near = np.concatenate([ai + 1e-3 * np.exp(2j * np.pi * np.arange(64) / 64) for ai in a])
    z = np.concatenate([z, near])
    for _ in range(200):
        g = np.zeros_like(z)
        F = lens_map(eps, a, z) - w
        for e, ai in zip(eps, a):
            g = g + e / (z - ai) ** 2
        # J dz = -F with df = dz + conj(g) conj(dz)
        det = 1.0 - np.abs(g) ** 2
        dz = (np.conj(g) * np.conj(F) - F) / det
        step = np.minimum(1.0, 0.5 / np.maximum(np.abs(dz), 1e-300))
        z = z + dz * step
    F = np.abs(lens_map(eps, a, z) - w)
    ok = np.isfinite(F) & (F < 1e-12)
    sols = []
    for zz in z[ok]:
        if all(abs(zz - s) > 1e-9 * max(1, abs(s)) for s in sols):
            sols.append(zz)
    return np.array(sols)


def brute_force_magnification(eps, a, wc, rho, u1=0.0, uniform=True, h_coarse=4e-3,
                              box=2.6, refine=200, pad=0.5, weight=None):
    """Inverse-ray shooting on a Cartesian grid (independent of the polar
    sectors): a coarse pass over [-box, box]^2 finds the pixels whose rays land
    within (1 + pad) rho of the source centre; each connected bounding box is
    then sampled at pixel size rho / refine, skipping the points that an
    earlier box already holds (the box of a ring-shaped image can contain
    the boxes of other images).  Surface brightness: uniform (1/pi)
    or linear limb darkening, times weight((w - w_c) / rho) if given (not
    renormalised); A = sum I h^2 / rho^2."""
    xs = np.arange(-box, box, h_coarse) + 0.5 * h_coarse
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    Z = X + 1j * Y
    d = np.abs(lens_map(eps, a, Z) - wc)
    hit = d < (1.0 + pad) * rho + 3 * h_coarse
    # label boxes by a simple flood fill over hit pixels
    from scipy import ndimage
    lab, n = ndimage.label(hit)
    total = 0.0
    h = rho / refine
    I0 = 3.0 / (np.pi * (3.0 - u1))
    done = []  # boxes already sampled: (x0, x1, y0, y1)
    for obj in ndimage.find_objects(lab):
        xi, yi = obj
        x0, x1 = xs[xi.start] - 2 * h_coarse, xs[xi.stop - 1] + 2 * h_coarse
        y0, y1 = xs[yi.start] - 2 * h_coarse, xs[yi.stop - 1] + 2 * h_coarse
        fx = np.arange(x0, x1, h) + 0.5 * h
        fy = np.arange(y0, y1, h) + 0.5 * h
        for k in range(0, len(fx), 256):
            FX, FY = np.meshgrid(fx[k:k + 256], fy, indexing="ij")
            wn = (lens_map(eps, a, FX + 1j * FY) - wc) / rho
            dd = np.abs(wn)
            inside = dd < 1.0
            for bx0, bx1, by0, by1 in done:
                inside &= ~((FX >= bx0) & (FX < bx1) & (FY >= by0) & (FY < by1))
            if uniform:
                I = np.full(dd.shape, 1.0 / np.pi)
            else:
                rt2 = np.where(inside, dd * dd, 0.0)
                I = I0 * (1.0 - u1 * (1.0 - np.sqrt(1.0 - rt2)))
            if weight is not None:
                I = I * weight(wn)
            total += np.sum(I[inside])
        done.append((fx[0] - 0.5 * h, fx[-1] + 0.5 * h, fy[0] - 0.5 * h, fy[-1] + 0.5 * h))
    return total * h * h / (rho * rho)
