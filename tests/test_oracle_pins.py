"""Pins of the FP64 oracle against closed forms, brute force, library routines
and invariants (no GPU).  Each test names the mathematical fact it checks.

A plausible mistake in the oracle fails at least one of these:
  * wrong lens placement / masses      -> point-source closed form, symmetry
  * dropped polynomial term / sign     -> numpy roots, Newton images, invariant
  * bad validation tolerance / frame   -> image counts, Newton images
  * wrong limb / sector coverage       -> Witt-Mao areas (incl. ring case), brute force
  * quadrature weights / normalisation -> Witt-Mao, LD superposition integral
  * derivative chain                   -> finite differences
"""
import numpy as np
import pytest

from paper_2510_02639_gb300 import inputs as I
from tests import closed_forms as CF

G = I.grid()


def far_single(u0=0.0, rho=1e-3, u1=0.5, **kw):
    # A binary whose companion is negligible (q = 1e-10) and far (s = 20):
    # the single-lens limit, with the primary at the origin to 5e-10.
    return I.binary(q=1e-10, s=20.0, u0=u0, alpha=0.0, t0=0.0, tE=1.0, rho=rho, u1=u1, **kw)


# ---------------------------------------------------------------- point source
@pytest.mark.parametrize("u", [0.01, 0.1, 0.5, 1.0, 3.0])
def test_point_source_single_lens_limit(oracle_mod, u):
    """(a) As q -> 0 the binary point-source magnification tends to
    (u^2 + 2) / (u sqrt(u^2 + 4))."""
    p = far_single()
    eps, a = oracle_mod.lens(p)
    A, n, _, st = oracle_mod.point_source(p, G, [a[0] + u])
    assert st[0] == 0 and n[0] == 3
    assert abs(A[0] / CF.single_lens_point(u) - 1) < 1e-7


def test_signed_invariant_binary(oracle_mod):
    """(c) For a binary lens and a source inside a caustic (five images) the
    signed magnifications sum to 1 (Witt & Mao 1995)."""
    rng = np.random.default_rng(7)
    checked = 0
    for q, s in [(0.1, 1.0), (1.0, 1.0), (0.5, 1.5), (1e-3, 1.0), (0.3, 0.7)]:
        p = I.binary(q=q, s=s)
        eps, a = oracle_mod.lens(p)
        ws = rng.uniform(-0.25, 0.25, 60) + 1j * rng.uniform(-0.25, 0.25, 60)
        A, n, z, st = oracle_mod.point_source(p, G, ws)
        for i in range(len(ws)):
            assert n[i] in (3, 5)
            if n[i] != 5:
                continue
            zz = z[i, :5]
            gam = np.array([np.sum(eps / (x - a) ** 2) for x in zz])
            signed = np.sum(1.0 / (1.0 - np.abs(gam) ** 2))
            assert abs(signed - 1.0) < 1e-9
            checked += 1
    assert checked >= 20


@pytest.mark.parametrize("r", [30.0, 100.0, 300.0])
def test_far_field(oracle_mod, r):
    """(e) Far from the lenses A -> 1.  The positive image gives 1 + 1/u^4 and
    the negative image beside each mass i (z ~ a_i - eps_i/conj(w)) gives
    eps_i^2/u^4, so A - 1 -> (1 + sum_i eps_i^2)/u^4 + O(u^-5) (2/u^4 for one
    lens)."""
    for q in (0.3, 1e-3):
        p = I.binary(q=q, s=1.0)
        eps, a = oracle_mod.lens(p)
        lead = (1.0 + np.sum(eps ** 2)) / r ** 4
        for ph in (0.3, 1.7, 4.0):
            w = r * np.exp(1j * ph)
            A, n, _, _ = oracle_mod.point_source(p, G, [w])
            assert n[0] == 3
            assert abs((A[0] - 1.0) / lead - 1.0) < 4.0 / r


# ---------------------------------------------------------------- polynomial
@pytest.mark.parametrize("n_lens", [2, 3])
def test_roots_match_numpy_companion(oracle_mod, n_lens):
    """EA roots equal the eigenvalues of the companion matrix (numpy.roots) of
    the oracle's own coefficients."""
    rng = np.random.default_rng(3)
    p = I.binary(q=2e-3, s=1.1) if n_lens == 2 else I.triple(q2=0.05, q3=0.02, s2=1.1, s3=0.9, psi=1.0)
    for _ in range(10):
        w = complex(rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3))
        b = oracle_mod.poly(p, w, 0.0)
        assert len(b) == (6 if n_lens == 2 else 11)
        z, ok = oracle_mod.roots(p, w)
        assert ok
        ref = np.roots(b[::-1])
        for zz in ref:
            assert np.min(np.abs(z - zz)) < 1e-8 * max(1.0, abs(zz))


@pytest.mark.parametrize("n_lens", [2, 3])
def test_newton_images_are_roots_and_validated(oracle_mod, n_lens):
    """Every solution of the lens equation found by plain 2-D Newton from many
    starts is a root of the polynomial and is kept by the oracle's validation;
    the oracle keeps no other root."""
    rng = np.random.default_rng(11)
    if n_lens == 2:
        p = I.binary(q=0.2, s=1.0)
    else:
        p = I.triple(q2=0.1, q3=0.05, s2=1.0, s3=0.9, psi=1.2)
    eps, a = oracle_mod.lens(p)
    for _ in range(6):
        w = complex(rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2))
        sols = CF.newton_images(eps, a, w, n_start=1500)
        A, n, z, st = oracle_mod.point_source(p, G, [w])
        got = z[0, : n[0]]
        assert len(sols) == n[0], (sols, got)
        for s_ in sols:
            assert np.min(np.abs(got - s_)) < 1e-9
        allroots, _ = oracle_mod.roots(p, w)
        b = oracle_mod.poly(p, w, 0.0)
        for s_ in sols:
            scale = np.sum(np.abs(b) * np.abs(s_) ** np.arange(len(b)))
            assert abs(np.polyval(b[::-1], s_)) < 1e-11 * scale


def test_small_mass_ratio_counts(oracle_mod):
    """Validation in the lightest-lens frame keeps exactly 3 or 5 images down to
    q = 1e-7 (the tiny image beside the planet is kept, spurious roots beside it
    are rejected)."""
    rng = np.random.default_rng(5)
    for q in (1e-5, 1e-6, 1e-7):
        for s in (0.6, 1.0, 1.8):
            p = I.binary(q=q, s=s)
            ws = rng.uniform(-0.3, 0.3, 40) + 1j * rng.uniform(-0.3, 0.3, 40)
            A, n, z, st = oracle_mod.point_source(p, G, ws)
            assert set(np.unique(n)) <= {3, 5}
            assert np.all(st == 0)


def test_triple_reduces_to_binary(oracle_mod):
    """A triple lens whose third mass is negligible gives the binary result
    (mass fractions eps2 = q2, eps1 = 1 - q2 <-> q = q2 / (1 - q2))."""
    q2 = 0.01
    tri = I.triple(q2=q2, q3=1e-10, s2=1.05, s3=4.0, psi=0.7, rho=1e-2, u0=0.05, alpha=0.4, tE=10.0, u1=0.6)
    bi = I.binary(q=q2 / (1 - q2), s=1.05, rho=1e-2, u0=0.05, alpha=0.4, tE=10.0, u1=0.6)
    t = np.linspace(-1.0, 1.0, 5)
    ws = oracle_mod.source_centre(bi, t)
    At, nt, _, _ = oracle_mod.point_source(tri, G, ws)
    Ab, nb, _, _ = oracle_mod.point_source(bi, G, ws)
    assert np.all(nt == nb + 1)  # plus the tiny image beside the far third mass
    np.testing.assert_allclose(At, Ab, rtol=1e-8)
    g = I.grid(n_r=48, n_theta=192)
    Aft, _ = oracle_mod.magnification(tri, t, g)
    Afb, _ = oracle_mod.magnification(bi, t, g)
    np.testing.assert_allclose(Aft, Afb, rtol=2e-6)


# ---------------------------------------------------------------- finite source
@pytest.mark.parametrize("u_over_rho,rho", [(0.3, 0.05), (2.0, 0.05), (10.0, 0.01), (1.5, 1e-3)])
def test_uniform_disk_witt_mao(oracle_mod, u_over_rho, rho):
    """(b) Uniform disk, single-lens limit: the ICRS quadrature (uniform rule)
    converges to the exact image area (Green's theorem; equivalent to the
    Witt-Mao elliptic-integral form).  u < rho is the ring case (gap filling
    across the ring's interior and the full-circle sector)."""
    u = u_over_rho * rho
    p = far_single(rho=rho, u1=0.0)
    g = I.grid(n_r=512, n_theta=2048, uniform=1, n_limb=1000)
    A, st = oracle_mod.magnification(p, [u], g)
    ref = CF.single_lens_uniform_disk(u, rho)
    # the radial midpoint sum converges as N_r^-1.5 where an image edge runs
    # along a row (square-root end of the covered length); 1e-4 at N_r = 512
    assert abs(A[0, 0] / ref - 1.0) < 1e-4, (A, ref)


@pytest.mark.parametrize("u_over_rho,rho,u1", [(3.0, 0.05, 0.5), (0.5, 0.05, 0.6), (2.0, 5e-3, 0.3)])
def test_limb_darkened_disk(oracle_mod, u_over_rho, rho, u1):
    """(iii) Linear limb darkening, single-lens limit: the LD per-point rule
    converges to the superposition-of-uniform-disks integral."""
    u = u_over_rho * rho
    p = far_single(rho=rho, u1=u1)
    g = I.grid(n_r=512, n_theta=2048, n_limb=1000)
    A, st = oracle_mod.magnification(p, [u], g)
    ref = CF.single_lens_ld_disk(u, rho, u1)
    assert abs(A[0, 0] / ref - 1.0) < 1e-4, (A, ref)


def test_quadratic_law_reduces_to_linear():
    """The quadratic superposition integral with u2 = 0 is the linear one."""
    for u, rho, u1 in ((0.15, 0.05, 0.5), (0.02, 0.05, 0.6)):
        assert CF.single_lens_quadratic_ld_disk(u, rho, u1, 0.0) == pytest.approx(
            CF.single_lens_ld_disk(u, rho, u1), rel=1e-12)


@pytest.mark.parametrize("u_over_rho,rho,u1,u2,split", [
    (3.0, 0.05, 0.4, 0.25, 0), (0.5, 0.05, 0.3, 0.3, 0), (2.0, 5e-3, 0.5, 0.2, 0),
    (3.0, 0.05, 0.4, 0.25, 1), (0.5, 0.05, 0.3, 0.3, 1), (2.0, 5e-3, 0.5, 0.2, 1)])
def test_quadratic_limb_darkened_disk(oracle_mod, u_over_rho, rho, u1, u2, split):
    """(iii) Quadratic limb darkening (u2 != 0), single-lens limit, with the
    literal per-point rule (f(delta) on the whole brightness) and the
    split-profile rule (the limb value with f_U, the rest with f): both
    converge to the superposition-of-uniform-disks integral, which pins the
    law, its normalisation I0 = 1/(pi (1 - u1/3 - u2/6)) and the limb value."""
    u = u_over_rho * rho
    p = dict(far_single(rho=rho, u1=u1), u2=u2)
    g = I.grid(n_r=512, n_theta=2048, n_limb=1000, ld_split=split)
    A, st = oracle_mod.magnification(p, [u], g)
    ref = CF.single_lens_quadratic_ld_disk(u, rho, u1, u2)
    assert abs(A[0, 0] / ref - 1.0) < 1e-4, (A, ref)


def test_power_series_law_reduces_to_quadratic():
    """The power-series superposition integral with a = 0 is the quadratic
    one (two different integration variables), and a pure a_2 (a_4) term is
    the linear (quadratic-in-mu) law written another way: 1 - a (1 - mu) with
    a_2 = u1; 1 - a_4 (1 - mu^2) = 1 - 2 a_4 (1 - mu) + a_4 (1 - mu)^2.  (To
    1e-6: the uniform-disk integrals under both are accurate to ~1e-7.)"""
    for u, rho in ((0.15, 0.05), (0.02, 0.05)):
        ref = CF.single_lens_quadratic_ld_disk(u, rho, 0.4, 0.25)
        assert CF.single_lens_profile_disk(u, rho, 0.4, 0.25, [0, 0, 0, 0]) == pytest.approx(ref, rel=1e-6)
        assert CF.single_lens_profile_disk(u, rho, 0.0, 0.0, [0, 0.5, 0, 0]) == pytest.approx(
            CF.single_lens_ld_disk(u, rho, 0.5), rel=1e-6)
        assert CF.single_lens_profile_disk(u, rho, 0.0, 0.0, [0, 0, 0, 0.3]) == pytest.approx(
            CF.single_lens_quadratic_ld_disk(u, rho, 0.6, -0.3), rel=1e-6)


@pytest.mark.parametrize("u_over_rho,rho,a", [
    (3.0, 0.05, (0.6, 0.0, 0.0, 0.0)), (0.5, 0.05, (0.3, 0.2, -0.1, 0.05)), (2.0, 5e-3, (0.0, 0.3, 0.2, 0.0)),
    (1.2, 0.05, (0.8, -0.4, 0.3, -0.1))])
def test_power_series_limb_darkened_disk(oracle_mod, u_over_rho, rho, a):
    """(iii) The power-series law in mu^(1/2) (the four-coefficient law, read
    as the paper's arbitrary radial profiles), with u1 = 0.2 on top,
    single-lens limit: the per-point rule converges to the
    superposition-of-uniform-disks integral in v = mu^(1/2), which pins the
    law, its normalisation and the limb value."""
    u = u_over_rho * rho
    p = dict(far_single(rho=rho, u1=0.2), a1=a[0], a2=a[1], a3=a[2], a4=a[3])
    g = I.grid(n_r=512, n_theta=2048, n_limb=1000)
    A, st = oracle_mod.magnification(p, [u], g)
    ref = CF.single_lens_profile_disk(u, rho, 0.2, 0.0, a)
    assert abs(A[0, 0] / ref - 1.0) < 1e-4, (A, ref)


@pytest.mark.parametrize("case", [
    dict(q=0.2, s=1.0, w=0.02 + 0.01j, uniform=1, u1=0.0),
    dict(q=0.05, s=1.3, w=0.3 - 0.05j, uniform=0, u1=0.5),
    dict(q=1.0, s=0.8, w=0.05 + 0.04j, uniform=0, u1=0.7),
])
def test_brute_force_binary(oracle_mod, case):
    """(d) Binary lens, rho = 0.05: the oracle agrees with Cartesian inverse-ray
    shooting (independent of the polar sectors) to the brute force's pixel error."""
    rho = 0.05
    w = case["w"]
    p = I.binary(q=case["q"], s=case["s"], rho=rho, u1=case["u1"], t0=0.0, tE=1.0, u0=w.imag, alpha=0.0)
    g = I.grid(n_r=200, n_theta=800, uniform=case["uniform"])
    A, st = oracle_mod.magnification(p, [w.real], g)
    eps, a = oracle_mod.lens(p)
    ref = CF.brute_force_magnification(eps, a, w, rho, u1=case["u1"], uniform=bool(case["uniform"]),
                                       refine=120)
    assert abs(A[0, 0] / ref - 1.0) < 2e-3, (A, ref)


@pytest.mark.parametrize("case", [
    dict(q2=0.2, q3=0.1, s2=1.0, s3=0.7, psi=1.0, w=0.02 + 0.03j, uniform=1, u1=0.0),
    dict(q2=0.1, q3=0.05, s2=0.9, s3=0.6, psi=2.2, w=-0.05 + 0.02j, uniform=0, u1=0.5),
    dict(q2=0.3, q3=0.2, s2=1.2, s3=0.5, psi=0.4, w=0.1 - 0.1j, uniform=0, u1=0.6),
])
def test_brute_force_triple(oracle_mod, case):
    """(d) Triple lens with third masses of 5-20 % (eight or six images, one
    case at A_ps ~ 135 next to a caustic, one with a ring-shaped image whose
    box holds the others), rho = 0.05: the oracle agrees with Cartesian
    inverse-ray shooting to the brute force's pixel error.  A wrong triple
    polynomial coefficient, a missed image or a sector that clips one would
    show at the percent level."""
    rho = 0.05
    w = case["w"]
    p = I.triple(q2=case["q2"], q3=case["q3"], s2=case["s2"], s3=case["s3"], psi=case["psi"], rho=rho,
                 u1=case["u1"], t0=0.0, tE=1.0, u0=w.imag, alpha=0.0)
    g = I.grid(n_r=200, n_theta=800, uniform=case["uniform"])
    A, st = oracle_mod.magnification(p, [w.real], g)
    assert st[0, 0] == 0
    eps, a = oracle_mod.lens(p)
    ref = CF.brute_force_magnification(eps, a, w, rho, u1=case["u1"], uniform=bool(case["uniform"]),
                                       refine=120)
    assert abs(A[0, 0] / ref - 1.0) < 5e-4, (A, ref)


@pytest.mark.parametrize("case", [(0.05, 1.3, 0.3 - 0.05j), (1.0, 0.8, 0.05 + 0.04j), (0.2, 1.0, 0.02 + 0.01j)])
def test_brute_force_power_series_binary(oracle_mod, case):
    """(d) Binary lens, rho = 0.05, the four-coefficient law in mu^(1/2)
    (u1 = 0, a = 0.6, 0.3, -0.2, 0.1): the oracle at 200 x 800 agrees with
    Cartesian inverse-ray shooting whose brightness is the law written out
    here, I0 [1 - sum_k a_k (1 - mu^(k/2))] with I0 = 1 / (pi (1 - sum_k a_k
    k/(k+4))), to 5e-4."""
    q, s, w = case
    a = (0.6, 0.3, -0.2, 0.1)
    I0 = 1.0 / (np.pi * (1.0 - sum(a[k - 1] * k / (k + 4.0) for k in range(1, 5))))

    def weight(wn):  # the law over the uniform brute force's 1/pi
        mu = np.sqrt(1.0 - np.minimum(np.abs(wn) ** 2, 1.0))
        return np.pi * I0 * (1.0 - sum(a[k - 1] * (1.0 - mu ** (k / 2.0)) for k in range(1, 5)))

    rho = 0.05
    p = I.binary(q=q, s=s, rho=rho, u1=0.0, t0=0.0, tE=1.0, u0=w.imag, alpha=0.0)
    p.update(a1=a[0], a2=a[1], a3=a[2], a4=a[3])
    A, st = oracle_mod.magnification(p, [w.real], I.grid(n_r=200, n_theta=800))
    eps, al = oracle_mod.lens(p)
    ref = CF.brute_force_magnification(eps, al, w, rho, uniform=True, refine=120, weight=weight)
    assert abs(A[0, 0] / ref - 1.0) < 5e-4, (A, ref)


def test_full_disk_spot_leaves_magnification(oracle_mod):
    """A spot covering the whole disk (centre 0, radius 1) scales every ray
    and the unlensed flux alike: the magnification is the unspotted one
    (which pins the spot flux's normalisation, F_spot = 1)."""
    p = I.binary(q=1e-3, s=1.0, rho=1e-2, u1=0.5, u0=0.005, alpha=0.5)
    t = np.linspace(-0.05, 0.05, 5)
    A0, _ = oracle_mod.magnification(p, t, G)
    A1, _ = oracle_mod.magnification(dict(p, spot_x=0.0, spot_y=0.0, spot_r=1.0, spot_c=0.6), t, G)
    np.testing.assert_allclose(A1, A0, rtol=1e-10)


@pytest.mark.parametrize("spot", [(0.3, -0.2, 0.4, 0.7), (-0.5, 0.1, 0.3, 0.5)])
def test_spot_brute_force(oracle_mod, spot):
    """A spotted, linearly limb-darkened source, single-lens limit and a
    binary: the oracle agrees with Cartesian inverse-ray shooting weighted by
    the spot, normalised by a brute-force sum of the spotted disk's flux on a
    fine grid (independent of the oracle's spot-flux quadrature), to the brute
    force's pixel error."""
    sx, sy, sr, sc = spot
    rho, u1 = 0.05, 0.5
    spot_d = dict(spot_x=sx, spot_y=sy, spot_r=sr, spot_c=sc)

    def weight(wn):
        return np.where(np.abs(wn - (sx + 1j * sy)) < sr, 1.0 - sc, 1.0)

    # unlensed flux of the spotted disk, relative to the unspotted one
    n = 4000
    xs = (np.arange(n) + 0.5) / n * 2.0 - 1.0
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    R2 = X * X + Y * Y
    ins = R2 < 1.0
    Ild = 1.0 - u1 * (1.0 - np.sqrt(np.where(ins, 1.0 - R2, 0.0)))
    flux = np.sum((Ild * weight(X + 1j * Y))[ins]) / np.sum(Ild[ins])
    for q, s_, w in ((1e-10, 20.0, 0.08 + 0.0j), (0.05, 1.3, 0.3 - 0.05j)):
        p = dict(I.binary(q=q, s=s_, rho=rho, u1=u1, t0=0.0, tE=1.0, u0=w.imag, alpha=0.0), **spot_d)
        g = I.grid(n_r=200, n_theta=800)
        A, st = oracle_mod.magnification(p, [w.real], g)
        eps, a = oracle_mod.lens(p)
        wc = oracle_mod.source_centre(p, [w.real])[0]
        ref = CF.brute_force_magnification(eps, a, wc, rho, u1=u1, uniform=False, refine=120,
                                           weight=weight) / flux
        assert abs(A[0, 0] / ref - 1.0) < 2e-3, (A, ref, q)


def test_mirror_symmetry(oracle_mod):
    """(vi) Both lenses lie on the real axis, so the map commutes with complex
    conjugation: (alpha, u0) -> (-alpha, -u0) conjugates every source position
    and leaves the magnification unchanged."""
    p = I.binary(q=1e-3, s=1.0, rho=1e-3, u1=0.5, u0=0.01, alpha=0.5)
    pm = dict(p, alpha=-0.5, u0=-0.01)
    t = np.linspace(-0.5, 0.5, 21)
    A, _ = oracle_mod.magnification(p, t, G)
    Am, _ = oracle_mod.magnification(pm, t, G)
    np.testing.assert_allclose(A, Am, rtol=1e-11)


def test_centred_ring_radial_rule(oracle_mod):
    """(v) Source centred on a single lens: the image is an annulus whose edges
    run along the rows, the angular rule is exact and the whole error is the
    radial midpoint sum of a step function, |error| <= 2 dr / (r_out - r_in)
    relative; A -> sqrt(1 + 4/rho^2) as N_r grows."""
    rho = 0.01
    p = far_single(rho=rho, u1=0.0)
    ref = np.sqrt(1.0 + 4.0 / rho ** 2)
    for nr in (64, 512):
        g = I.grid(n_r=nr, n_theta=256, uniform=1)
        A, st = oracle_mod.magnification(p, [0.0], g)
        boxes, _ = oracle_mod.sectors(p, 0.0, g)
        dr = (boxes[0, 1] - boxes[0, 0]) / nr
        assert boxes[0, 4] == 1.0  # full-circle sector
        assert abs(A[0, 0] / ref - 1.0) <= 2.0 * dr / rho


def test_sectors_cover_all_images(oracle_mod):
    """Every ray that lands inside the source (Cartesian brute force) lies in one
    of the oracle's sectors, and the sectors do not overlap."""
    p = I.binary(q=1e-3, s=1.0, rho=1e-3, u1=0.5, u0=0.01, alpha=0.5)
    eps, a = oracle_mod.lens(p)
    for t in (-0.3, -0.05, 0.0, 0.12):
        boxes, st = oracle_mod.sectors(p, t, G)
        wc = oracle_mod.source_centre(p, t)[0]
        # dense rays around the Einstein ring where the images are
        r = np.linspace(0.9, 1.1, 1201)
        th = np.linspace(-np.pi, np.pi, 6001, endpoint=False)
        R, TH = np.meshgrid(r, th, indexing="ij")
        z = R * np.exp(1j * TH)
        inside = np.abs(CF.lens_map(eps, a, z) - wc) < p["rho"]
        cov = np.zeros_like(inside)
        for (rlo, rhi, tlo, wd, per) in boxes:
            inr = (R >= rlo) & (R <= rhi)
            d = np.mod(TH - tlo, 2 * np.pi)
            inth = np.ones_like(inr) if per else d <= wd
            assert not np.any(cov & inr & inth & inside)
            cov |= inr & inth
        assert np.all(cov[inside])


def test_sectors_cover_images_next_to_an_interval_edge(oracle_mod):
    """The epochs of tests/golden/interval_edge_epochs.json, whose lowest image
    angle sits within 1e-7 rad above a theta-bin edge that starts an angular
    interval: every valid image-limb point lies inside one of the oracle's
    sectors (a sector built from a subset of its image's points would leave
    the image's far end outside)."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "interval_edge_epochs.json")
    gold = json.load(open(path))
    params, t = I.binary_batch(**gold["batch"])
    g = I.grid(**gold["grid"])
    for row in gold["epochs"]:
        p, tt = params[row["set"]], float(t[row["set"], row["epoch"]])
        boxes, _ = oracle_mod.sectors(p, tt, g)
        lp = oracle_mod.limb_points(p, tt, g)
        v = lp[..., 2] > 0
        R, TH = lp[..., 0][v], lp[..., 1][v]
        cov = np.zeros(R.shape, bool)
        for (rlo, rhi, tlo, wd, per) in boxes:
            d = np.mod(TH - tlo, 2 * np.pi)
            cov |= (R >= rlo) & (R <= rhi) & ((d <= wd) if not per else True)
        assert np.all(cov), (row["set"], row["epoch"], int((~cov).sum()))


def test_close_image_pairs_against_newton(oracle_mod):
    """At the epochs of tests/golden/near_critical_epochs.json, the limb
    point whose two closest images are nearest each other (just inside a
    fold caustic): the oracle's images are all the solutions of the lens
    equation that damped 2-D Newton from many starts finds (no polynomial
    involved), each within 1e-7."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "near_critical_epochs.json")
    gold = json.load(open(path))
    params, t = I.binary_batch(**gold["batch"])
    g = I.grid(**gold["grid"])
    K = int(g["n_limb"])
    for row in gold["epochs"]:
        p, tt = params[row["set"]], float(t[row["set"], row["epoch"]])
        lp = oracle_mod.limb_points(p, tt, g)
        best, kb = np.inf, -1
        for k in range(K):
            v = lp[k, :, 2] > 0
            if v.sum() < 2:
                continue
            z = lp[k, v, 0] * np.exp(1j * lp[k, v, 1])
            d = np.abs(z[:, None] - z[None, :]) + np.eye(len(z)) * 1e9
            if d.min() < best:
                best, kb = float(d.min()), k
        v = lp[kb, :, 2] > 0
        zo = lp[kb, v, 0] * np.exp(1j * lp[kb, v, 1])
        eps, a = oracle_mod.lens(p)
        wc = oracle_mod.source_centre(p, tt)[0]
        w = wc + p["rho"] * np.exp(2j * np.pi * kb / K)
        sols = CF.newton_images(eps, a, w, n_start=3000)
        assert len(sols) == len(zo), (row["set"], row["epoch"], kb, len(sols), len(zo))
        for z in zo:
            assert np.min(np.abs(sols - z)) < 1e-7


def test_forward_mode_matches_fd(oracle_mod):
    """(vii) The oracle's 8-direction forward-mode derivative equals central
    finite differences of its own primal.  The primal is piecewise smooth
    (inclusion flags jump, and the extremal limb point behind a sector bound
    can change), so a pair (epoch, parameter) is compared only where two step
    sizes give the same difference quotient; nearly all pairs qualify."""
    p = I.binary(q=0.05, s=1.2, rho=0.02, u1=0.5, u0=0.1, alpha=0.8, tE=20.0, t0=0.0)
    g = I.grid(n_r=48, n_theta=160, n_limb=200)
    t = np.array([-3.0, -1.0, 0.4, 1.3, 2.5, 6.0])
    A, dA, _ = oracle_mod.magnification_fwd(p, t, g)
    keys = ["t0", "tE", "u0", "alpha", "s", "q", "rho", "u1"]
    rel = {"tE", "s", "q", "rho"}
    compared = agreed = 0
    for i, k in enumerate(keys):
        fd = []
        for h0 in (1e-7, 2e-7):
            h = h0 * p[k] if k in rel else h0
            Ap, _ = oracle_mod.magnification(dict(p, **{k: p[k] + h}), t, g)
            Am, _ = oracle_mod.magnification(dict(p, **{k: p[k] - h}), t, g)
            fd.append((Ap[0] - Am[0]) / (2 * h))
        for e in range(len(t)):
            scale = max(1.0, abs(fd[0][e]))
            if abs(fd[0][e] - fd[1][e]) > 2e-5 * scale:
                continue
            compared += 1
            agreed += abs(dA[0, e, i] - fd[0][e]) <= 5e-5 * scale
    assert compared >= 40
    assert agreed == compared


def test_all_core_build_equals_the_serial_oracle(oracle_mod):
    """The OpenMP build that times the all-core CPU baseline runs the same
    source over independent epochs: bitwise the serial build's A and
    status, including a spotted and a power-series set."""
    params, t = I.binary_batch()
    ps = [params[5], dict(params[9], a1=0.3, a3=-0.1),
          dict(params[13], spot_x=0.2, spot_y=0.1, spot_r=0.3, spot_c=0.4)]
    tt = np.stack([t[5, 4990:4996], t[9, ::1700][:6], t[13, 5000:5006]])
    g = I.grid()
    A1, s1 = oracle_mod.magnification(ps, tt, g)
    A2, s2 = oracle_mod.magnification_all_cores(ps, tt, g)
    np.testing.assert_array_equal(A1, A2)
    np.testing.assert_array_equal(s1, s2)


def test_image_tolerance_convention_does_not_change_results(oracle_mod):
    """img_tol is a convention: true images have FP64 residuals ~1e-15 and the
    polynomial's spurious roots residuals ~1e-2 or more, so img_tol = 1e-3
    (the default) and 1e-5 classify every root alike and give the same
    magnifications and status on caustic-crossing epochs and on random
    epochs of the batch (q down to 1e-5)."""
    params, t = I.caustic_crossing_binary(n_epochs=40)
    bparams, bt = I.binary_batch()
    rng = np.random.default_rng(17)
    picks = [(int(rng.integers(64)), int(rng.integers(10000))) for _ in range(24)]
    cases = [(params[0], t[0, i]) for i in range(40)] + [(bparams[s], bt[s, e]) for s, e in picks]
    for p, tt in cases:
        A3, s3 = oracle_mod.magnification(p, [tt], I.grid(img_tol=1e-3))
        A5, s5 = oracle_mod.magnification(p, [tt], I.grid(img_tol=1e-5))
        assert A3[0, 0] == pytest.approx(A5[0, 0], rel=1e-12), (p, tt)
        assert s3[0, 0] == s5[0, 0]


def test_paper_gradient_rules_change_tangents_only(oracle_mod):
    """The paper's gradient rules (grad_rule = 1: sigmoid indicator
    derivative of steepness S, fixed f'(delta) = 2/3) leave the magnification
    bitwise unchanged; for a uniform source (f_U' = 1 already) with S -> 0 the
    sigmoid term vanishes linearly in S, so the derivative tends to the exact
    one; for limb darkening the fixed f' changes the boundary terms."""
    params, t = I.caustic_crossing_binary()
    ts = t[:, 200:260:10]
    gu = I.grid(uniform=1)
    A0, d0, _ = oracle_mod.magnification_fwd(params, ts, gu)
    for S in (1e-3, 2e-3):
        A1, d1, _ = oracle_mod.magnification_fwd(params, ts, dict(gu, grad_rule=1, s_fac=S))
        assert np.array_equal(A0, A1)
        diff = d1 - d0
        if S == 1e-3:
            ref = diff
        else:
            # linear in S: doubling S doubles the sigmoid term
            np.testing.assert_allclose(diff, 2.0 * ref, rtol=1e-6, atol=1e-12 * np.abs(d0).max())
            assert np.abs(diff).max() <= 1e-2 * np.abs(d0).max()
    gl = I.grid()
    A2, d2, _ = oracle_mod.magnification_fwd(params, ts, gl)
    A3, d3, _ = oracle_mod.magnification_fwd(params, ts, dict(gl, grad_rule=1, s_fac=1e-9))
    assert np.array_equal(A2, A3)
    assert np.abs(d3 - d2).max() > 1e-3 * np.abs(d2).max()   # the fixed f' matters
