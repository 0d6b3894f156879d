"""Pins of the surrogate's FP64 oracle (oracle/mlp.py) against things other
than itself: finite differences of the loss, torch's BF16 conversion, the
closed-form first Adam step and the SiLU derivative."""
import numpy as np
import pytest

from oracle import mlp as M


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.uniform(-6, 6, 5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 3.0e38, -2.5e-30]])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.bf16_round(x), want)


def test_bf16_ties_to_even():
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 (even: 1); 1 + 3*2^-8
    # halfway between 1 + 2^-7 and 1 + 2^-6 (even: 1 + 2^-6)
    assert M.bf16_round(1.0 + 2.0 ** -8) == 1.0
    assert M.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6


def test_silu_prime_finite_difference():
    z = np.linspace(-8, 8, 101)
    h = 1e-6
    fd = (M.silu(z + h) - M.silu(z - h)) / (2 * h)
    np.testing.assert_allclose(M.silu_prime(z), fd, rtol=1e-8, atol=1e-10)


def test_parameter_count():
    assert M.N_PARAMS == 7 * 128 + 128 + 3 * (128 * 128 + 128) + 2 * 128 + 2 == 50818


def test_backward_matches_finite_differences():
    """FP64 network without rounding: the analytic gradient of the mean NLL
    against central differences on randomly chosen parameters of every
    layer."""
    rng = np.random.default_rng(2)
    theta = M.init_theta(3).astype(np.float64)
    theta += 0.05 * rng.standard_normal(theta.size)
    X = rng.standard_normal((9, 7))
    y = rng.standard_normal(9)
    Y, cache = M.forward(theta, X, bf16=False)
    L, dY = M.nll(Y, y)
    g = M.backward(cache, dY)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in M.SHAPES])
    idx = np.concatenate([rng.integers(offs[i], offs[i + 1], 6) for i in range(len(M.SHAPES))])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h; tm[i] -= h
        fd = (M.nll(M.forward(tp, X, bf16=False)[0], y)[0] - M.nll(M.forward(tm, X, bf16=False)[0], y)[0]) / (2 * h)
        assert abs(g[i] - fd) <= 1e-7 * max(1.0, abs(fd)), (i, g[i], fd)


def test_nll_gradient_closed_form():
    """At s = 0 the NLL is (y - mu)^2 / 2 + const: d/dmu = mu - y, d/ds =
    (1 - (y - mu)^2) / 2 (per sample, divided by n)."""
    Y = np.array([[0.3, 0.0], [-1.0, 0.0]])
    y = np.array([1.0, -0.5])
    L, dY = M.nll(Y, y)
    assert abs(L - 0.5 * np.mean((y - Y[:, 0]) ** 2)) < 1e-15
    np.testing.assert_allclose(dY[:, 0], (Y[:, 0] - y) / 2)
    np.testing.assert_allclose(dY[:, 1], (1 - (y - Y[:, 0]) ** 2) / 4)


def test_adam_first_step_is_signed_lr():
    """Step 1: m_hat = g, v_hat = g^2, so the update is lr g / (|g| + eps)."""
    rng = np.random.default_rng(4)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    t2, m, v = M.adam(th, np.zeros(50), np.zeros(50), g, 1, 1e-3)
    np.testing.assert_allclose(t2, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_rounded_forward_is_close_to_exact():
    """BF16 rounding changes outputs only at the BF16 precision level."""
    rng = np.random.default_rng(5)
    theta = M.init_theta(6)
    X = rng.uniform(-1, 1, (64, 7))
    Yr, _ = M.forward(theta, X, bf16=True)
    Ye, _ = M.forward(theta, X, bf16=False)
    assert np.max(np.abs(Yr - Ye)) < 0.05 * np.max(np.abs(Ye)) + 1e-3


def test_ld_second_moment_closed_form():
    """<r^2>/rho^2 of the linear law I = 1 - u + u sqrt(1 - r^2) on the unit
    disk, by quadrature, against the closed form (15 - 7u) / (10 (3 - u))
    used by the surrogate's second-order estimate."""
    from scipy.integrate import quad
    for u in (0.0, 0.3, 0.55, 0.8):
        I = lambda r: 1.0 - u + u * np.sqrt(max(0.0, 1.0 - r * r))
        num = quad(lambda r: I(r) * r ** 3, 0, 1, epsabs=1e-14)[0]
        den = quad(lambda r: I(r) * r, 0, 1, epsabs=1e-14)[0]
        assert abs(num / den - (15 - 7 * u) / (10 * (3 - u))) < 1e-10


PROFILE_SETS = [  # (u1, u2, (a1, a2, a3, a4))
    (0.0, 0.0, (0.0, 0.0, 0.0, 0.0)),
    (0.4, 0.25, (0.0, 0.0, 0.0, 0.0)),
    (0.0, 0.0, (0.6, 0.3, -0.2, 0.1)),
    (0.3, 0.1, (0.2, 0.0, 0.15, 0.0)),
]


def test_profile_second_moment_quadrature():
    """<r^2>/rho^2 of profile_r2 against quadrature of the law written out,
    I = 1 - u1 (1 - mu) - u2 (1 - mu)^2 - sum_k a_k (1 - mu^(k/2)) with
    mu = sqrt(1 - r^2) (the normalisation cancels), and the linear law's
    closed form.  A dropped term, a wrong power or a sign error in any
    coefficient moves the ratio by far more than the tolerance."""
    from scipy.integrate import quad
    for u1, u2, a in PROFILE_SETS:
        def I(r):
            mu = np.sqrt(max(0.0, 1.0 - r * r))
            return (1.0 - u1 * (1.0 - mu) - u2 * (1.0 - mu) ** 2
                    - sum(a[k - 1] * (1.0 - mu ** (k / 2.0)) for k in range(1, 5)))
        num = quad(lambda r: I(r) * r ** 3, 0, 1, epsabs=1e-14, limit=200)[0]
        den = quad(lambda r: I(r) * r, 0, 1, epsabs=1e-14, limit=200)[0]
        p = {"u1": u1, "u2": u2, **{"a%d" % k: a[k - 1] for k in range(1, 5)}}
        assert abs(M.profile_r2(p) - num / den) < 1e-9, (u1, u2, a)
    for u in (0.0, 0.55):
        assert abs(M.profile_r2({"u1": u}) - (15 - 7 * u) / (10 * (3 - u))) < 1e-14
    assert abs(M.profile_r2({"u1": 0.0}) - 0.5) < 1e-15  # uniform disk: <r^2> = rho^2 / 2


def test_second_order_estimate_single_lens_profiles(oracle_mod):
    """Far single lens, power-series and quadratic laws: the second-order
    estimate with the law's own second moment reproduces the closed-form
    disk magnification of that law to O((rho/u)^4), and the feature status
    carries ST_PROFILE (no network input holds u2 or a1..a4) but no other bit."""
    from tests import closed_forms as CF
    from paper_2510_02639_gb300 import inputs as I
    rho, u_over_rho = 0.01, 10.0
    u = u_over_rho * rho
    for u1, u2, a in PROFILE_SETS[1:]:
        p = I.binary(q=1e-9, s=50.0, rho=rho, u1=u1, u0=u, t0=0.0, tE=1.0, alpha=0.0)
        p.update(u2=u2, **{"a%d" % k: a[k - 1] for k in range(1, 5)})
        f, Aps, st = M.features(p, [0.0], I.grid())
        exact = CF.single_lens_profile_disk(u, rho, u1, u2, a, n_v=64, n_limb=2000)
        est = Aps[0] * np.exp(f[0, 7] * 1e-4)
        assert abs(est / exact - 1.0) < 3.0 * (rho / u) ** 4, (u1, u2, a, est, exact)
        assert abs(Aps[0] / exact - 1.0) > 10 * abs(est / exact - 1.0)
        assert int(st[0]) == M.ST_PROFILE


def test_feature_status_spot(oracle_mod):
    """A spotted source sets ST_SPOT (the estimate assumes a radially
    symmetric source), dark or bright and on a uniform grid too; a zero
    contrast or a zero radius is no spot.  A uniform grid ignores the law's
    terms beyond u1, so it sets no ST_PROFILE."""
    from paper_2510_02639_gb300 import inputs as I
    base = I.binary(q=1e-9, s=50.0, rho=0.01, u1=0.5, u0=0.1, t0=0.0, tE=1.0, alpha=0.0)
    for sp, want in (((0.3, 0.1, 0.4, 0.5), M.ST_SPOT), ((0.3, 0.1, 0.4, -0.5), M.ST_SPOT),
                     ((0.3, 0.1, 0.4, 0.0), 0), ((0.3, 0.1, 0.0, 0.5), 0)):
        p = dict(base, spot_x=sp[0], spot_y=sp[1], spot_r=sp[2], spot_c=sp[3])
        for uniform in (0, 1):
            _, _, st = M.features(dict(p, u2=0.2), [0.0], dict(I.grid(), uniform=uniform))
            assert int(st[0]) == want | (0 if uniform else M.ST_PROFILE), (sp, uniform, int(st[0]))


def test_second_order_estimate_single_lens(oracle_mod):
    """Far single lens (q = 1e-9, s = 50): the second-order finite-source
    estimate b from the 32 limb point-source magnifications reproduces the
    closed-form limb-darkened disk magnification to O((rho/u)^4)."""
    from tests import closed_forms as CF
    from paper_2510_02639_gb300 import inputs as I
    rho, u1 = 0.01, 0.6
    for u_over_rho in (8.0, 20.0):
        u = u_over_rho * rho
        p = I.binary(q=1e-9, s=50.0, rho=rho, u1=u1, u0=u, t0=0.0, tE=1.0, alpha=0.0)
        # the lens of mass 1/(1+q) sits at -q s/(1+q) ~ 0; the source centre at (0, u)
        f, Aps, st = M.features(p, [0.0], I.grid())
        exact = CF.single_lens_ld_disk(u, rho, u1)
        est = Aps[0] * np.exp(f[0, 7] * 1e-4)
        assert abs(est / exact - 1.0) < 3.0 * (rho / u) ** 4, (u_over_rho, est, exact, Aps[0])
        assert abs(Aps[0] / exact - 1.0) > 10 * abs(est / exact - 1.0)


def test_limb_roughness_single_lens_closed_form(oracle_mod):
    """Single lens (q = 1e-9, s = 50; the source centre at (0, u)): H of the
    features equals the angular harmonics of order >= 3 of the closed-form
    point-lens magnification A(x) = (x^2 + 2) / (x sqrt(x^2 + 4)) around the
    limb, projected on a fine grid of 4096 angles: orders +-3..+-15, and
    C_16 + C_-16 for the Nyquist bin.  Bin m of the 32-point transform holds
    sum_j C_{m + 32 j}, so the two differ by at most sum_{|n| >= 17} |C_n| / A_c
    (aliasing), plus 27 times the largest deviation of the oracle's
    point-source magnification from the closed form at the 32 limb points
    (each bin averages those deviations).  ST_ROUGH is set exactly where
    H > 1e-3."""
    from paper_2510_02639_gb300 import inputs as I
    rho, q, s = 0.01, 1e-9, 50.0
    a1 = -q * s / (1.0 + q)
    eps1 = 1.0 / (1.0 + q)

    def A_pl(z):
        x = np.abs(z - a1) / np.sqrt(eps1)
        return (x * x + 2.0) / (x * np.sqrt(x * x + 4.0))

    phi = np.linspace(0.0, 2.0 * np.pi, 4096, endpoint=False)
    seen = set()
    for u_over_rho in (2.5, 5.0, 12.0, 40.0):
        u = u_over_rho * rho
        p = I.binary(q=q, s=s, rho=rho, u1=0.5, u0=u, t0=0.0, tE=1.0, alpha=0.0)
        f, Aps, st, H = M.features(p, [0.0], I.grid(), return_roughness=True)
        wc = 1j * u
        Ak = A_pl(wc + rho * np.exp(1j * phi))
        C = {m: np.mean(Ak * np.exp(-1j * m * phi)) for m in range(-127, 128)}
        H_cf = (sum(abs(C[m]) + abs(C[-m]) for m in range(3, 16)) + abs(C[16] + C[-16])) / A_pl(wc)
        alias = sum(abs(C[m]) for m in C if abs(m) >= 17) / A_pl(wc)
        zk = wc + rho * np.exp(1j * np.pi * np.arange(32) / 16.0)
        dev = np.max(np.abs(oracle_mod.point_source(p, I.grid(), zk)[0] - A_pl(zk))) / A_pl(wc)
        assert dev < 1e-7  # the companion's constant deflection shifts the source by ~q / s
        assert abs(H[0] - H_cf) <= alias + 27.0 * dev + 1e-12, (u_over_rho, H[0], H_cf, alias, dev)
        rough = bool(st[0] & M.ST_ROUGH)
        assert rough == (H_cf > M.ROUGH_MAX), (u_over_rho, H_cf)
        seen.add(rough)
    assert seen == {True, False}


def test_inference_bound_covers_random_activation_roundings():
    """The first-order bound of inference_bound holds for a network whose
    hidden activations are perturbed by random relative errors of at most
    2^-8 (the BF16 rounding it models): a dropped layer or a wrong sign in
    the back-propagated sensitivities would let a perturbation escape."""
    rng = np.random.default_rng(3)
    th = M.init_theta(4).astype(np.float64) + 0.02 * rng.standard_normal(M.N_PARAMS)
    X = rng.uniform(-1, 1, (400, 7))
    Yr, bound = M.inference_bound(th, X)
    p = M.unpack(th)
    worst = 0.0
    for trial in range(20):
        x = M.bf16_round(X)
        for l in range(4):
            z = x @ M.bf16_round(p[f"W{l}"]).T + p[f"b{l}"]
            x = M.silu(z)
            x = x * (1.0 + M.U_BF16 * rng.choice([-1.0, 1.0], x.shape) * rng.uniform(0.5, 1.0, x.shape))
        Y = x @ M.bf16_round(p["W4"]).T + p["b4"]
        worst = max(worst, float(np.max(np.abs(Y - Yr) / bound)))
    assert worst <= 1.05, worst
    assert worst >= 0.05, worst   # the bound is not vacuous


def test_reference_gradient_is_the_plain_backward_on_rounded_values():
    """gradient_term_scale's gradient equals the FD-pinned plain backward of
    the network whose weights and inputs are already BF16 values."""
    rng = np.random.default_rng(6)
    th = M.init_theta(7).astype(np.float64) + 0.02 * rng.standard_normal(M.N_PARAMS)
    d = M.unpack(th)
    for l in range(5):
        d[f"W{l}"] = M.bf16_round(d[f"W{l}"])
    thr = M.pack(d)
    X = M.bf16_round(rng.uniform(-1, 1, (64, 7)))
    y = rng.standard_normal(64)
    gr, sc, L = M.gradient_term_scale(thr, X, y)
    Y, cache = M.forward(thr, X, bf16=False)
    L2, dY = M.nll(Y, y)
    np.testing.assert_allclose(gr, M.backward(cache, dY), rtol=1e-12, atol=1e-15)
    assert L == pytest.approx(L2, rel=1e-14)
    assert np.all(sc >= np.abs(gr) - 1e-15)
