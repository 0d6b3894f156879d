"""Pins of the oracle's linear-flux marginalised likelihood (Appendix B).

Each pin reaches the same quantity by a route that does not use the oracle's
Woodbury evaluation: the dense Gaussian log-density with B = C + M Lambda M^T
formed explicitly, central differences, and weighted least squares."""
import numpy as np
import pytest

from oracle import likelihood as LK


def _case(rng, n):
    A = 1.0 + rng.gamma(1.5, 2.0, n)             # magnifications >= 1
    sigma = rng.uniform(0.005, 0.05, n)
    FS, Fb = rng.uniform(0.3, 3.0), rng.uniform(0.5, 2.0)
    F = (A - 1.0) * FS + Fb + rng.normal(0.0, sigma)
    mu = rng.uniform(-1.0, 2.0, 2)
    lam = rng.uniform(0.5, 20.0, 2)
    return A, F, sigma, mu, lam


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_woodbury_equals_dense_density(seed):
    rng = np.random.default_rng(seed)
    A, F, sigma, mu, lam = _case(rng, 40)
    # B is ill-conditioned (sigma^2 ~ 1e-5 beside M Lambda M^T ~ 1e2): the
    # dense solve carries ~1e-11 relative rounding
    assert LK.nll(A, F, sigma, mu, lam) == pytest.approx(LK.nll_dense(A, F, sigma, mu, lam), rel=1e-9)


def test_dense_density_is_the_gaussian_log_density():
    """nll_dense + n/2 ln(2 pi) equals -log N(F | M mu, B) from scipy."""
    from scipy.stats import multivariate_normal
    rng = np.random.default_rng(5)
    A, F, sigma, mu, lam = _case(rng, 25)
    M = np.stack([A - 1.0, np.ones_like(A)], axis=1)
    B = np.diag(sigma ** 2) + M @ np.diag(lam) @ M.T
    ref = -multivariate_normal(mean=M @ mu, cov=B).logpdf(F)
    assert LK.nll_dense(A, F, sigma, mu, lam) + 0.5 * len(A) * np.log(2 * np.pi) == pytest.approx(ref, rel=1e-10)


@pytest.mark.parametrize("seed", [10, 11])
def test_gradient_wrt_A_by_central_differences(seed):
    rng = np.random.default_rng(seed)
    A, F, sigma, mu, lam = _case(rng, 30)
    g = LK.nll_grad_A(A, F, sigma, mu, lam)
    for e in range(len(A)):
        # differences of the Woodbury value (the dense one's rounding, ~1e-9
        # absolute, would dominate a difference quotient)
        h = 1e-4 * max(1.0, abs(A[e]))
        Ap, Am = A.copy(), A.copy()
        Ap[e] += h
        Am[e] -= h
        fd = (LK.nll(Ap, F, sigma, mu, lam) - LK.nll(Am, F, sigma, mu, lam)) / (2 * h)
        assert g[e] == pytest.approx(fd, rel=1e-5, abs=1e-6 * np.abs(g).max())


def test_posterior_mean_flat_prior_is_weighted_least_squares():
    rng = np.random.default_rng(7)
    A, F, sigma, mu, lam = _case(rng, 60)
    lam = np.array([1e14, 1e14])
    M = np.stack([A - 1.0, np.ones_like(A)], axis=1)
    w = 1.0 / sigma
    ls = np.linalg.lstsq(M * w[:, None], F * w, rcond=None)[0]
    np.testing.assert_allclose(LK.posterior_mean(A, F, sigma, mu, lam), ls, rtol=1e-8)


def test_chain_rule_through_parameters():
    """With A(p) = A0 + J p, the chained gradient equals differences in p."""
    rng = np.random.default_rng(9)
    A0, F, sigma, mu, lam = _case(rng, 35)
    J = rng.normal(0.0, 0.3, (35, 8))
    nllp = lambda p: LK.nll(A0 + J @ p, F, sigma, mu, lam)
    p0 = np.zeros(8)
    _, g = LK.nll_and_grad(A0, J, F, sigma, mu, lam)
    for q in range(8):
        d = np.zeros(8)
        d[q] = 1e-4
        fd = (nllp(p0 + d) - nllp(p0 - d)) / 2e-4
        assert g[q] == pytest.approx(fd, rel=1e-5, abs=1e-6 * np.abs(g).max())
