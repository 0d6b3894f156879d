"""Linear-flux marginalised likelihood of a microlensing light curve (FP64).

TEST INFRASTRUCTURE ONLY: like the rest of ``oracle/``, only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs use it.

Appendix B of the paper (Miyazaki & Kawahara, arXiv:2510.02639).  One data
set j has fluxes F (n epochs), diagonal covariance C = diag(sigma^2) and the
model F = (A - 1) F_S + F_base, which is linear in beta = (F_S, F_base):

    M = [[A_1 - 1, 1], ..., [A_n - 1, 1]]   (n x 2 design matrix)
    beta ~ N(mu, Lambda),  Lambda = diag(lambda_S, lambda_base).

Marginalising beta gives F ~ N(M mu, B), B = C + M Lambda M^T, and the
negative log-likelihood of Eq. (NLL)

    NLL = 1/2 (F - M mu)^T B^-1 (F - M mu) + 1/2 ln |B|,

evaluated with the matrix inversion lemma (Woodbury identity) printed right
after it:

    B^-1  = C^-1 - C^-1 M K^-1 M^T C^-1,   K = Lambda^-1 + M^T C^-1 M,
    ln|B| = ln|C| + ln|Lambda| + ln|K|.

As printed, the NLL carries no n/2 ln(2 pi) term.

Gradient with respect to the magnifications (matrix calculus on the same
expression; dM = e_e e_1^T dA_e):

    dNLL/dA_e = c_e [ (K^-1 m_e)_1 - (F_e - m_e . a) a_1 ],

with c_e = 1/sigma_e^2, m_e = (A_e - 1, 1) and a = mu + K^-1 M^T C^-1 (F -
M mu), the posterior mean of beta (the paper's a(theta)).  The gradient with
respect to the lens parameters is the chain sum_e dNLL/dA_e dA_e/dp.

Pins (tests/test_oracle_likelihood.py): the Woodbury form against the dense
Gaussian log-density with B built explicitly; dNLL/dA against central
differences of the NLL; a against the weighted least-squares solution in the
limit of a flat prior.
"""
from __future__ import annotations

import numpy as np


def _terms(A, F, sigma, mu, lam):
    A = np.asarray(A, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    M = np.stack([A - 1.0, np.ones_like(A)], axis=1)          # n x 2
    c = 1.0 / sigma ** 2                                      # C^-1 (diagonal)
    r = F - M @ mu                                            # F - M mu
    K = np.diag(1.0 / lam) + M.T @ (c[:, None] * M)           # Lambda^-1 + M^T C^-1 M
    v = M.T @ (c * r)                                         # M^T C^-1 (F - M mu)
    return M, c, r, K, v


def nll(A, F, sigma, mu, lam) -> float:
    """Eq. (NLL) of one data set through the Woodbury identity."""
    M, c, r, K, v = _terms(A, F, sigma, mu, lam)
    Kinv_v = np.linalg.solve(K, v)
    quad = np.sum(c * r * r) - v @ Kinv_v                    # r^T B^-1 r
    logdet = (np.sum(np.log(np.asarray(sigma, dtype=np.float64) ** 2)) + np.sum(np.log(lam))
              + np.linalg.slogdet(K)[1])                      # ln|C| + ln|Lambda| + ln|K|
    return 0.5 * quad + 0.5 * logdet


def nll_dense(A, F, sigma, mu, lam) -> float:
    """The same NLL from B = C + M Lambda M^T formed explicitly (small n)."""
    A = np.asarray(A, dtype=np.float64)
    M = np.stack([A - 1.0, np.ones_like(A)], axis=1)
    B = np.diag(np.asarray(sigma, dtype=np.float64) ** 2) + M @ np.diag(lam) @ M.T
    r = np.asarray(F, dtype=np.float64) - M @ np.asarray(mu, dtype=np.float64)
    return 0.5 * r @ np.linalg.solve(B, r) + 0.5 * np.linalg.slogdet(B)[1]


def posterior_mean(A, F, sigma, mu, lam) -> np.ndarray:
    """a = mu + K^-1 M^T C^-1 (F - M mu): the posterior mean of (F_S, F_base)."""
    M, c, r, K, v = _terms(A, F, sigma, mu, lam)
    return np.asarray(mu, dtype=np.float64) + np.linalg.solve(K, v)


def nll_grad_A(A, F, sigma, mu, lam) -> np.ndarray:
    """dNLL/dA_e for every epoch of one data set."""
    M, c, r, K, v = _terms(A, F, sigma, mu, lam)
    a = np.asarray(mu, dtype=np.float64) + np.linalg.solve(K, v)
    Kinv = np.linalg.inv(K)
    resid = np.asarray(F, dtype=np.float64) - M @ a           # F_e - m_e . a
    return c * ((M @ Kinv[:, 0]) - resid * a[0])


def nll_and_grad(A, dA, F, sigma, mu, lam):
    """NLL and dNLL/dp of one data set, given A [n] and dA/dp [n, P]."""
    g = nll_grad_A(A, F, sigma, mu, lam)
    return nll(A, F, sigma, mu, lam), g @ np.asarray(dA, dtype=np.float64)
