"""GPU parity of the linear-flux marginalised likelihood (Appendix B) and its
gradient (icrs_marginal_nll_grad) against the oracle.

The NLL kernel's arithmetic is checked on the GPU's own magnifications: the
oracle's Woodbury NLL of those A values must agree to 1e-10 (FP64 sums in
another order).  The end-to-end NLL against the oracle's own A then differs
only through the forward error of A (1e-5 relative per epoch), bounded below
by sum_e |dnll/dA_e| 1e-5 A_e.  The gradient chains dnll/dA_e through dA/dp;
it is compared with the oracle's chain of its FP64 forward-mode dA/dp under
the adjoint tests' per-component bound weighted by |dnll/dA_e|, plus the
first-order effect of A's forward error on dnll/dA_e.
"""
import numpy as np
import pytest

from oracle import likelihood as LK
from paper_2510_02639_gb300 import inputs as I

pytestmark = pytest.mark.gpu

RTOL, ATOL, TAU = 2e-3, 5e-4, 1e-5


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_02639_gb300 import build as B
    B.build()
    from paper_2510_02639_gb300 import icrs
    return icrs


def _data(n_sets, n_epochs, stride):
    params, t, centre, noise = I.adjoint_batch()
    params = params[:n_sets]
    t = np.ascontiguousarray(t[:n_sets, ::stride][:, :n_epochs])
    noise = np.ascontiguousarray(noise[:n_sets, ::stride][:, :n_epochs])
    return params, t, centre, noise


def test_marginal_nll_and_gradient(G, oracle_mod):
    import torch
    params, t, centre, noise = _data(3, 60, 80)
    g = I.grid()
    S, E = t.shape
    # data: F = (A_centre - 1) F_S + F_base + noise with F_S = 1.3, F_base = 0.8
    Ac, _ = oracle_mod.magnification([centre] * S, t, g)
    F = (Ac - 1.0) * 1.3 + 0.8 + noise
    sigma = np.full_like(F, 0.01)
    prior = np.tile(np.array([1.0, 1.0, 4.0, 4.0]), (S, 1))
    dev = "cuda"
    pd = G.params_to_device(params)
    tt = torch.tensor(t, device=dev)
    nll, grad, fl, A, st = G.marginal_nll_grad(pd, tt, G.grid_from_dict(g, 2), torch.tensor(F, device=dev),
                                               torch.tensor(sigma, device=dev), torch.tensor(prior, device=dev))
    nll_f, _, fl_f, A_f, _ = G.marginal_nll_grad(pd, tt, G.grid_from_dict(g, 2), torch.tensor(F, device=dev),
                                                 torch.tensor(sigma, device=dev), torch.tensor(prior, device=dev),
                                                 grad=False)
    nll, grad, fl, A = (x.cpu().numpy() for x in (nll, grad, fl, A))
    nll_f, A_f = nll_f.cpu().numpy(), A_f.cpu().numpy()
    Ao, dAo, _ = oracle_mod.magnification_fwd(params, t, g)
    assert np.all(np.abs(A / Ao - 1.0) <= TAU)
    # the forward-only call and the derivative call give the same A (same method)
    assert np.all(np.abs(A_f / A - 1.0) <= TAU)
    for s in range(S):
        args = (F[s], sigma[s], prior[s, :2], prior[s, 2:])
        # the kernel's arithmetic on the GPU's own A
        assert nll[s] == pytest.approx(LK.nll(A[s], *args), rel=1e-10, abs=1e-8)
        assert nll_f[s] == pytest.approx(LK.nll(A_f[s], *args), rel=1e-10, abs=1e-8)
        np.testing.assert_allclose(fl[s], LK.posterior_mean(A[s], *args), rtol=1e-9)
        # end to end against the oracle's A
        gA = LK.nll_grad_A(Ao[s], *args)
        bound = np.sum(np.abs(gA) * TAU * Ao[s])
        assert abs(nll[s] - LK.nll(Ao[s], *args)) <= bound, (s, nll[s], LK.nll(Ao[s], *args), bound)
        go = gA @ dAo[s]
        # bound: the adjoint's per-component bound on dA/dp weighted by
        # |dnll/dA_e|, plus the change of dnll/dA_e caused by A's forward
        # error (d(dnll/dA_e)/dA_e ~ c_e a_0^2, doubled for the coupling
        # through the posterior mean)
        a0 = LK.posterior_mean(Ao[s], *args)[0]
        dg = 2.0 * a0 ** 2 / sigma[s] ** 2 * TAU * Ao[s]
        adA = np.abs(dAo[s])
        tol = RTOL * (np.abs(gA) @ adA) + ATOL * np.sum(np.abs(gA)) * adA.max(axis=0) + dg @ adA
        tol[7] += np.sum(np.abs(gA) * TAU * Ao[s])
        assert np.all(np.abs(grad[s] - go) <= tol), (s, grad[s], go, tol)


def test_marginal_nll_invalid_prior_gives_nan(G):
    import torch
    params, t, centre, noise = _data(2, 8, 500)
    g = I.grid()
    S, E = t.shape
    dev = "cuda"
    F = torch.ones((S, E), dtype=torch.float64, device=dev)
    sigma = torch.full((S, E), 0.01, dtype=torch.float64, device=dev)
    prior = torch.tensor([[0.0, 0.0, 1.0, 1.0], [0.0, 0.0, -1.0, 1.0]], dtype=torch.float64, device=dev)
    nll, _, _, _, _ = G.marginal_nll_grad(G.params_to_device(params), torch.tensor(t, device=dev),
                                          G.grid_from_dict(g, 2), F, sigma, prior, grad=False)
    nll = nll.cpu().numpy()
    assert np.isfinite(nll[0]) and np.isnan(nll[1])
