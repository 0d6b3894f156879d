"""Seeded synthetic workloads shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the method: it only draws parameter sets and
epoch times with numpy's seeded generator and fixes the default grid.  The
shapes and distributions are those of the five benchmark workloads: a caustic
crossing binary light curve, a 64-set binary batch, a triple-lens light curve,
an adjoint batch around one binary point, and the surrogate's training/query
distribution.
"""
from __future__ import annotations

import numpy as np

# Default grid (Sec. 3.2-3.3: N_limb ~ 500; polar grid N_r x N_theta per sector).
DEFAULT_GRID = dict(
    n_r=64, n_theta=256, n_limb=500, n_bins_r=32, n_bins_theta=128,
    max_iter=100, uniform=0, delta_c=0.02, margin=0.05, img_tol=1e-3, ld_split=0,
    grad_rule=0, s_fac=100.0,
)


def grid(**kw) -> dict:
    g = dict(DEFAULT_GRID)
    g.update(kw)
    return g


def binary(t0=0.0, tE=20.0, u0=0.01, alpha=0.5, rho=1e-3, u1=0.5, s=1.0, q=1e-3, u2=0.0) -> dict:
    return dict(t0=t0, tE=tE, u0=u0, alpha=alpha, rho=rho, u1=u1, n_lens=2, s=s, q=q,
                q2=0.0, q3=0.0, s2=0.0, s3=0.0, psi=0.0, u2=u2)


def triple(t0=0.0, tE=30.0, u0=0.005, alpha=2.0, rho=5e-4, u1=0.6,
           q2=1e-3, q3=3e-4, s2=1.0, s3=0.8, psi=1.2, u2=0.0) -> dict:
    return dict(t0=t0, tE=tE, u0=u0, alpha=alpha, rho=rho, u1=u1, n_lens=3, s=0.0, q=0.0,
                q2=q2, q3=q3, s2=s2, s3=s3, psi=psi, u2=u2)


def caustic_crossing_binary(n_epochs: int = 500):
    """Binary s=1, q=1e-3, rho=1e-3, u=0.5, u0=0.01, alpha=0.5, tE=20 d,
    epochs uniform in [-0.5, 0.5] d."""
    p = binary()
    t = np.linspace(-0.5, 0.5, n_epochs)
    return [p], t[None, :]


# Source laws applied on top of a workload's sets (bench.py --law,
# profile_case laws): the sets' own linear law, a quadratic term, the
# four-coefficient power series in mu^(1/2) in place of u1, or a dark
# circular spot (centre (0.3, -0.2) rho, radius 0.4 rho, contrast 0.5).
SOURCE_LAWS = {
    "linear": {},
    "quadratic": dict(u2=0.2),
    "power4": dict(u1=0.0, a1=0.6, a2=0.3, a3=-0.2, a4=0.1),
    "spot": dict(spot_x=0.3, spot_y=-0.2, spot_r=0.4, spot_c=0.5),
}


def binary_batch(n_sets: int = 64, n_epochs: int = 10_000, seed: int = 2):
    """log10 q ~ U[-5,-1], s log-uniform [0.3, 3], rho log-uniform [1e-4, 1e-2],
    u0 ~ U[-0.1, 0.1], alpha ~ U[0, 2 pi), u ~ U[0.3, 0.8], tE = 20 d, t0 = 0;
    epochs uniform (sorted) in [t0 - 2 tE, t0 + 2 tE]."""
    rng = np.random.default_rng(seed)
    params, times = [], []
    for _ in range(n_sets):
        q = 10.0 ** rng.uniform(-5, -1)
        s = 10.0 ** rng.uniform(np.log10(0.3), np.log10(3.0))
        rho = 10.0 ** rng.uniform(-4, -2)
        u0 = rng.uniform(-0.1, 0.1)
        alpha = rng.uniform(0, 2 * np.pi)
        u1 = rng.uniform(0.3, 0.8)
        p = binary(t0=0.0, tE=20.0, u0=u0, alpha=alpha, rho=rho, u1=u1, s=s, q=q)
        params.append(p)
        times.append(np.sort(rng.uniform(-40.0, 40.0, n_epochs)))
    return params, np.stack(times)


def triple_curve(n_epochs: int = 2000):
    """Triple lens q2=1e-3, q3=3e-4, s2=1, s3=0.8, psi=1.2, rho=5e-4, u=0.6,
    u0=0.005, alpha=2.0, tE=30 d; epochs uniform in [-0.1 tE, 0.1 tE]."""
    p = triple()
    t = np.linspace(-3.0, 3.0, n_epochs)
    return [p], t[None, :]


def adjoint_batch(n_sets: int = 256, n_epochs: int = 5000, seed: int = 4, noise: float = 0.01):
    """256 sets around (s, q, rho, u0, alpha, tE, u) = (0.9, 1e-4, 8e-4, 0.02, 1.0, 25, 0.5),
    each parameter scaled by (1 + 0.01 N(0,1)) (t0 shifted by 0.01 tE N(0,1));
    5000 epochs in [-2 tE, 2 tE].  Returns (params, t, centre, noise_draws); the
    data are y = A(centre) + noise * noise_draws (flux F = A)."""
    rng = np.random.default_rng(seed)
    centre = binary(t0=0.0, tE=25.0, u0=0.02, alpha=1.0, rho=8e-4, u1=0.5, s=0.9, q=1e-4)
    params = []
    for _ in range(n_sets):
        p = dict(centre)
        for k in ("tE", "u0", "alpha", "rho", "u1", "s", "q"):
            p[k] = centre[k] * (1.0 + 0.01 * rng.standard_normal())
        p["t0"] = centre["t0"] + 0.01 * centre["tE"] * rng.standard_normal()
        params.append(p)
    t = np.tile(np.linspace(-50.0, 50.0, n_epochs), (n_sets, 1))
    draws = rng.standard_normal((n_sets, n_epochs))
    return params, t, centre, noise * draws


def param_matrix(params) -> np.ndarray:
    """[S, 8] array (t0, tE, u0, alpha, s, q, rho, u1)."""
    return np.array([[p["t0"], p["tE"], p["u0"], p["alpha"], p["s"], p["q"], p["rho"], p["u1"]]
                     for p in params])
