"""Gated surrogate of the finite-source magnification (orchestration only).

The surrogate is not in the paper.  All arithmetic runs in the CUDA library:
features and point-source magnification, ICRS targets, the network's
training and inference on tensor cores, the gate, and ICRS on the routed
epochs.  This module sequences those calls, shuffles the training data and
calibrates the gate.

Target: y = 1e4 log(A_ICRS / A_ps) minus b, the second-order finite-source
estimate of the feature kernel (features[:, 7]: the disk average of the
point-source magnification from its 32 limb values and the limb-darkening
law's second moment).  Prediction: A = A_ps exp(1e-4 (b + mu)).
Gate: an epoch is accepted when its point-source solves are clean (no caustic
inside the disk), its caustic feature is >= caustic_min, the predicted
standard deviation exp(s / 2) is <= sigma_max, |mu| <= mu_max, |b| <= b_max,
and A_ps <= A_max (A_small when rho < rho_min).
Everything else runs through ICRS.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import icrs
from . import inputs as I


def init_theta(seed: int = 0) -> np.ndarray:
    """Uniform He initialisation, zero biases, a 10x smaller output layer."""
    rng = np.random.default_rng(seed)
    parts = []
    for out, inp, last in ((128, 7, False), (128, 128, False), (128, 128, False), (128, 128, False), (2, 128, True)):
        lim = np.sqrt(6.0 / inp) * (0.1 if last else 1.0)
        parts.append(rng.uniform(-lim, lim, out * inp))
        parts.append(np.zeros(out))
    th = np.concatenate(parts).astype(np.float32)
    assert th.size == icrs.MLP_NPARAM
    return th


@dataclass
class Dataset:
    feat: object      # [n, 8] float32 (device)
    A_ps: object      # [n] float64
    st: object        # [n] int32 point-source status
    A: object         # [n] float64 ICRS magnification
    target: object    # [n] float32, 1e4 log(A / A_ps) - b (b = feat[:, 7])
    params: object    # device icrs_params of the sets
    t: object         # [S, E] float64 times


def make_dataset(n_sets: int, n_epochs: int, seed: int, grid: dict | None = None, device="cuda") -> Dataset:
    """Sets from the binary batch distribution (log10 q ~ U[-5,-1], s log-uniform
    [0.3, 3], rho log-uniform [1e-4, 1e-2], ...), epochs uniform over
    [t0 - 2 tE, t0 + 2 tE]."""
    import torch
    g = grid or I.grid()
    params, t = I.binary_batch(n_sets=n_sets, n_epochs=n_epochs, seed=seed)
    pd = icrs.params_to_device(params, device)
    tt = torch.tensor(t, dtype=torch.float64, device=device)
    gr = icrs.grid_from_dict(g, 2)
    feat, Aps, st = icrs.surrogate_features(pd, tt, gr)
    A, _ = icrs.magnification(pd, tt, gr)
    A = A.reshape(-1)
    target = icrs.surrogate_target(A, Aps, feat)
    return Dataset(feat, Aps, st, A, target, pd, tt)


class Surrogate:
    def __init__(self, seed: int = 0, device="cuda"):
        import torch
        self.device = device
        self.theta = torch.tensor(init_theta(seed), device=device)
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.pack = icrs.mlp_pack(self.theta)
        self.step = 0
        self.err = torch.zeros(1, dtype=torch.int32, device=device)

    def train(self, data: Dataset, epochs: int = 20, batch: int = 8192, lr: float = 2e-3, lr_min: float = 5e-5,
              clip: float = 400.0, seed: int = 0):
        """Adam on the mean Gaussian NLL with a cosine learning-rate schedule.
        Samples with a flagged point-source solve or |y| > clip are left out
        (the gate routes such epochs to ICRS anyway).  Returns per-epoch mean
        losses."""
        import torch
        keep = (data.st == 0) & (data.target.abs() <= clip) & torch.isfinite(data.target)
        feat = data.feat[keep].contiguous()
        y = data.target[keep].contiguous()
        n = feat.shape[0]
        nb = max(1, n // batch)
        ws = icrs.mlp_workspace(batch, self.device)
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        gen = torch.Generator(device=self.device)
        gen.manual_seed(seed)
        total = epochs * nb
        out = []
        fb = torch.empty((batch, 8), dtype=torch.float32, device=self.device)
        yb = torch.empty((batch,), dtype=torch.float32, device=self.device)
        for ep in range(epochs):
            # the shuffle is an input (random draws); the gather runs in the library
            perm = torch.randperm(n, device=self.device, generator=gen).to(torch.int32)
            acc = torch.zeros((), dtype=torch.float64, device=self.device)
            for b in range(nb):
                icrs.surrogate_batch(feat, y, perm[b * batch:(b + 1) * batch], fb, yb)
                k = ep * nb + b
                lr_k = lr_min + 0.5 * (lr - lr_min) * (1.0 + np.cos(np.pi * k / total))
                self.step += 1
                icrs.mlp_train_step(self.theta, self.m, self.v, self.pack, self.step, lr_k, fb, yb, workspace=ws,
                                    loss=loss, err=self.err)
                acc += loss[0].double()
            out.append(float(acc.item()) / nb)
        if int(self.err.item()) != 0:
            raise icrs.IcrsError("tensor-core completion wait timed out during training")
        return out

    def predict(self, feat):
        return icrs.mlp_infer(self.pack, self.theta, feat, err=self.err)

    def gated_magnification(self, params_dev, t, grid, gate, feat=None, A_ps=None, st=None,
                            return_index=False):
        """A [S * E] through the gate (a Gate from calibrate()): accepted
        epochs from the surrogate, routed epochs from ICRS.  Returns (A,
        number routed), and the routed indices (items s * E + e, the first
        k entries) when return_index is set."""
        if feat is None:
            feat, A_ps, st = icrs.surrogate_features(params_dev, t, grid)
        pred = self.predict(feat)
        A, idx, nr = icrs.surrogate_gate(pred, feat, A_ps, st, gate.sigma_max, gate.mu_max, gate.b_max,
                                         gate.caustic_min, gate.A_max, gate.rho_min, gate.A_small)
        k = int(nr.item())
        if k:
            icrs.magnification_indexed(params_dev, t, grid, idx, k, A)
        return (A, k, idx[:k]) if return_index else (A, k)


def preselected_magnification(params_dev, t, grid, caustic_min: float, b_max: float, n_ext: int = 0,
                              mode: int = 1, A_max: float = 10.0, rho_min: float = 5e-4, A_small: float = 2.0,
                              feat=None, A_ps=None, st=None, return_index=False):
    """A [S * E] with the non-learned preselection (icrs_epoch_gate): epochs
    near a caustic, and those within n_ext epochs of one on the same light
    curve, run ICRS; the others get the second-order estimate (mode 1) or the
    point-source value (mode 0).  Returns (A, number routed[, indices])."""
    S = params_dev.numel() // icrs.PARAMS_DTYPE.itemsize
    E = t.shape[-1]
    if feat is None:
        feat, A_ps, st = icrs.surrogate_features(params_dev, t, grid)
    A, idx, nr = icrs.epoch_gate(feat, A_ps, st, S, E, n_ext, mode, b_max, caustic_min, A_max, rho_min, A_small)
    k = int(nr.item())
    if k:
        icrs.magnification_indexed(params_dev, t, grid, idx, k, A)
    return (A, k, idx[:k]) if return_index else (A, k)


@dataclass
class Gate:
    sigma_max: float
    mu_max: float
    b_max: float
    caustic_min: float
    A_max: float
    rho_min: float
    A_small: float


# Validation labels are ICRS at the headline grid, which is itself off by
# 1e-4 to 1e-2 on rare epochs (a sector shared by two images, small sources
# at moderate magnification).  No smooth model can predict those labels, so
# each calibration below tolerates up to EXCEED_FRAC exceedances per accepted
# validation epoch instead of none.
EXCEED_FRAC = 1e-4


def _loosest_prefix(ok_sorted, err_sorted, thr: float, frac: float) -> int:
    """Largest i such that, among the first i + 1 entries with ok_sorted set,
    at most floor(frac x their number) have err_sorted > thr; -1 if none."""
    import torch
    ok = ok_sorted.to(torch.int64)
    n_ok = torch.cumsum(ok, 0)
    n_bad = torch.cumsum(ok * (err_sorted > thr).to(torch.int64), 0)
    good = n_bad <= torch.floor(frac * n_ok.double()).to(torch.int64)
    idx = torch.nonzero(good)
    return int(idx.max().item()) if idx.numel() else -1


def calibrate(sur: Surrogate, val: Dataset, tol: float = 1e-4, margin: float = 2.0, mu_max: float = 2.0,
              b_max: float = 10.0, caustic_min: float = -1.0, A_max: float = 10.0, rho_min: float = 5e-4,
              A_small: float = 2.0, exceed_frac: float = EXCEED_FRAC) -> Gate:
    """Gate thresholds.  The physical ones are fixed:
      - |b| <= 10 (the second-order estimate within 1e-3), together with the
        limb roughness of the feature status (ICRS_ST_ROUGH: structure on
        the source's scale, where higher orders are not negligible);
      - |mu| <= 2 (the network corrects the estimate only slightly);
      - min |det J| >= 0.1 over the 33 point-source solves;
      - A_ps <= 10, and A_ps <= 2 when rho < 5e-4 (small sources away from
        the far field, and all sources at high magnification, are where
        ICRS at the headline grid itself still moves by 1e-4 between grid
        refinements, so no surrogate can track it to 1e-4).
    sigma_max is the largest value at which the accepted validation epochs
    stay within tol / margin of ICRS, up to exceed_frac of them."""
    import torch
    pred = sur.predict(val.feat)
    mu, s = pred[:, 0].double(), pred[:, 1].double()
    sig = torch.exp(0.5 * s)
    b = val.feat[:, 7].double()
    err = (val.A_ps * torch.exp((b + mu) / icrs.TARGET_SCALE) / val.A - 1.0).abs()
    base = ((val.st == 0) & (val.feat[:, 6] >= caustic_min) & (mu.abs() <= mu_max) & (b.abs() <= b_max)
            & (val.A_ps <= torch.where(val.feat[:, 4] >= float(np.log10(rho_min)) + 3.0, A_max, A_small)))
    order = torch.argsort(sig)
    last = _loosest_prefix(base[order], err[order], tol / margin, exceed_frac)
    smax = float(sig[order][last].item()) if last >= 0 else 0.0
    return Gate(smax, mu_max, b_max, caustic_min, A_max, rho_min, A_small)


def _clean_without_network(st):
    """Feature status that lets the non-learned rules (icrs_epoch_gate)
    accept an epoch: clean apart from ICRS_ST_PROFILE, since the second-order
    estimate uses each radial law's own second moment."""
    return (st & ~icrs.ST_PROFILE) == 0


def calibrate_point_source(val: Dataset, tol: float = 1e-4, margin: float = 2.0, use_estimate: bool = False,
                           exceed_frac: float = EXCEED_FRAC):
    """The method without the network: A = A_ps (use_estimate: A = A_ps
    exp(1e-4 b), the second-order estimate) where the solves are clean and the
    caustic feature is at least c; returns the smallest c whose accepted
    validation epochs stay within tol / margin (up to exceed_frac of them
    beyond it)."""
    import torch
    Aest = val.A_ps * torch.exp(val.feat[:, 7].double() / icrs.TARGET_SCALE) if use_estimate else val.A_ps
    err = (Aest / val.A - 1.0).abs()
    c = val.feat[:, 6].double()
    ok = _clean_without_network(val.st)
    order = torch.argsort(c, descending=True)
    last = _loosest_prefix(ok[order], err[order], tol / margin, exceed_frac)
    return float(c[order][last].item()) if last >= 0 else 2.0


def calibrate_estimate(val: Dataset, tol: float = 1e-4, margin: float = 2.0,
                       caustic_grid=(-6.0, -3.0, -2.0, -1.5, -1.0, -0.5, 0.0),
                       b_grid=(1.0, 3.0, 10.0, 30.0, 100.0, 300.0), A_max: float = 10.0, rho_min: float = 5e-4,
                       A_small: float = 2.0, exceed_frac: float = EXCEED_FRAC):
    """The second-order estimate without the network, A = A_ps exp(1e-4 b),
    with the same A_ps <= A_max cut: the (caustic_min, b_max) that accepts
    the most validation epochs while they stay within tol / margin (up to
    exceed_frac of them beyond it).  Returns (caustic_min, b_max)."""
    import torch
    b = val.feat[:, 7].double()
    err = (val.A_ps * torch.exp(b / icrs.TARGET_SCALE) / val.A - 1.0).abs()
    best, best_n = (2.0, 0.0), -1
    for c in caustic_grid:
        for bm in b_grid:
            sel = (_clean_without_network(val.st) & (val.feat[:, 6] >= c) & (b.abs() <= bm)
                   & (val.A_ps <= torch.where(val.feat[:, 4] >= float(np.log10(rho_min)) + 3.0, A_max, A_small)))
            n = int(sel.sum().item())
            n_bad = int((err[sel] > tol / margin).sum().item())
            if n > best_n and n_bad <= int(np.floor(exceed_frac * n)):
                best, best_n = (float(c), float(bm)), n
    return best
