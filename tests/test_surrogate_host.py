"""Host logic of the surrogate's gate calibration (no GPU): the exceedance
budget of _loosest_prefix and its use by calibrate() on a synthetic
validation set."""
import numpy as np
import torch

from paper_2510_02639_gb300 import surrogate as SG


def test_loosest_prefix_budget():
    ok = torch.tensor([1, 1, 0, 1, 1, 1, 1, 1, 1, 1], dtype=torch.bool)
    err = torch.tensor([0, 0, 9, 0, 5, 0, 0, 0, 0, 5.0])
    # no budget: stop before the first accepted exceedance (entry 2 is not accepted)
    assert SG._loosest_prefix(ok, err, 1.0, 0.0) == 3
    # one exceedance per four accepted entries: the whole list
    assert SG._loosest_prefix(ok, err, 1.0, 0.25) == 9
    # the first accepted entry already exceeds: nothing
    assert SG._loosest_prefix(torch.tensor([True]), torch.tensor([2.0]), 1.0, 0.5) == -1
    # brute force on random lists
    rng = np.random.default_rng(0)
    for _ in range(200):
        n = int(rng.integers(1, 40))
        o = torch.tensor(rng.random(n) < 0.8)
        e = torch.tensor(rng.random(n))
        f = float(rng.choice([0.0, 0.1, 0.3]))
        want = -1
        for i in range(n):
            acc = o[: i + 1].numpy()
            bad = int(np.sum(acc & (e[: i + 1].numpy() > 0.9)))
            if bad <= int(np.floor(f * acc.sum())):
                want = i
        assert SG._loosest_prefix(o, e, 0.9, f) == want


class _FakeSur:
    def __init__(self, sig):
        self.sig = sig

    def predict(self, feat):
        n = feat.shape[0]
        return torch.stack([torch.zeros(n), 2.0 * torch.log(self.sig)], 1).float()


def test_calibrate_tolerates_rare_label_outliers():
    """10,000 validation epochs with sigma = 1..10,000 (in units of 1e-6);
    every label is exact except one outlier at sigma rank 100.  Without a
    budget sigma_max stops below it; with a budget of 1e-4 it reaches the
    top."""
    n = 10_000
    sig = torch.arange(1, n + 1, dtype=torch.float64) * 1e-6
    feat = torch.zeros(n, 8)
    A = torch.ones(n, dtype=torch.float64)
    A[99] = 1.0 + 1e-3
    val = SG.Dataset(feat=feat, A_ps=torch.ones(n, dtype=torch.float64), st=torch.zeros(n, dtype=torch.int32),
                     A=A, target=torch.zeros(n), params=None, t=None)
    g0 = SG.calibrate(_FakeSur(sig), val, exceed_frac=0.0)
    g1 = SG.calibrate(_FakeSur(sig), val, exceed_frac=1e-4)
    assert abs(g0.sigma_max - 99e-6) < 1e-9
    assert abs(g1.sigma_max - 1e-2) < 1e-8
