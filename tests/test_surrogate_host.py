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


def test_status_rules_of_the_two_gates():
    """The learned gate's calibration accepts only clean feature status; the
    non-learned rules (second-order estimate, point source) also accept
    ICRS_ST_PROFILE, since their estimate uses each radial law's moment, and
    reject ICRS_ST_SPOT and the solve and roughness bits.  Exact labels, so
    only the status decides."""
    from paper_2510_02639_gb300 import icrs
    bits = [0, icrs.ST_PROFILE, icrs.ST_SPOT, icrs.ST_ROUGH, icrs.ST_LIMB | icrs.ST_PROFILE]
    n = len(bits)
    st = torch.tensor(bits, dtype=torch.int32)
    feat = torch.zeros(n, 8)
    feat[:, 4] = 3.0  # log10 rho + 3 = 0: rho = 1 (above rho_min)
    one = torch.ones(n, dtype=torch.float64)
    val = SG.Dataset(feat=feat, A_ps=one, st=st, A=one.clone(), target=torch.zeros(n), params=None, t=None)
    assert SG._clean_without_network(st).tolist() == [True, True, False, False, False]
    # every accepted epoch is exact, so the loosest rule wins: the smallest
    # caustic threshold and b_max of the grids
    assert SG.calibrate_estimate(val) == (-6.0, 1.0)
    g = SG.calibrate(_FakeSur(torch.full((n,), 1e-6, dtype=torch.float64)), val)
    assert abs(g.sigma_max - 1e-6) < 1e-12
    # a wrong label under ICRS_ST_PROFILE: every non-learned candidate rule
    # accepts it and so none qualifies (the (2, 0) sentinel), while the
    # learned rule never sees it
    val.A[1] = 2.0
    assert SG.calibrate_estimate(val, exceed_frac=0.0) == (2.0, 0.0)
    g = SG.calibrate(_FakeSur(torch.full((n,), 1e-6, dtype=torch.float64)), val, exceed_frac=0.0)
    assert abs(g.sigma_max - 1e-6) < 1e-12
