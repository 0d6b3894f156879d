"""Writes tests/golden/near_critical_epochs.json: four epochs of the binary
scoring batch (inputs.binary_batch(n_sets=5000, n_epochs=2000, seed=503))
at which a limb point lies just inside a fold caustic, so that two of its
five images form a close pair (the script checks, on the oracle's
image-limb points, that some limb point has five images of which two are
closer than 3e-2).  An FP32 polynomial can round such a pair into a pair of
false roots (seen for pairs up to 2.6e-2 apart).  It stores the FP64 oracle magnification at the 1024 x 2048
grid, N_limb = 500.  It calls only oracle/.

The epochs were picked from the 10 million of that batch as the ones whose
result depended on where the root iteration started.

Run:  python tests/golden/make_near_critical_epochs.py   (a minute)
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

PICKS = [(166, 963), (1577, 968), (3497, 1093), (2975, 1004)]
GRID = dict(n_r=1024, n_theta=2048)


def closest_pair(oracle, p, t, g):
    """Smallest distance between two images of one limb point with five images."""
    lp = oracle.limb_points(p, t, g)
    best = np.inf
    for k in range(lp.shape[0]):
        v = lp[k, :, 2] > 0
        if v.sum() != 5:
            continue
        z = lp[k, v, 0] * np.exp(1j * lp[k, v, 1])
        d = np.abs(z[:, None] - z[None, :]) + np.eye(5) * 1e9
        best = min(best, float(d.min()))
    return best


def main():
    import oracle
    from paper_2510_02639_gb300 import inputs as I
    oracle.build()
    params, t = I.binary_batch(n_sets=5000, n_epochs=2000, seed=503)
    g = I.grid(**GRID)
    rows = []
    for s, e in PICKS:
        sep = closest_pair(oracle, params[s], float(t[s, e]), g)
        assert sep < 3e-2, (s, e, sep)
        A, st = oracle.magnification([params[s]], [t[s, e]], g)
        rows.append({"set": s, "epoch": e, "closest_pair": sep, "A": float(A[0, 0]), "status": int(st[0, 0])})
    out = {"description": "FP64 oracle magnifications of inputs.binary_batch(n_sets=5000, n_epochs=2000, "
                          "seed=503) epochs with a close image pair at a limb point",
           "batch": {"n_sets": 5000, "n_epochs": 2000, "seed": 503},
           "grid": GRID,
           "epochs": rows}
    with open(os.path.join(HERE, "near_critical_epochs.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
