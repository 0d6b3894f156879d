"""Writes tests/golden/interval_edge_epochs.json: five epochs of the binary
scoring batch (inputs.binary_batch(n_sets=5000, n_epochs=2000, seed=503))
in which one image's lowest angle lies within 1e-7 rad above the first edge
of its angular interval (theta bins of width 2 pi / 128), so close that the
FP32 angle of that point can fall on the other side of the edge while its
FP64 angle bins it inside the interval.  The script checks that property on
the oracle's image-limb points and stores the FP64 oracle magnification at
the 1024 x 2048 grid, N_limb = 500.  It calls only oracle/.

The epochs were picked from the 10 million of that batch as the ones whose
sector construction is sensitive to how an angle next to an interval's
first edge is unwrapped.

Run:  python tests/golden/make_interval_edge_epochs.py   (seconds)
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

PICKS = [(1652, 1223), (2035, 1186), (3239, 800), (3208, 1396), (2843, 328)]
GRID = dict(n_r=1024, n_theta=2048)


def edge_gap(oracle, p, t, g):
    """Smallest (theta - first edge of its interval) over the points of each
    interval's first bin, for intervals preceded by an empty bin."""
    lp = oracle.limb_points(p, t, g)
    v = lp[..., 2] > 0
    th = lp[..., 1][v]
    bt = int(g["n_bins_theta"])
    ht = 2.0 * np.pi / bt
    tb = np.clip(np.floor((th + np.pi) / ht).astype(int), 0, bt - 1)
    occ = np.zeros(bt, bool)
    occ[tb] = True
    best = np.inf
    for b in np.flatnonzero(occ):
        if occ[(b - 1) % bt]:
            continue
        gap = float((th[tb == b] - (-np.pi + b * ht)).min())
        best = min(best, gap)
    return best


def main():
    import oracle
    from paper_2510_02639_gb300 import inputs as I
    oracle.build()
    params, t = I.binary_batch(n_sets=5000, n_epochs=2000, seed=503)
    g = I.grid(**GRID)
    rows = []
    for s, e in PICKS:
        gap = edge_gap(oracle, params[s], float(t[s, e]), g)
        assert 0.0 <= gap < 1e-7, (s, e, gap)
        A, st = oracle.magnification([params[s]], [t[s, e]], g)
        rows.append({"set": s, "epoch": e, "edge_gap": gap, "A": float(A[0, 0]), "status": int(st[0, 0])})
    out = {"description": "FP64 oracle magnifications of inputs.binary_batch(n_sets=5000, n_epochs=2000, "
                          "seed=503) epochs with an image angle just above an angular interval's first edge",
           "batch": {"n_sets": 5000, "n_epochs": 2000, "seed": 503},
           "grid": GRID,
           "epochs": rows}
    with open(os.path.join(HERE, "interval_edge_epochs.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
