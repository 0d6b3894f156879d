"""Writes tests/golden/batch_qualification.json: the accuracy-qualification
sample of the 64-set binary batch (inputs.binary_batch(), seed 2).  It calls
only oracle/.

Sample (512 epochs):
  - the epoch of highest point-source magnification of every set (64);
  - 288 random (set, epoch) pairs;
  - 80 epochs of small sources (rho < 3e-4) at moderate point-source
    magnification, 2 <= A_ps <= 10, where the radial quadrature converges
    slowest;
  - 80 epochs whose source centre lies inside a caustic (five point-source
    images), where images sit close together.
For each: the FP64 oracle magnification at 1024 x 2048 (the benchmark's
grid), 2048 x 4096 and 4096 x 8192 (N_limb = 500).  The finest value is the
reference and the difference of the last two doublings bounds its own error
(Richardson: the quadrature error falls at least linearly with the grid
spacing, so the remaining error of the finest grid is below that
difference).

Run:  python tests/golden/make_batch_qualification.py   (about 7 minutes on
      8 cores; processes started with spawn)
"""
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

GRIDS = [dict(n_r=1024, n_theta=2048), dict(n_r=2048, n_theta=4096), dict(n_r=4096, n_theta=8192)]


def one(args):
    s, e, cls = args
    import oracle
    from paper_2510_02639_gb300 import inputs as I
    params, t = I.binary_batch()
    vals, sts = [], []
    for g in GRIDS:
        A, st = oracle.magnification([params[s]], [t[s, e]], I.grid(**g))
        vals.append(float(A[0, 0]))
        sts.append(int(st[0, 0]))
    return s, e, cls, vals, sts


def main():
    import oracle
    from paper_2510_02639_gb300 import inputs as I
    oracle.build()
    params, t = I.binary_batch()
    S, E = t.shape
    g = I.grid()
    Aps = np.zeros((S, E))
    nimg = np.zeros((S, E), dtype=int)
    for s in range(S):
        w = oracle.source_centre(params[s], t[s])
        A, n, _, _ = oracle.point_source(params[s], g, w)
        Aps[s], nimg[s] = A, n
    rng = np.random.default_rng(4242)
    picks = {}
    for s in range(S):
        picks[(s, int(np.argmax(Aps[s])))] = "peak"
    while len(picks) < 64 + 288:
        k = (int(rng.integers(S)), int(rng.integers(E)))
        picks.setdefault(k, "random")
    small = [(s, e) for s in range(S) if params[s]["rho"] < 3e-4
             for e in np.flatnonzero((Aps[s] >= 2.0) & (Aps[s] <= 10.0))]
    inside = [(s, int(e)) for s in range(S) for e in np.flatnonzero(nimg[s] == 5)]
    for cls, pool_, n in (("small_rho_moderate_A", small, 80), ("inside_caustic", inside, 80)):
        order = rng.permutation(len(pool_))
        added = 0
        for i in order:
            k = (int(pool_[i][0]), int(pool_[i][1]))
            if k in picks:
                continue
            picks[k] = cls
            added += 1
            if added == n:
                break
    items = [(s, e, c) for (s, e), c in sorted(picks.items())]
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        rows = pool.map(one, items, chunksize=1)
    out = {"description": "FP64 oracle magnifications of the accuracy-qualification sample of the "
                          "64 x 10,000 binary batch (inputs.binary_batch(), seed 2), N_limb = 500, "
                          "at each grid of `grids`",
           "grids": GRIDS,
           "epochs": [{"set": s, "epoch": e, "class": c, "A": v, "status": st} for s, e, c, v, st in rows]}
    with open(os.path.join(HERE, "batch_qualification.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
