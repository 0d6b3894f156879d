"""Writes tests/golden/batch_converged.json: converged magnifications of a
fixed sample of the 64-set binary batch (seed 2), from the FP64 oracle at a
2048 x 4096 polar grid (radial error ~ N_r^-1.5 ~ 1e-5).  It calls only
oracle/.  The sample: for 16 sets (every 4th), the epoch of highest
point-source magnification and two random epochs, 48 in all.

Run:  python tests/golden/make_batch_converged.py   (about 5 CPU minutes,
      parallel over processes started with spawn)
"""
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

REF_GRID = dict(n_r=2048, n_theta=4096, n_limb=500)


def one(args):
    s, e = args
    import oracle
    from paper_2510_02639_gb300 import inputs as I
    params, t = I.binary_batch()
    A, st = oracle.magnification([params[s]], [t[s, e]], I.grid(**REF_GRID))
    return s, e, float(A[0, 0]), int(st[0, 0])


def main():
    import oracle
    from paper_2510_02639_gb300 import inputs as I
    oracle.build()
    params, t = I.binary_batch()
    rng = np.random.default_rng(2024)
    picks = []
    g = I.grid()
    for s in range(0, 64, 4):
        w = oracle.source_centre(params[s], t[s])
        Aps = oracle.point_source(params[s], g, w)[0]
        picks.append((s, int(np.argmax(Aps))))
        picks += [(s, int(e)) for e in rng.integers(0, t.shape[1], 2)]
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        rows = pool.map(one, picks)
    out = {"description": "FP64 oracle magnifications of sampled epochs of the 64 x 10,000 binary batch "
                          "(inputs.binary_batch(), seed 2) at a 2048 x 4096 grid, N_limb = 500",
           "grid": REF_GRID, "epochs": [{"set": s, "epoch": e, "A": A, "status": st} for s, e, A, st in rows]}
    with open(os.path.join(HERE, "batch_converged.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
