"""Writes tests/golden/triple_qualification.json: the triple-lens light curve
(inputs.triple_curve(): q2 = 1e-3, q3 = 3e-4, s2 = 1, s3 = 0.8, psi = 1.2,
rho = 5e-4, u1 = 0.6, 2000 epochs) on 32 epochs (the 16 of highest
point-source magnification and 16 spread over the curve), from the FP64
oracle at 1024 x 2048 (the benchmark's grid), 2048 x 4096 and 4096 x 8192,
N_limb = 500.  It calls only oracle/.  The finest value is the reference;
the difference of the last two doublings bounds its own error.

Run:  python tests/golden/make_triple_qualification.py   (a few minutes on
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
    e, cls = args
    import oracle
    from paper_2510_02639_gb300 import inputs as I
    params, t = I.triple_curve()
    vals, sts = [], []
    for g in GRIDS:
        A, st = oracle.magnification(params, [t[0, e]], I.grid(**g))
        vals.append(float(A[0, 0]))
        sts.append(int(st[0, 0]))
    return e, cls, vals, sts


def main():
    import oracle
    from paper_2510_02639_gb300 import inputs as I
    oracle.build()
    params, t = I.triple_curve()
    w = oracle.source_centre(params[0], t[0])
    Aps = oracle.point_source(params[0], I.grid(), w)[0]
    picks = {int(e): "peak" for e in np.argsort(-Aps)[:16]}
    for e in np.linspace(0, t.shape[1] - 1, 16).astype(int):
        picks.setdefault(int(e), "spread")
    items = sorted(picks.items())
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        rows = pool.map(one, items, chunksize=1)
    out = {"description": "FP64 oracle magnifications of the triple-lens curve (inputs.triple_curve()), "
                          "N_limb = 500, at each grid of `grids`",
           "grids": GRIDS,
           "epochs": [{"epoch": e, "class": c, "A": v, "status": st} for e, c, v, st in rows]}
    with open(os.path.join(HERE, "triple_qualification.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
