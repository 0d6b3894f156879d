"""Small, self-contained launches of the library's kernels for profilers.

    python -m paper_2510_02639_gb300.profile_case mag --n-r 1024 --n-theta 2048
    python -m paper_2510_02639_gb300.profile_case der
    python -m paper_2510_02639_gb300.profile_case diag
    python -m paper_2510_02639_gb300.profile_case laws --sets-stride 1 --epochs-stride 10
    python -m paper_2510_02639_gb300.profile_case mlp_infer --queries 1048576
    python -m paper_2510_02639_gb300.profile_case mlp_train --queries 65536

mag / der: one icrs_magnification / icrs_chi2_grad launch on a strided slice
of the 64-set binary batch (every --sets-stride-th set, every
--epochs-stride-th epoch).  diag: the same slice through
icrs_magnification_diag; prints the clock share of the root and sector
phases against the ray phase, and the counts of FP64 fallbacks.  laws: the
mag launch on the same slice for the sets' linear law and for the same sets
with inputs.SOURCE_LAWS' power4 and spot laws, each event-timed after one
untimed launch.  mlp_infer / mlp_train: one inference launch or
one training step of the surrogate on synthetic features.  Each case runs its
launch once untimed and once more, so a profiler can skip the first
(`-s 1` style filters) or take both.
"""
from __future__ import annotations

import argparse

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["mag", "der", "diag", "laws", "mlp_infer", "mlp_train"])
    ap.add_argument("--n-r", type=int, default=1024)
    ap.add_argument("--n-theta", type=int, default=2048)
    ap.add_argument("--sets-stride", type=int, default=2)
    ap.add_argument("--epochs-stride", type=int, default=1000)
    ap.add_argument("--queries", type=int, default=1 << 20)
    args = ap.parse_args(argv)

    import torch

    from . import build as B
    B.build()
    from . import icrs
    from . import inputs as I
    from . import surrogate as SG

    if args.case == "diag":
        params, t = I.binary_batch()
        sel = list(range(0, len(params), args.sets_stride))
        tt = torch.tensor(np.ascontiguousarray(t[sel][:, :: args.epochs_stride]), device="cuda")
        g = icrs.grid_from_dict(I.grid(n_r=args.n_r, n_theta=args.n_theta), 2)
        pd = icrs.params_to_device([params[s] for s in sel])
        A, st, sect, cnt, _ = icrs.magnification_diag(pd, tt, g)
        torch.cuda.synchronize()
        c = cnt.reshape(-1, 16).long().sum(0).tolist()
        root, rays = sum(c[4:12]), c[12]
        nsect = int(((st.long() >> 8) & 0xFF).sum().item())
        nray = nsect * args.n_r * args.n_theta
        print(f"diag: {tt.numel()} epochs at {args.n_r}x{args.n_theta}; sectors {nsect}, rays {nray}")
        print(f"  block clocks: root and sector phases {root} ({100 * root / max(root + rays, 1):.1f}%), "
              f"ray phase {rays} ({100 * rays / max(root + rays, 1):.1f}%)")
        print(f"  FP64 polishes {c[0]}, FP64 validations {c[1]}, FP64 rays {c[2]} ({c[2] / max(nray, 1):.2e} of rays), "
              f"FP64 crossings {c[3]}")
        return
    if args.case == "laws":
        params, t = I.binary_batch()
        sel = list(range(0, len(params), args.sets_stride))
        tt = torch.tensor(np.ascontiguousarray(t[sel][:, :: args.epochs_stride]), device="cuda")
        g = icrs.grid_from_dict(I.grid(n_r=args.n_r, n_theta=args.n_theta), 2)
        for name in ("linear", "power4", "spot"):
            pd = icrs.params_to_device([dict(params[s], **I.SOURCE_LAWS[name]) for s in sel])
            A, st = icrs.magnification(pd, tt, g)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            icrs.magnification(pd, tt, g, out=A, status=st)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            print(f"laws: {name}: {tt.numel()} epochs at {args.n_r}x{args.n_theta}, {ms:.1f} ms, "
                  f"{tt.numel() / ms * 1e3:.0f} magnifications/s, finite {bool(torch.isfinite(A).all())}")
        return
    if args.case in ("mag", "der"):
        params, t = I.binary_batch()
        sel = list(range(0, len(params), args.sets_stride))
        ps = [params[s] for s in sel]
        tt = torch.tensor(np.ascontiguousarray(t[sel][:, :: args.epochs_stride]), device="cuda")
        g = icrs.grid_from_dict(I.grid(n_r=args.n_r, n_theta=args.n_theta), 2)
        pd = icrs.params_to_device(ps)
        for _ in range(2):
            if args.case == "mag":
                A, st = icrs.magnification(pd, tt, g)
            else:
                y = torch.ones_like(tt)
                _, _, A, _ = icrs.chi2_grad(pd, tt, g, y, torch.full_like(tt, 0.01))
        torch.cuda.synchronize()
        msg = f"{args.case}: {tt.numel()} epochs at {args.n_r}x{args.n_theta}, sum A = {float(A.sum()):.6f}"
        if args.case == "mag":
            nsect = int(((st.long() >> 8) & 0xFF).sum().item())
            msg += f", sectors {nsect}, rays {nsect * args.n_r * args.n_theta}"
        print(msg)
        return
    rng = np.random.default_rng(0)
    n = args.queries
    f = np.zeros((n, 8), dtype=np.float32)
    f[:, :7] = rng.uniform(-1, 1, (n, 7))
    feat = torch.tensor(f, device="cuda")
    th = torch.tensor(SG.init_theta(0), device="cuda")
    pack = icrs.mlp_pack(th)
    if args.case == "mlp_infer":
        for _ in range(2):
            out = icrs.mlp_infer(pack, th, feat)
        torch.cuda.synchronize()
        print(f"mlp_infer: {n} queries, sum = {float(out.sum()):.6f}")
    else:
        y = torch.tensor(rng.standard_normal(n).astype(np.float32), device="cuda")
        m, v = torch.zeros_like(th), torch.zeros_like(th)
        ws = icrs.mlp_workspace(n)
        for step in (1, 2):
            icrs.mlp_train_step(th, m, v, pack, step, 1e-3, feat, y, workspace=ws)
        torch.cuda.synchronize()
        print(f"mlp_train: {n} samples, |theta| = {float(th.abs().sum()):.6f}")


if __name__ == "__main__":
    main()
