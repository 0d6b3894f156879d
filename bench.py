"""Benchmark: limb-darkened binary-lens finite-source magnifications per second
at relative error <= 1e-4, chi^2 gradients per second, and the FP32 roofline
fraction of the fused ICRS kernel.

Headline workload: the 64-set binary batch with 10,000 epochs per set.
  - parameters: log10 q ~ U[-5,-1], s log-uniform [0.3, 3], rho log-uniform
    [1e-4, 1e-2], u ~ U[0.3, 0.8];
  - epochs uniform in [t0 - 2 tE, t0 + 2 tE];
  - 500 limb points, and the accuracy-qualified polar grid of 1024 x 2048
    rays per sector.
The qualification is measured in the same run. The GPU magnifications of
the 512-epoch qualification sample are compared with the oracle's 4096 x
8192 values (tests/golden/batch_qualification.json), whose own error is
bounded by their last Richardson difference; the line reports the error
distribution. The fixed 64 x 256 grid is measured as a secondary line with
its own measured error, which is above 1e-4.

One step is one call of icrs_magnification over the whole batch, a single
fused kernel launch. Inputs are resident in HBM. A 256 MiB write flushes the
L2 between timed steps, and each step is timed with CUDA events on the
launching stream.

The same line also carries:
  - "chi2_grad": chi^2 gradient evaluations per second on the adjoint batch.
    One unit is one set's 8-parameter gradient over its 5,000-epoch light
    curve. The batch is 256 sets around s=0.9, q=1e-4, rho=8e-4, each
    parameter perturbed by 1%, on the 64 x 256 grid.
  - "surrogate": the gated MLP path against plain ICRS at the headline grid.
    It is trained and calibrated on epochs of the batch distribution, then
    scored on unseen ones: speed-up, fraction routed to ICRS and maximum
    relative error. The point-source-only rule is reported beside it.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload and grid (the baseline arm).

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LD binary magnifications/s at rel.err<=1e-4; chi^2 grads/s; % FP32 peak"
FLOPS_PER_RAY = {2: 30.0, 3: 40.0}   # algorithmic FP32 flops per ray (lens map + brightness)
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
HEADLINE_GRID = dict(n_r=1024, n_theta=2048)
FIXED_GRID = dict(n_r=64, n_theta=256)
GOLDEN = os.path.join(ROOT, "tests", "golden", "batch_qualification.json")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def fp32_peak_tflops():
    mp = peaks()
    mhz = float(mp.get("sm_max_mhz", SM_MAX_MHZ))
    return SM_COUNT * FP32_LANES * 2.0 * mhz * 1e6 / 1e12


def workload(name, rank=0):
    from paper_2510_02639_gb300 import inputs as I
    if name == "batch":
        params, t = I.binary_batch(seed=2 + 1000 * rank)
        desc = dict(workload="binary_batch_64x10000", sets=64, epochs=10000)
    elif name == "caustic":
        params, t = I.caustic_crossing_binary()
        desc = dict(workload="binary_caustic_crossing_500", sets=1, epochs=500)
    elif name == "triple":
        params, t = I.triple_curve()
        desc = dict(workload="triple_2000", sets=1, epochs=2000)
    else:
        raise SystemExit(f"unknown workload {name}")
    return params, t, desc


def reduce_max(x: float, world: int, device) -> float:
    """Maximum of a per-rank time over the ranks of the job (x itself when
    the job has one rank): each replica's throughput counts against the
    slowest rank's clock."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    v = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(v, op=dist.ReduceOp.MAX)
    return float(v.item())


def job_rate(units_per_rank: int, world: int, steps: int, t_max_s: float) -> float:
    """Whole-job throughput of weak-scaling replicas: every rank processes
    units_per_rank per step, timed by the slowest rank."""
    return units_per_rank * world * steps / t_max_s


class ClockSampler:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
        except Exception:
            return None
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        mx = float(rows[0][2])
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for i, n in enumerate(names):
                if r[5 + i].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(rows)}


def grid_desc(g):
    return f"{g['n_r']}x{g['n_theta']}"


def run_reference(args, rank, world):
    """FP64 oracle on all host cores (its OpenMP-over-epochs build) at the
    headline grid: each step one bounded sample of (set, epoch) pairs of the
    workload."""
    if rank != 0:
        return
    import oracle
    from paper_2510_02639_gb300 import inputs as I
    params, t, desc = workload(args.workload)
    if args.law != "linear" and int(params[0]["n_lens"]) == 2:
        params = [dict(p, **I.SOURCE_LAWS[args.law]) for p in params]
        desc = dict(desc, law=args.law, law_params=I.SOURCE_LAWS[args.law])
    g = I.grid(**HEADLINE_GRID)
    rng = np.random.default_rng(7)
    n = args.ref_sample
    picks = [(int(rng.integers(len(params))), int(rng.integers(t.shape[1]))) for _ in range(n)]
    ps = [params[s] for s, _ in picks]
    tp = np.array([[t[s, e]] for s, e in picks])
    oracle.build_omp()
    cores = os.cpu_count() or 1

    def step():
        oracle.magnification_all_cores(ps, tp, g)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    val = n / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "magnifications/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(desc, grid=grid_desc(HEADLINE_GRID), n_limb=500),
            "cpu_baseline": {"value": val, "unit": "magnifications/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} random (set, epoch) pairs of the workload per step, OpenMP over "
                                       f"epochs on {cores} host cores"},
            "e2e": {"value": val, "unit": "magnifications/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(params, t, g, seconds=10.0):
    """The oracle as it stands on the host: one thread (random single epochs
    for ~seconds), and its OpenMP build on all cores (a fixed sample sized
    for about the same time)."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(11)
    n = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        s, e = int(rng.integers(len(params))), int(rng.integers(t.shape[1]))
        oracle.magnification([params[s]], [t[s, e]], g)
        n += 1
    dt = time.perf_counter() - t0
    one = n / dt
    cores = os.cpu_count() or 1
    m = max(cores, int(one * seconds * cores * 0.8))
    picks = [(int(rng.integers(len(params))), int(rng.integers(t.shape[1]))) for _ in range(m)]
    oracle.build_omp()
    t1 = time.perf_counter()
    oracle.magnification_all_cores([params[s] for s, _ in picks], np.array([[t[s, e]] for s, e in picks]), g)
    dt_all = time.perf_counter() - t1
    return {"value": m / dt_all, "unit": "magnifications/s", "cores": cores, "kind": "oracle",
            "sample": f"{m} random (set, epoch) pairs of the workload at {grid_desc(g)}, FP64, OpenMP over epochs "
                      f"on {cores} host cores, {dt_all:.1f} s",
            "single_core": {"value": one, "cores": 1,
                            "sample": f"{n} random (set, epoch) pairs, one thread, {dt:.1f} s"}}


def accuracy(icrs, I, g, dev):
    """Relative error of the GPU magnification at grid g on the 512-epoch
    qualification sample of the batch (tests/golden/batch_qualification.json:
    every set's peak epoch, random epochs, small sources at moderate
    magnification, sources inside a caustic) against the oracle's finest
    grid (4096 x 8192), whose own error is bounded by its last Richardson
    difference (4096 x 8192 against 2048 x 4096)."""
    import torch
    gold = json.load(open(GOLDEN))
    params, t = I.binary_batch()
    rows = gold["epochs"]
    ps = [params[r["set"]] for r in rows]
    tp = torch.tensor([[t[r["set"], r["epoch"]]] for r in rows], dtype=torch.float64, device=dev)
    ref = np.array([r["A"][-1] for r in rows])
    ref_err = np.abs(np.array([r["A"][-1] / r["A"][-2] - 1.0 for r in rows]))
    A, _ = icrs.magnification(icrs.params_to_device(ps, dev), tp, icrs.grid_from_dict(g, 2))
    e = np.abs(A.cpu().numpy().ravel() / ref - 1.0)
    cls = np.array([r["class"] for r in rows])
    fine = gold["grids"][-1]
    return {"max_rel_err": float(e.max()), "p99_rel_err": float(np.quantile(e, 0.99)),
            "median_rel_err": float(np.median(e)), "n": int(len(e)), "n_above_1e-4": int((e > 1e-4).sum()),
            "n_certified_1e-4": int(((e + ref_err) <= 1e-4).sum()),
            "max_rel_err_by_class": {c: float(e[cls == c].max()) for c in sorted(set(cls))},
            "reference_max_richardson_bound": float(ref_err.max()),
            "reference": f"FP64 oracle at {fine['n_r']}x{fine['n_theta']} (error bound: its difference from "
                         f"the previous doubling), tests/golden/batch_qualification.json"}


def accuracy_triple(icrs, I, g, dev):
    """Relative error of the GPU on the 32 triple-lens epochs of
    tests/golden/triple_qualification.json against the oracle at the finest
    grid (4096 x 8192) and, for parity, on the same grid."""
    import torch
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "triple_qualification.json")))
    params, t = I.triple_curve()
    rows = gold["epochs"]
    tp = torch.tensor([[t[0, r["epoch"]] for r in rows]], dtype=torch.float64, device=dev)
    A, _ = icrs.magnification(icrs.params_to_device(params, dev), tp, icrs.grid_from_dict(g, 3))
    A = A.cpu().numpy().ravel()
    ref = np.array([r["A"][-1] for r in rows])
    same = [r["A"][[(x["n_r"], x["n_theta"]) for x in gold["grids"]].index((g["n_r"], g["n_theta"]))]
            for r in rows] if any((x["n_r"], x["n_theta"]) == (g["n_r"], g["n_theta"]) for x in gold["grids"]) else None
    e = np.abs(A / ref - 1.0)
    out = {"max_rel_err": float(e.max()), "median_rel_err": float(np.median(e)), "n": int(len(e)),
           "reference_max_richardson_bound": float(np.max(np.abs([r["A"][-1] / r["A"][-2] - 1.0 for r in rows]))),
           "reference": "FP64 oracle at 4096x8192, tests/golden/triple_qualification.json"}
    if same is not None:
        out["max_rel_err_vs_oracle_same_grid"] = float(np.max(np.abs(A / np.array(same) - 1.0)))
    return out


def secondary_steps(args):
    """Timed and warm-up steps of the secondary lines (at most 3 each, so
    that a long headline run does not multiply their cost)."""
    return max(1, min(args.steps, 3)), max(1, min(args.warmup, 3))


def timed_steps(fn, steps, warmup, flush, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        fn()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def chi2_bench(icrs, I, args, dev, stream, flush, n_sets, grid=None):
    """Timed icrs_chi2_grad steps over the adjoint batch (first n_sets sets)."""
    import torch
    grid = grid or I.grid(**FIXED_GRID)
    params, t, centre, noise = I.adjoint_batch()
    params, t, noise = params[:n_sets], t[:n_sets], noise[:n_sets]
    g = icrs.grid_from_dict(grid, 2)
    pd = icrs.params_to_device(params, dev)
    tt = torch.tensor(t, dtype=torch.float64, device=dev)
    # data: magnification of the centre parameters plus Gaussian noise (F = A)
    Ac, _ = icrs.magnification(icrs.params_to_device([centre] * len(params), dev), tt, g)
    y = (Ac + torch.tensor(noise, device=dev)).contiguous()
    sig = torch.full_like(y, 0.01)
    out = {}

    def step():
        out["r"] = icrs.chi2_grad(pd, tt, g, y, sig, stream=stream)

    steps, warm = secondary_steps(args)
    ms = timed_steps(step, steps, warm, flush, stream)
    sec = float(np.sum(ms)) / 1e3
    grad = out["r"][1]
    return {"value": len(params) * steps / sec, "unit": "chi^2 gradients/s",
            "epochs_per_s": len(params) * t.shape[1] * steps / sec,
            "ms_per_step": sec / steps * 1e3, "steps": steps, "warmup": warm,
            "workload": f"adjoint_batch_{len(params)}x{t.shape[1]}", "grid": grid_desc(grid), "params": 8,
            "dtype": "f32", "finite": bool(torch.isfinite(grad).all().item()), "gpu_launches": steps}


def chi2_accuracy(icrs, I, dev, grid, n_epochs=12):
    """Largest error of icrs_chi2_grad against the oracle's FP64 forward mode
    (chi^2 gradient of one adjoint-batch set on n_epochs of its epochs),
    per parameter relative to the oracle's sum_e |dchi2_e/dp|."""
    import torch
    import oracle
    params, t, centre, noise = I.adjoint_batch(n_sets=1)
    idx = np.linspace(0, t.shape[1] - 1, n_epochs).astype(int)
    # epochs around the peak, where the finite source matters
    idx = np.clip(idx // 8 + t.shape[1] * 7 // 16, 0, t.shape[1] - 1)
    ts = np.ascontiguousarray(t[:, idx])
    Ao, dAo, _ = oracle.magnification_fwd(params, ts, grid)
    Ac, _ = oracle.magnification([centre], ts, grid)
    y = Ac + noise[:, idx]
    sig = np.full_like(y, 0.01)
    r = (y - Ao) / sig
    w = -2.0 * r / sig                                # dchi2/dA per epoch
    go = (w[0][:, None] * dAo[0]).sum(0)
    scale = (np.abs(w[0])[:, None] * np.abs(dAo[0])).sum(0)
    chi2, grad, A, st = icrs.chi2_grad(icrs.params_to_device(params, dev), torch.tensor(ts, device=dev),
                                       icrs.grid_from_dict(grid, 2), torch.tensor(y, device=dev),
                                       torch.tensor(sig, device=dev))
    g = grad.cpu().numpy()[0]
    return {"epochs": int(len(idx)), "max_rel_err_vs_oracle_fwd": float(np.max(np.abs(g - go) / scale)),
            "A_max_rel_err": float(np.max(np.abs(A.cpu().numpy() / Ao - 1.0))),
            "reference": f"oracle FP64 forward mode at {grid['n_r']}x{grid['n_theta']}; error of each component "
                         "over sum_e |dchi2_e/dp|"}


def nll_bench(icrs, I, args, dev, stream, flush, n_sets, grid):
    """Timed icrs_marginal_nll_grad steps (linear-flux marginalised likelihood
    and its gradient, one derivative launch plus one reduction) over the
    adjoint batch with F = (A - 1) F_S + F_base + noise, F_S = F_base = 1."""
    import torch
    params, t, centre, noise = I.adjoint_batch()
    params, t, noise = params[:n_sets], t[:n_sets], noise[:n_sets]
    g = icrs.grid_from_dict(grid, 2)
    pd = icrs.params_to_device(params, dev)
    tt = torch.tensor(t, dtype=torch.float64, device=dev)
    Ac, _ = icrs.magnification(icrs.params_to_device([centre] * len(params), dev), tt, g)
    F = (Ac + torch.tensor(noise, device=dev)).contiguous()
    sig = torch.full_like(F, 0.01)
    prior = torch.tensor([[1.0, 1.0, 0.25, 0.25]] * len(params), dtype=torch.float64, device=dev)
    ws = torch.empty(int(icrs.lib.icrs_marginal_nll_workspace_bytes(len(params), t.shape[1])), dtype=torch.uint8,
                     device=dev)
    out = {}

    def step():
        out["r"] = icrs.marginal_nll_grad(pd, tt, g, F, sig, prior, workspace=ws, stream=stream)

    steps, warm = secondary_steps(args)
    ms = timed_steps(step, steps, warm, flush, stream)
    sec = float(np.sum(ms)) / 1e3
    nll, grad, fl = out["r"][0], out["r"][1], out["r"][2]
    return {"value": len(params) * steps / sec, "unit": "marginal NLL gradients/s",
            "epochs_per_s": len(params) * t.shape[1] * steps / sec,
            "ms_per_step": sec / steps * 1e3, "steps": steps, "warmup": warm,
            "workload": f"adjoint_batch_{len(params)}x{t.shape[1]}",
            "grid": grid_desc(grid), "params": 8, "finite": bool(torch.isfinite(grad).all().item()),
            "flux_posterior_mean": [float(x) for x in fl.mean(0).tolist()], "gpu_launches": 2 * steps}


def surrogate_bench(args, dev):
    """Train, calibrate and score the gated surrogate at the headline grid."""
    import torch
    from paper_2510_02639_gb300 import icrs
    from paper_2510_02639_gb300 import inputs as I
    from paper_2510_02639_gb300 import surrogate as SG
    gd = I.grid(**HEADLINE_GRID)
    g = icrs.grid_from_dict(gd, 2)
    t0 = time.perf_counter()
    train = SG.make_dataset(args.sur_train_sets, 2000, seed=501, grid=gd)
    val = SG.make_dataset(max(1, args.sur_train_sets // 4), 2000, seed=502, grid=gd)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    sur = SG.Surrogate(seed=0)
    t1 = time.perf_counter()
    losses = sur.train(train, epochs=args.sur_epochs)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    gate = SG.calibrate(sur, val)
    c_ps = SG.calibrate_point_source(val)
    c_est, b_est = SG.calibrate_estimate(val)
    del train, val
    # scoring on unseen sets: plain ICRS (event-timed) against the gated path
    params, t = I.binary_batch(n_sets=args.sur_query_sets, n_epochs=2000, seed=503)
    pd = icrs.params_to_device(params, dev)
    tt = torch.tensor(t, dtype=torch.float64, device=dev)
    icrs.magnification(pd, tt[:, :10].contiguous(), g)  # warm-up launch
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    e[0].record()
    A_plain, st_plain = icrs.magnification(pd, tt, g)
    e[1].record()
    A_gate, k, idx = sur.gated_magnification(pd, tt, g, gate, return_index=True)
    e[2].record()
    torch.cuda.synchronize()
    feat, Aps, st = icrs.surrogate_features(pd, tt, g)
    n = A_gate.numel()
    Ap = A_plain.reshape(-1)
    err = (A_gate / Ap - 1.0).abs()
    routed = torch.zeros(n, dtype=torch.bool, device=dev)
    routed[idx.long()] = True
    # plain ICRS epochs that flag themselves (non-converged roots, illegal
    # image count, merged sectors, grid edge, NaN)
    flagged = (st_plain.reshape(-1) & 0x1F) != 0

    def err_stats(mask):
        em = torch.where(mask, err, torch.zeros_like(err))
        return {"n": int(mask.sum()), "max_rel_err": float(em.max()), "n_above_1e-4": int((em > 1e-4).sum())}
    ps_ok = (st == 0) & (feat[:, 6] >= c_ps)
    ps_err = torch.where(ps_ok, (Aps / Ap - 1.0).abs(), torch.zeros_like(err))
    est_ok = ((st == 0) & (feat[:, 6] >= c_est) & (feat[:, 7].abs() <= b_est)
              & (Aps <= torch.where(feat[:, 4] >= float(np.log10(gate.rho_min)) + 3.0, gate.A_max, gate.A_small)))
    Aest = Aps * torch.exp(feat[:, 7].double() / icrs.TARGET_SCALE)
    est_err = torch.where(est_ok, (Aest / Ap - 1.0).abs(), torch.zeros_like(err))
    t_plain, t_gate = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    # the non-learned preselection through the library (icrs_epoch_gate +
    # indexed ICRS), calibrated like the estimate rule, without and with an
    # n_ext = 2 extension along each light curve
    presel = {}
    for n_ext in (0, 2):
        ee = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ee[0].record()
        A_pre, k_pre = SG.preselected_magnification(pd, tt, g, c_est, b_est, n_ext=n_ext, mode=1,
                                                    A_max=gate.A_max, rho_min=gate.rho_min, A_small=gate.A_small)
        ee[1].record()
        torch.cuda.synchronize()
        t_pre = ee[0].elapsed_time(ee[1])
        err_pre = (A_pre / Ap - 1.0).abs()
        presel[f"n_ext_{n_ext}"] = {"speedup": t_plain / t_pre, "routed_frac": k_pre / n, "ms": t_pre,
                                    "max_rel_err": float(err_pre.max()),
                                    "n_above_1e-4": int((err_pre > 1e-4).sum())}
    return {"speedup": t_plain / t_gate, "queries": n, "routed_frac": k / n,
            "max_rel_err_vs_plain": float(err.max()),
            "vs_plain": {"accepted": err_stats(~routed), "routed_plain_unflagged": err_stats(routed & ~flagged),
                         "routed_plain_flagged": err_stats(routed & flagged),
                         "note": "accepted: surrogate vs ICRS at this grid (ICRS itself under-resolves a sector "
                                 "holding two images in adjacent theta bins); routed: the indexed ICRS launch vs "
                                 "the full launch (warm starts differ; flagged epochs merged sectors)"},
            "plain_ms": t_plain, "gated_ms": t_gate,
            "gated_magnifications_per_s": n / t_gate * 1e3, "grid": grid_desc(gd),
            "train_samples": int(args.sur_train_sets * 2000), "train_epochs": args.sur_epochs,
            "train_s": t_train, "data_s": t_data, "final_loss": losses[-1],
            "gate": {"sigma_max": gate.sigma_max, "mu_max": gate.mu_max, "b_max": gate.b_max,
                     "caustic_min": gate.caustic_min, "A_max": gate.A_max, "rho_min": gate.rho_min,
                     "A_small": gate.A_small},
            "point_source_only": {"accepted_frac": float(ps_ok.float().mean()), "caustic_min": c_ps,
                                  "max_rel_err": float(ps_err.max())},
            "second_order_estimate_only": {"accepted_frac": float(est_ok.float().mean()), "caustic_min": c_est,
                                           "b_max": b_est,
                                           "max_rel_err": float(est_err.max())},
            "preselection_gate": presel,
            "dtype": "bf16 weights / fp32 accumulate"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="icrs", choices=["icrs", "reference"])
    ap.add_argument("--workload", default="batch", choices=["batch", "caustic", "triple"])
    ap.add_argument("--law", default="linear", choices=["linear", "quadratic", "power4", "spot"],
                    help="source law of the headline and fixed-grid lines (binary workloads); the qualification "
                         "sample holds the linear law, so another law reports no accuracy")
    ap.add_argument("--ref-sample", type=int, default=64, help="oracle epochs per reference step (all host cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--chi2-sets", type=int, default=256, help="sets of the adjoint batch per chi^2 step (0: skip)")
    ap.add_argument("--chi2-sets-qualified", type=int, default=8,
                    help="sets of the adjoint batch per chi^2 step at the headline grid (0: skip)")
    ap.add_argument("--sur-train-sets", type=int, default=1000,
                    help="surrogate training sets x 2000 epochs (0: skip); 1000 = the configuration's 2M samples")
    ap.add_argument("--sur-query-sets", type=int, default=5000,
                    help="surrogate scoring sets x 2000 epochs; 5000 = the configuration's 10M queries")
    ap.add_argument("--sur-epochs", type=int, default=30)
    ap.add_argument("--clocks-csv", default="", help="where the nvidia-smi samples of the timed steps go "
                                                     "({rank} is replaced); default /tmp/clocks_rank{rank}.csv")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    from paper_2510_02639_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    from paper_2510_02639_gb300 import icrs
    from paper_2510_02639_gb300 import inputs as I

    params, t, desc = workload(args.workload, rank)
    n_lens = int(params[0]["n_lens"])
    if args.law != "linear":
        if n_lens != 2:
            raise SystemExit("--law applies to the binary workloads")
        params = [dict(p, **I.SOURCE_LAWS[args.law]) for p in params]
        desc = dict(desc, law=args.law, law_params=I.SOURCE_LAWS[args.law])
    g = I.grid(**HEADLINE_GRID)
    grid = icrs.grid_from_dict(g, n_lens)
    dev = torch.device("cuda", local)
    pd = icrs.params_to_device(params, dev)
    tt = torch.tensor(t, dtype=torch.float64, device=dev)
    S, E = tt.shape
    A = torch.empty((S, E), dtype=torch.float64, device=dev)
    st = torch.empty((S, E), dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        icrs.magnification(pd, tt, grid, out=A, status=st, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clk = ClockSampler(args.clocks_csv.format(rank=rank) if args.clocks_csv else f"/tmp/clocks_rank{rank}.csv")
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with clk:
        time.sleep(0.3)
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_local = float(np.sum(step_ms)) / 1e3
    t_max = reduce_max(t_local, world, dev)
    value = job_rate(S * E, world, args.steps, t_max)

    # rays evaluated (sector count in status bits 8..15)
    stc = st.cpu().numpy().astype(np.int64)
    n_sect = (stc >> 8) & 0xFF
    rays = float(n_sect.sum()) * g["n_r"] * g["n_theta"]
    flops = rays * FLOPS_PER_RAY[n_lens]
    kern_s = t_local / args.steps
    achieved = flops / kern_s / 1e12
    peak = fp32_peak_tflops()

    # end to end through the C ABI with host buffers (pinned), copies timed
    h_params = pd.cpu().pin_memory()
    h_t = tt.cpu().pin_memory()
    h_A = torch.empty((S, E), dtype=torch.float64).pin_memory()
    h_st = torch.empty((S, E), dtype=torch.int32).pin_memory()
    d_params = torch.empty_like(pd)
    d_t = torch.empty_like(tt)
    torch.cuda.synchronize()
    n_e2e = secondary_steps(args)[0]
    w0 = time.perf_counter()
    for _ in range(n_e2e):
        d_params.copy_(h_params, non_blocking=True)
        d_t.copy_(h_t, non_blocking=True)
        icrs.magnification(d_params, d_t, grid, out=A, status=st, stream=stream)
        h_A.copy_(A, non_blocking=True)
        h_st.copy_(st, non_blocking=True)
        torch.cuda.synchronize()
    w = reduce_max((time.perf_counter() - w0) / n_e2e, world, dev)
    e2e = {"value": job_rate(S * E, world, 1, w), "unit": "magnifications/s",
           "h2d_bytes_per_step": int(h_params.numel() + h_t.numel() * 8),
           "d2h_bytes_per_step": int(h_A.numel() * 8 + h_st.numel() * 4)}

    qualified = args.workload == "batch" and args.law == "linear"
    acc = accuracy(icrs, I, g, dev) if qualified else (
        accuracy_triple(icrs, I, g, dev) if args.workload == "triple" else None)

    # the fixed 64 x 256 grid (secondary)
    gf = I.grid(**FIXED_GRID)
    gridf = icrs.grid_from_dict(gf, n_lens)
    fs, fw = secondary_steps(args)
    msf = timed_steps(lambda: icrs.magnification(pd, tt, gridf, out=A, status=st, stream=stream), fs, fw, flush,
                      stream)
    fixed = {"grid": grid_desc(gf),
             "value": job_rate(S * E, world, fs, reduce_max(float(np.sum(msf)) / 1e3, world, dev)),
             "unit": "magnifications/s", "ms_per_step": float(np.mean(msf)),
             "accuracy": accuracy(icrs, I, gf, dev) if qualified else None}

    chi2 = chi2_bench(icrs, I, args, dev, stream, flush, args.chi2_sets) if args.chi2_sets > 0 else None
    chi2_q = None
    if args.chi2_sets_qualified > 0:
        gq = I.grid(**HEADLINE_GRID)
        chi2_q = chi2_bench(icrs, I, args, dev, stream, flush, args.chi2_sets_qualified, grid=gq)
        if rank == 0 and not args.no_cpu_baseline:
            chi2_q["accuracy"] = chi2_accuracy(icrs, I, dev, gq)
    nll = nll_bench(icrs, I, args, dev, stream, flush, args.chi2_sets, I.grid(**FIXED_GRID)) \
        if args.chi2_sets > 0 else None
    sur = surrogate_bench(args, dev) if (args.sur_train_sets > 0 and args.workload == "batch" and rank == 0) else None

    clocks = clk.summary() if rank == 0 else None
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(params, t, g)
    line = {
        "metric": METRIC, "value": value, "unit": "magnifications/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": dict(desc, grid=grid_desc(g), n_limb=g["n_limb"], l2="flushed (256 MiB write) between steps",
                       parallelism=f"replicas{world}" if world > 1 else "single"),
        "accuracy": acc,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "note": f"ray-stage algorithmic FP32 flops ({FLOPS_PER_RAY[n_lens]:.0f}/ray, {rays:.3e} rays/step) "
                             f"over the step's event time (binary: the linear instantiation does the work, the generic one skips "
                             f"every set of a linear batch); peak = 152 SM x 128 FP32 lanes x 2 x max SM clock "
                             f"(derived, no measured FP32 entry)"},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "fixed_grid": fixed,
        "chi2_grad": chi2,
        "chi2_grad_qualified_grid": chi2_q,
        "marginal_nll_grad": nll,
        "surrogate": sur,
        "clocks": clocks,
        # binary: the linear and the generic instantiation of the forward
        # kernel per step (each skips the other's sets); triple: one
        "gpu_launches": args.steps * (2 if n_lens == 2 else 1),
        "status_flags": {k: int(np.count_nonzero(stc & b)) for k, b in
                         [("nonconv", 1), ("imgcount", 2), ("sectcap", 4), ("edge", 8), ("nan", 16), ("overflow", 32)]},
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
