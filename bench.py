"""Benchmark: limb-darkened binary-lens finite-source magnifications per second.

Workload (default): 64 binary-lens parameter sets x 10,000 epochs (log10 q ~
U[-5,-1], s log-uniform [0.3, 3], rho log-uniform [1e-4, 1e-2], u ~
U[0.3, 0.8], epochs uniform in [t0 - 2 tE, t0 + 2 tE]), 64 x 256 polar grid per
sector, 500 limb points.  One step = one call of icrs_magnification over the
whole batch (one fused kernel launch).  Inputs are resident in HBM; the L2 is
flushed (a 256 MiB write) between timed steps and each step is timed with CUDA
events on the launching stream.

The same line carries "chi2_grad": chi^2 gradient evaluations per second
(one unit = one parameter set's gradient over its 5,000-epoch light curve,
8 parameters) on the adjoint batch, 256 sets around s=0.9, q=1e-4,
rho=8e-4, each perturbed by 1%.  One call of icrs_chi2_grad does the whole
batch, timed like the magnification steps.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the baseline arm).

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

    def summary(self, gpu_index=0):
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


def run_reference(args, rank, world):
    """FP64 oracle on the host cores: each step one bounded sample (single thread)."""
    if rank != 0:
        return
    import oracle
    from paper_2510_02639_gb300 import inputs as I
    params, t, desc = workload(args.workload)
    g = I.grid()
    rng = np.random.default_rng(7)
    n = args.ref_sample
    picks = [(int(rng.integers(len(params))), int(rng.integers(t.shape[1]))) for _ in range(n)]
    oracle.build()

    def step():
        for s, e in picks:
            oracle.magnification([params[s]], [t[s, e]], g)

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
            "data": "synthetic", "config": dict(desc, grid="64x256", n_limb=500),
            "cpu_baseline": {"value": val, "unit": "magnifications/s", "cores": 1, "kind": "oracle",
                             "sample": f"{n} random (set, epoch) pairs of the workload per step"},
            "e2e": {"value": val, "unit": "magnifications/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(params, t, g, seconds=12.0):
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
    return {"value": n / dt, "unit": "magnifications/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} random (set, epoch) pairs of the workload, FP64 single thread, {dt:.1f} s"}


def chi2_bench(icrs, I, args, dev, stream, flush, n_sets):
    """Timed icrs_chi2_grad steps over the adjoint batch (first n_sets sets)."""
    import torch
    params, t, centre, noise = I.adjoint_batch()
    params, t, noise = params[:n_sets], t[:n_sets], noise[:n_sets]
    g = icrs.grid_from_dict(I.grid(), 2)
    pd = icrs.params_to_device(params, dev)
    tt = torch.tensor(t, dtype=torch.float64, device=dev)
    # data: magnification of the centre parameters plus Gaussian noise (F = A)
    Ac, _ = icrs.magnification(icrs.params_to_device([centre] * len(params), dev), tt, g)
    y = (Ac + torch.tensor(noise, device=dev)).contiguous()
    sig = torch.full_like(y, 0.01)
    for _ in range(args.warmup):
        icrs.chi2_grad(pd, tt, g, y, sig, stream=stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        chi2, grad, A, st = icrs.chi2_grad(pd, tt, g, y, sig, stream=stream)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    sec = float(np.sum([a.elapsed_time(b) for a, b in ev])) / 1e3
    ok = bool(torch.isfinite(grad).all().item())
    return {"value": len(params) * args.steps / sec, "unit": "chi^2 gradients/s",
            "epochs_per_s": len(params) * t.shape[1] * args.steps / sec,
            "ms_per_step": sec / args.steps * 1e3, "steps": args.steps, "warmup": args.warmup,
            "workload": f"adjoint_batch_{len(params)}x{t.shape[1]}", "params": 8, "dtype": "f32",
            "finite": ok, "gpu_launches": args.steps}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="icrs", choices=["icrs", "reference"])
    ap.add_argument("--workload", default="batch", choices=["batch", "caustic", "triple"])
    ap.add_argument("--ref-sample", type=int, default=400)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--chi2-sets", type=int, default=256, help="sets of the adjoint batch per chi^2 step (0: skip)")
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
    g = I.grid()
    grid = icrs.grid_from_dict(g, n_lens)
    dev = torch.device("cuda", local)
    pd = icrs.params_to_device(params, dev)
    tt = torch.tensor(t, dtype=torch.float64, device=dev)
    S, E = tt.shape
    A = torch.empty((S, E), dtype=torch.float64, device=dev)
    st = torch.empty((S, E), dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        icrs.magnification(pd, tt, grid, out=A, status=st, stream=stream)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clk = ClockSampler(os.path.join(ROOT, "gpurun_out", f"clocks_rank{rank}.csv") if os.path.isdir(
        os.path.join(ROOT, "gpurun_out")) else f"/tmp/clocks_rank{rank}.csv")
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with clk:
        time.sleep(0.3)
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            icrs.magnification(pd, tt, grid, out=A, status=st, stream=stream)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_local = float(np.sum(step_ms)) / 1e3
    t_max = t_local
    if world > 1:
        x = torch.tensor([t_local], device=dev)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t_max = float(x.item())
    units = S * E * world * args.steps
    value = units / t_max

    # rays evaluated (sector count in status bits 8..15)
    stc = st.cpu().numpy().astype(np.int64)
    n_sect = (stc >> 8) & 0xFF
    rays = float(n_sect.sum()) * g["n_r"] * g["n_theta"]
    flops = rays * FLOPS_PER_RAY[n_lens]
    kern_s = t_local / args.steps
    achieved = flops / kern_s / 1e12
    peak = fp32_peak_tflops()

    # end-to-end through the C ABI with host buffers (pinned), copies timed
    e2e = None
    if True:
        h_params = pd.cpu().pin_memory()
        h_t = tt.cpu().pin_memory()
        h_A = torch.empty((S, E), dtype=torch.float64).pin_memory()
        h_st = torch.empty((S, E), dtype=torch.int32).pin_memory()
        d_params = torch.empty_like(pd)
        d_t = torch.empty_like(tt)
        torch.cuda.synchronize()
        n_e2e = max(2, min(args.steps, 5))
        w0 = time.perf_counter()
        for _ in range(n_e2e):
            d_params.copy_(h_params, non_blocking=True)
            d_t.copy_(h_t, non_blocking=True)
            icrs.magnification(d_params, d_t, grid, out=A, status=st, stream=stream)
            h_A.copy_(A, non_blocking=True)
            h_st.copy_(st, non_blocking=True)
            torch.cuda.synchronize()
        w = (time.perf_counter() - w0) / n_e2e
        e2e = {"value": S * E * world / w, "unit": "magnifications/s",
               "h2d_bytes_per_step": int(h_params.numel() + h_t.numel() * 8),
               "d2h_bytes_per_step": int(h_A.numel() * 8 + h_st.numel() * 4)}

    chi2 = chi2_bench(icrs, I, args, dev, stream, flush, args.chi2_sets) if args.chi2_sets > 0 else None

    clocks = clk.summary() if rank == 0 else None
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world >= 1:
        cpu = cpu_baseline(params, t, g)
    line = {
        "metric": METRIC, "value": value, "unit": "magnifications/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": dict(desc, grid=f"{g['n_r']}x{g['n_theta']}", n_limb=g["n_limb"], l2="flushed (256 MiB write) between steps",
                       parallelism=f"replicas{world}" if world > 1 else "single"),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "note": f"ray-stage algorithmic FP32 flops ({FLOPS_PER_RAY[n_lens]:.0f}/ray, {rays:.3e} rays/step) "
                             f"over the fused kernel's event time; peak = 152 SM x 128 FP32 lanes x 2 x max SM clock"},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "chi2_grad": chi2,
        "clocks": clocks,
        "gpu_launches": args.steps,
        "status_flags": {k: int(np.count_nonzero(stc & b)) for k, b in
                         [("nonconv", 1), ("imgcount", 2), ("sectcap", 4), ("edge", 8), ("nan", 16), ("overflow", 32)]},
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
