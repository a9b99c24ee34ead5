"""Benchmark: FDFD solves/s to relative residual 1e-6, data-driven vs plain GMRES.

Workload (default): PCA-augmented GMRES(200) on 128x128 Yee grids (40 nm cells,
1550 nm, 10-cell PML, Gaussian line source), 32 synthetic design trajectories x
16 steps = 512 permittivities.  448 training fields (28 trajectories) are
solved by the library in complex128, their k = 20 leading principal components
are fitted on the GPU, and one timed step solves the 64 held-out problems
(4 trajectories) with augmented GMRES, complex64 Arnoldi inside FP64
refinement, to true relative residual 1e-6.  The plain-GMRES solves/s on the
same 64 problems is measured alongside.

`value` is the device-resident throughput (inputs in HBM, every kernel of the
solve timed); `e2e` repeats the step through the C ABI from host buffers
(permittivities uploaded, operators and sources built, solutions downloaded).
Under torchrun every rank solves its own copy of the batch (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = ("PCA-augmented GMRES(200), k=20 PCs of 448 training fields, "
            "64 held-out 128x128 FDFD solves to rel. residual 1e-6")
METRIC = "FDFD solves/s to rel-residual 1e-6 on 1 GB300: CNN-augmented vs plain GMRES"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="c64", choices=["c64", "c128"])
    p.add_argument("--restart", type=int, default=200)
    p.add_argument("--k", type=int, default=20)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    return p.parse_args()


# ------------------------------------------------------------------ problem set
def problem_set(k_train_traj=28, n_traj=32, steps=16):
    from paper_1902_00090_gb300 import inputs
    g = inputs.grid_128()
    eps = inputs.trajectory_set(g, 2, n_traj, steps)
    n_train = k_train_traj * steps
    return g, eps[:n_train], eps[n_train:]


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ ours
def run_ours(args, rank, world):
    import torch
    import paper_1902_00090_gb300 as ddg

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    g, eps_train, eps_test = problem_set()
    ctx = ddg.Context()

    def build(eps_set):
        ops = [ddg.fdfd_operator(g, torch.as_tensor(e, device=dev)) for e in eps_set]
        bs = [ddg.fdfd_source(op, g.i_src, g.sigma_src, g.j_src) for op in ops]
        return ops, bs

    # --- training: complex128 solves of the training fields, PCA on the GPU
    t0 = time.time()
    ops_tr, bs_tr = build(eps_train)
    xs_tr, inf_tr, st = ddg.gmres_solve_batched(ctx, ops_tr, bs_tr, tol=1e-6, restart=200, maxit=5000,
                                                precision="c128")
    F = torch.stack(xs_tr)
    U, sig = ddg.pca_fit(ctx, F, args.k)
    torch.cuda.synchronize()
    train_s = time.time() - t0
    del F, xs_tr, ops_tr, bs_tr
    ops, bs = build(eps_test)
    n = len(ops)
    Us = [U] * n
    xs = [torch.zeros_like(b) for b in bs]

    def step_aug():
        for x in xs:
            x.zero_()
        return ddg.augmented_gmres_solve_batched(ctx, ops, bs, Us, x=xs, tol=1e-6, restart=args.restart,
                                                 maxit=5000, precision=args.precision)

    def step_plain():
        for x in xs:
            x.zero_()
        return ddg.gmres_solve_batched(ctx, ops, bs, x=xs, tol=1e-6, restart=args.restart, maxit=5000,
                                       precision=args.precision)

    def timed(step, K, W, profile=False, clocks=False):
        for _ in range(W):
            step()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(dev.index) if clocks else None
        if sampler:
            sampler.start()
        if profile:
            ctx.profile_enable(True)
        l0 = ctx.launches
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push(f"timed_{step.__name__}")
        e0.record()
        infos = None
        for _ in range(K):
            _, infos, st_ = step()
        e1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        ms = e0.elapsed_time(e1)
        launches = ctx.launches - l0
        prof = ctx.profile_read() if profile else None
        if profile:
            ctx.profile_enable(False)
        clk = sampler.stop() if sampler else None
        if world > 1:
            t = torch.tensor([ms], device=dev, dtype=torch.float64)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms = float(t.item())
        return ms, infos, launches, prof, clk

    K, W = args.steps, args.warmup
    ms, infos, launches, prof, clk = timed(step_aug, K, W, profile=True, clocks=True)
    conv = sum(i["converged"] for i in infos)
    # per-solve accuracy check against the FP64 true residual the library reports
    worst = max(i["true_rel_residual"] for i in infos)
    value = world * conv * K / (ms / 1e3)

    plain = None
    if not args.no_plain:
        pK, pW = max(1, K // 2), 1
        pms, pinf, _, _, _ = timed(step_plain, pK, pW)
        pconv = sum(i["converged"] for i in pinf)
        plain = {"value": world * pconv * pK / (pms / 1e3), "unit": "solves/s", "ms_per_step": pms / pK,
                 "iters_mean": float(np.mean([i["iters"] for i in pinf])), "converged": pconv, "steps": pK}

    # --- e2e: host buffers in, host buffers out, through the C ABI
    eps_host = torch.from_numpy(np.ascontiguousarray(eps_test)).pin_memory()
    x_host = torch.empty((n, g.D), dtype=torch.complex128).pin_memory()

    def step_e2e():
        eps_dev = eps_host.to(dev, non_blocking=True)
        o2 = [ddg.fdfd_operator(g, eps_dev[i]) for i in range(n)]
        b2 = [ddg.fdfd_source(op, g.i_src, g.sigma_src, g.j_src) for op in o2]
        _, inf, st_ = ddg.augmented_gmres_solve_batched(ctx, o2, b2, Us, tol=1e-6, restart=args.restart,
                                                        maxit=5000, precision=args.precision)
        x_host.copy_(torch.stack(_), non_blocking=True)
        return None, inf, st_

    eK = max(1, K // 2)
    ems, einf, elaunch, _, _ = timed(step_e2e, eK, 1)
    econv = sum(i["converged"] for i in einf)
    e2e = {"value": world * econv * eK / (ems / 1e3), "unit": "solves/s",
           "h2d_bytes_per_step": int(eps_host.numel() * 8), "d2h_bytes_per_step": int(x_host.numel() * 16)}

    # --- roofline of the dominant kernel class (live CUDA events, algorithmic bytes)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    dom = max(("dots", "update", "step", "residual", "cycle_end"), key=lambda c: prof[c][0])
    d_ms, d_bytes, d_n = prof[dom]
    achieved = d_bytes / (d_ms / 1e3) / 1e9
    total_ms = sum(v[0] for v in prof.values())
    roof = {"kernel": f"k_{dom}", "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None, "peak_source": peak_src,
            "launches": d_n, "avg_launch_us": round(d_ms * 1e3 / max(1, d_n), 2),
            "share_of_kernel_time": round(d_ms / total_ms, 4),
            "classes": {c: {"ms": round(v[0], 2), "GBps": round(v[1] / max(v[0], 1e-9) / 1e6, 1),
                            "launches": v[2]} for c, v in prof.items()}}

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "solves/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": round(ms / K, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64+f64" if args.precision == "c64" else "c128",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": "128x128", "dx_nm": 40, "wavelength_nm": 1550,
                   "npml": 10, "k": args.k, "restart": args.restart, "tol": 1e-6, "solves_per_step": n,
                   "predictor": "pca", "precision": args.precision,
                   "l2": "no flush: per-step working set (Krylov bases, 64 x 26 MB c64) exceeds L2",
                   "parallelism": f"replicas x{world}"},
        "augmented": {"iters_mean": float(np.mean([i["iters"] for i in infos])),
                      "first_step_rel_residual_mean": float(np.mean([i["first_step_rel_residual"] for i in infos])),
                      "converged": conv, "worst_true_rel_residual": worst},
        "plain": plain,
        "speedup_vs_plain": round(value / plain["value"], 3) if plain else None,
        "train_s": round(train_s, 2), "train_iters_mean": float(np.mean([i["iters"] for i in inf_tr])),
        "pca_sigma_ratio_k": float(sig[-1] / sig[0]),
        "roofline": roof, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
    }
    return line


# ------------------------------------------------------------------ oracle (CPU)
def oracle_sample(n_train=24, k=20, seed_traj=28):
    """Bounded CPU sample: one held-out augmented solve with the oracle (setup untimed)."""
    import scipy.sparse.linalg as spla
    from oracle import fdfd, gmres, pca
    g, eps_train, eps_test = problem_set()
    b = fdfd.source_for(g)
    idx = np.linspace(0, len(eps_train) - 1, n_train).astype(int)
    F = np.column_stack([spla.spsolve(fdfd.operator_for(g, eps_train[i]).tocsc(), b) for i in idx])
    U, _ = pca.pca_basis(F, k)
    A = fdfd.operator_for(g, eps_test[0])
    return g, A, b, U


def cpu_baseline(args):
    g, A, b, U = oracle_sample(k=args.k)
    from oracle import gmres
    t0 = time.time()
    x, info = gmres.augmented_gmres(A, b, U, tol=1e-6, restart=args.restart, maxit=5000)
    dt = time.time() - t0
    return {"value": round((1.0 if info.converged else 0.0) / dt, 5), "unit": "solves/s",
            "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"1 held-out 128x128 solve, augmented GMRES({args.restart}) with k={args.k} PCs of 24 "
                      f"oracle-solved training fields, complex128 numpy/scipy ({info.iters} iterations, "
                      f"{dt:.1f} s); BLAS threads = library default"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    g, A, b, U = oracle_sample(k=args.k)
    from oracle import gmres
    for _ in range(args.warmup):
        gmres.augmented_gmres(A, b, U, tol=1e-6, restart=args.restart, maxit=5000)
    t0 = time.time()
    conv = 0
    for _ in range(args.steps):
        x, info = gmres.augmented_gmres(A, b, U, tol=1e-6, restart=args.restart, maxit=5000)
        conv += int(info.converged)
    dt = time.time() - t0
    v = conv / dt
    cb = {"value": round(v, 5), "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
          "sample": "each step: 1 held-out 128x128 augmented solve (k=20 PCs of 24 oracle-solved "
                    "training fields), complex128 numpy/scipy"}
    return {"impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": WORKLOAD, "grid": "128x128", "k": args.k,
                                              "restart": args.restart, "tol": 1e-6},
            "cpu_baseline": cb,
            "e2e": {"value": round(v, 5), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, rank, world)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
