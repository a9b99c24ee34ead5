"""Benchmark: FDFD solves/s to relative residual 1e-6, data-driven vs plain GMRES.

Workload: 128x128 Yee grids (40 nm cells, 1550 nm, 10-cell PML, Gaussian line
source), 32 synthetic design trajectories x 16 steps = 512 permittivities.
The library solves the 448 training fields (28 trajectories) in complex128;
from them it fits k = 20 principal components and trains the subspace CNN
(k = 8 complex outputs) with its own kernels.  One timed step predicts the
subspaces of the 64 held-out problems (4 trajectories) with the CNN and solves
them with augmented GMRES(200) (complex64 Arnoldi inside FP64 refinement) to
true relative residual 1e-6; PCA-augmented and plain GMRES on the same 64
problems are timed alongside.

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

WORKLOAD = ("CNN-augmented GMRES(200), k=8 predicted vectors (network trained on the 448 training problems), "
            "64 held-out 128x128 FDFD solves to rel. residual 1e-6; PCA (k=20) and plain GMRES alongside")
METRIC = "FDFD solves/s to rel-residual 1e-6 on 1 GB300: CNN-augmented vs plain GMRES"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="c64", choices=["c64", "c128"])
    p.add_argument("--restart", type=int, default=200)
    p.add_argument("--k", type=int, default=20, help="PCA components")
    p.add_argument("--cnn-k", type=int, default=8)
    p.add_argument("--cnn-steps", type=int, default=800)
    p.add_argument("--cnn-batch", type=int, default=16)
    p.add_argument("--cnn-lr", type=float, default=3e-4)
    p.add_argument("--cnn-loss", default="residual", choices=["residual", "projection"],
                   help="Eq. 6 (unsupervised, trained on the right-hand sides) or Eq. 5 (solved fields)")
    p.add_argument("--cnn-base", default="pca", choices=["none", "pca"],
                   help="fixed offset of the CNN output: the leading principal components of the training fields")
    p.add_argument("--cnn-field", default="none", choices=["none", "background"],
                   help="extra CNN input: the field of the unpatterned background (one solve per grid)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-queue", action="store_true",
                   help="skip the solve-queue line (uneven grids, autotuned group width and lanes)")
    p.add_argument("--graphs", default="on", choices=["on", "off"],
                   help="run each restart cycle's Arnoldi steps as one CUDA graph launch")
    p.add_argument("--basis", default="f16", choices=["f32", "f16"],
                   help="storage of the Krylov basis (arithmetic stays FP32, the true residual FP64)")
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


# ------------------------------------------------------------------ ranks
def reduce_over_ranks(ms: float, solved: int, world: int, device=None):
    """Max of the timed region over ranks and the total solves of all ranks
    (torch.distributed; the identity on a single process)."""
    if world <= 1:
        return ms, solved
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    n = torch.tensor([solved], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(n.item()))


# ------------------------------------------------------------------ ours
def run_ours(args, rank, world):
    import torch
    import paper_1902_00090_gb300 as ddg

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    g, eps_train, eps_test = problem_set()
    src = (g.i_src, g.sigma_src, g.j_src)
    ctx = ddg.Context()
    ctx.set_graphs(args.graphs == "on")
    ctx.set_basis_storage(args.basis)

    def build(eps_set):
        ops = [ddg.fdfd_operator(g, torch.as_tensor(e, device=dev)) for e in eps_set]
        bs = [ddg.fdfd_source(op, *src) for op in ops]
        return ops, bs

    # --- training data: the library solves the 448 training fields in complex128
    t0 = time.time()
    ops_tr, bs_tr = build(eps_train)
    xs_tr, inf_tr, st = ddg.gmres_solve_batched(ctx, ops_tr, bs_tr, tol=1e-6, restart=200, maxit=5000,
                                                precision="c128")
    torch.cuda.synchronize()
    solve_train_s = time.time() - t0
    # --- PCA predictor (Sec. III): k leading components, fitted on the GPU
    t0 = time.time()
    U_pca, sig = ddg.pca_fit(ctx, torch.stack(xs_tr), args.k)
    torch.cuda.synchronize()
    pca_s = time.time() - t0
    # --- CNN predictor (Sec. III): trained on the same fields with the library's kernels
    t0 = time.time()
    field = None
    if args.cnn_field == "background":
        # the approximate-field input: one solve per grid, the design region
        # left unpatterned (slab in oxide)
        from paper_1902_00090_gb300 import inputs
        op_bg = ddg.fdfd_operator(g, torch.as_tensor(inputs.background_eps(g), device=dev))
        field, _, _ = ddg.gmres_solve(ctx, op_bg, ddg.fdfd_source(op_bg, *src), tol=1e-8, restart=200, maxit=20000,
                                      precision="c128")
    P = ddg.Predictor(k=args.cnn_k, input_field=field is not None)
    if field is not None:
        P.set_input_field(field, g.nx, g.ny)
    P.init_he(seed=0)
    if args.cnn_base == "pca":
        # the network learns corrections to the k leading principal components
        # (scaled to O(1) entries; zero head: training starts from that basis)
        U_base, _ = ddg.pca_fit(ctx, torch.stack(xs_tr), args.cnn_k)
        P.set_output_base(U_base, g.nx, g.ny, scale=float(np.sqrt(g.D)))
        P.zero_head()
    P.set_loss(args.cnn_loss)
    targets = bs_tr if args.cnn_loss == "residual" else xs_tr
    rng = np.random.default_rng(0)
    train_losses = []
    for it in range(args.cnn_steps):
        idx = rng.choice(len(ops_tr), args.cnn_batch, replace=False)
        train_losses.append(P.train_step([ops_tr[i] for i in idx], src, [targets[i] for i in idx], args.cnn_lr))
    torch.cuda.synchronize()
    cnn_s = time.time() - t0
    del xs_tr, ops_tr, bs_tr
    ops, bs = build(eps_test)
    n = len(ops)
    xs = [torch.zeros_like(b) for b in bs]
    U_cnn = [torch.empty((args.cnn_k, g.D), dtype=torch.complex128, device=dev) for _ in range(n)]

    def step_cnn():
        for x in xs:
            x.zero_()
        P.predict(ops, src, U=U_cnn)
        return ddg.augmented_gmres_solve_batched(ctx, ops, bs, U_cnn, x=xs, tol=1e-6, restart=args.restart,
                                                 maxit=5000, precision=args.precision)

    def step_pca():
        for x in xs:
            x.zero_()
        return ddg.augmented_gmres_solve_batched(ctx, ops, bs, [U_pca] * n, x=xs, tol=1e-6,
                                                 restart=args.restart, maxit=5000, precision=args.precision)

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
        l0 = ctx.launches + P.launches
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
        launches = ctx.launches + P.launches - l0
        prof = ctx.profile_read() if profile else None
        if profile:
            ctx.profile_enable(False)
        clk = sampler.stop() if sampler else None
        solved = K * int(sum(i["converged"] for i in infos))
        ms, solved = reduce_over_ranks(ms, solved, world, dev)
        return ms, infos, launches, prof, clk, solved

    def summary(infos):
        return {"iters_mean": float(np.mean([i["iters"] for i in infos])),
                "first_step_rel_residual_mean": float(np.nanmean([i["first_step_rel_residual"] for i in infos]))
                if any(i["first_step_rel_residual"] == i["first_step_rel_residual"] for i in infos) else None,
                "converged": int(sum(i["converged"] for i in infos)),
                "worst_true_rel_residual": float(max(i["true_rel_residual"] for i in infos))}

    K, W = args.steps, args.warmup
    ms, infos, launches, _, clk, solved = timed(step_cnn, K, W, clocks=True)
    value = solved / (ms / 1e3)
    # per-class kernel times: a second pass of the same step with CUDA events
    # around every launch (the events order the launches one after another, so
    # this pass runs a little slower than the one above)
    _, _, _, prof, _, _ = timed(step_cnn, K, 0, profile=True)
    # CNN inference alone (the predict call of one step)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    P.predict(ops, src, U=U_cnn)
    e1.record()
    torch.cuda.synchronize()
    predict_ms = e0.elapsed_time(e1)

    sK = max(1, K // 2)
    pms, pinf, _, _, _, psolved = timed(step_pca, sK, 1)
    pca = {"value": psolved / (pms / 1e3), "unit": "solves/s",
           "ms_per_step": pms / sK, "k": args.k, "fit_s": round(pca_s, 2), **summary(pinf)}
    plain = None
    plain_jacobi = None
    if not args.no_plain:
        qms, qinf, _, _, _, qsolved = timed(step_plain, sK, 1)
        plain = {"value": qsolved / (qms / 1e3), "unit": "solves/s",
                 "ms_per_step": qms / sK, **summary(qinf)}
        # the data-free baseline: plain GMRES with a Jacobi right preconditioner
        ctx.set_preconditioner("jacobi")
        jms, jinf, _, _, _, jsolved = timed(step_plain, 1, 0)
        ctx.set_preconditioner("none")
        plain_jacobi = {"value": jsolved / (jms / 1e3), "unit": "solves/s", "ms_per_step": jms, **summary(jinf)}

    # --- e2e: host buffers in, host buffers out, through the C ABI
    eps_host = torch.from_numpy(np.ascontiguousarray(eps_test)).pin_memory()
    x_host = torch.empty((n, g.D), dtype=torch.complex128).pin_memory()

    def step_e2e():
        eps_dev = eps_host.to(dev, non_blocking=True)
        o2 = [ddg.fdfd_operator(g, eps_dev[i]) for i in range(n)]
        b2 = [ddg.fdfd_source(op, *src) for op in o2]
        P.predict(o2, src, U=U_cnn)
        xs2, inf, st_ = ddg.augmented_gmres_solve_batched(ctx, o2, b2, U_cnn, tol=1e-6, restart=args.restart,
                                                          maxit=5000, precision=args.precision)
        x_host.copy_(torch.stack(xs2), non_blocking=True)
        return None, inf, st_

    eK = max(1, K // 2)
    ems, einf, _, _, _, esolved = timed(step_e2e, eK, 1)
    e2e = {"value": esolved / (ems / 1e3), "unit": "solves/s",
           "h2d_bytes_per_step": int(eps_host.numel() * 8), "d2h_bytes_per_step": int(x_host.numel() * 16)}

    # --- recycling along the design trajectories (the held-out set is 4
    # trajectories x 16 correlated steps): step t of every trajectory solved
    # together, with the CNN's vectors plus the previous step's solution as V
    n_traj = n // 16
    order = [[j * 16 + t for j in range(n_traj)] for t in range(16)]

    def step_recycle():
        P.predict(ops, src, U=U_cnn)
        prev = None
        infos = [None] * n
        for t, idx in enumerate(order):
            if prev is None:
                Us = [U_cnn[i] for i in idx]
            else:
                Us = [torch.cat([U_cnn[i], prev[j].reshape(1, -1)]) for j, i in enumerate(idx)]
            xr = [torch.zeros_like(bs[i]) for i in idx]
            xr, inf, st_ = ddg.augmented_gmres_solve_batched(ctx, [ops[i] for i in idx], [bs[i] for i in idx], Us,
                                                             x=xr, tol=1e-6, restart=args.restart, maxit=5000,
                                                             precision=args.precision)
            for j, i in enumerate(idx):
                infos[i] = inf[j]
            prev = xr
        return None, infos, 0

    rms, rinf, _, _, _, rsolved = timed(step_recycle, max(1, K // 2), 1)
    recycle = {"value": rsolved / (rms / 1e3), "unit": "solves/s", "ms_per_step": rms / max(1, K // 2),
               "batch": n_traj, "sequential_steps": 16, **summary(rinf)}

    # --- solve queue (secondary line; an error here is reported in the line and
    # does not cost the headline)
    queue = None
    if not args.no_queue:
        try:
            from paper_1902_00090_gb300 import autotune, inputs
            queue = queue_line(ddg, autotune, inputs, torch, dev, args)
        except Exception as e:  # noqa: BLE001
            queue = {"error": f"{type(e).__name__}: {e}"}

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
    # DRAM bytes over algorithmic bytes of the same kernels, from one ncu capture
    # per basis storage (dram__bytes_read.sum + dram__bytes_write.sum of one
    # launch at Arnoldi step 101, 64 solves of 128x128)
    ratio = ({"dots": 1.01, "update": 1.02} if args.basis == "f16" else {"dots": 1.01, "update": 1.03}).get(dom)
    roof = {"kernel": {"dots": "k_dots2", "update": "k_update2"}.get(dom, f"k_{dom}"), "bound": "hbm",
            "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "traffic": round(ratio * d_bytes / d_n) if ratio else None,
            "traffic_source": "ncu dram bytes / algorithmic bytes = %.2f for this kernel, times the mean "
                              "algorithmic bytes per launch" % ratio if ratio else None,
            "peak_source": peak_src, "timing": "CUDA events around every launch, profiled pass of the timed step",
            "launches": d_n, "avg_launch_us": round(d_ms * 1e3 / max(1, d_n), 2),
            "algorithmic_bytes_per_launch": round(d_bytes / max(1, d_n)),
            "share_of_kernel_time": round(d_ms / total_ms, 4),
            "classes": {c: {"ms": round(v[0], 2), "GBps": round(v[1] / max(v[0], 1e-9) / 1e6, 1),
                            "launches": v[2]} for c, v in prof.items()}}

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "solves/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": round(ms / K, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64+f64" if args.precision == "c64" else "c128",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": "128x128", "dx_nm": 40, "wavelength_nm": 1550,
                   "npml": 10, "restart": args.restart, "tol": 1e-6, "solves_per_step": n,
                   "predictor": f"cnn k={args.cnn_k} (6 levels, 32-128 channels, bf16, {args.cnn_loss} loss"
                                f"{', background-field input' if args.cnn_field == 'background' else ''}"
                                f"{', output offset = leading PCs of the training fields' if args.cnn_base == 'pca' else ''})",
                   "restart_policy": "augmented first cycle, then plain GMRES; V-only residual > 0.5 -> "
                                     "its step, then plain GMRES",
                   "precision": args.precision, "training_fields": len(eps_train),
                   "l2": "no flush: per-step working set (Krylov bases, 64 x 28 MB c64) exceeds L2",
                   "parallelism": f"replicas x{world}",
                   "step_loop": "CUDA graph per restart cycle" if args.graphs == "on" else "host-launched",
                   "krylov_basis_storage": {"f32": "FP32", "f16": "IEEE half (arithmetic FP32, true residual FP64)"}[
                       args.basis]},
        "cnn": {**summary(infos), "predict_ms_per_step": round(predict_ms, 2), "train_s": round(cnn_s, 2),
                "loss": "Eq. 6 (residual)" if args.cnn_loss == "residual" else "Eq. 5 (projection)",
                "train_steps": args.cnn_steps, "batch": args.cnn_batch, "lr": args.cnn_lr,
                "train_loss_first": float(np.mean(train_losses[:10])),
                "train_loss_last": float(np.mean(train_losses[-10:]))},
        "pca": pca,
        "plain": plain,
        "cnn_recycle": recycle,
        "plain_jacobi": plain_jacobi,
        "queue": queue,
        "speedup_vs_plain": round(value / plain["value"], 3) if plain else None,
        "pca_speedup_vs_plain": round(pca["value"] / plain["value"], 3) if plain else None,
        "solve_training_fields_s": round(solve_train_s, 2),
        "train_iters_mean": float(np.mean([i["iters"] for i in inf_tr])),
        "roofline": roof, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
    }
    return line


# ------------------------------------------------------------------ solve queue
def queue_line(ddg, autotune, inputs, torch, dev, args, restarts=(100, 200), widths=(32, 64)):
    """The batched-solves workload in small: 16 plain solves each of 128x128,
    192x192, 256x256 and 384x256 (one design trajectory per size), run through
    the solve queue with the group width, lane count and restart length (at
    most args.restart) chosen by the autotuner on the same 64 solves."""
    qops, qbs = [], []
    for t, (nx, ny) in enumerate([(128, 128), (192, 192), (256, 256), (384, 256)]):
        gq = inputs.grid_for(nx, ny)
        for e in inputs.trajectory_eps(gq, 4, t):
            qops.append(ddg.fdfd_operator(gq, torch.as_tensor(e, device=dev)))
            qbs.append(ddg.fdfd_source(qops[-1], gq.i_src, gq.sigma_src, gq.j_src))
    lanes = []
    for _ in range(2):
        c = ddg.Context()
        c.set_graphs(args.graphs == "on")
        c.set_basis_storage(args.basis)
        lanes.append(c)
    qkw = dict(tol=1e-6, maxit=20000, precision=args.precision)

    def run(ln, A, b, U, w, nl, tol, m, maxit, prec):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, infos, _ = ddg.gmres_solve_queue(ln[:nl], A, b, U=U, width=w, tol=tol, restart=m, maxit=maxit,
                                            precision=prec)
        torch.cuda.synchronize()
        return sum(1 for i in infos if i["converged"]) / (time.perf_counter() - t0)

    try:
        # warm-up: each lane's workspace at its largest group
        ddg.gmres_solve_queue(lanes[:1], qops, qbs, width=max(widths), restart=args.restart, **qkw)
        ddg.gmres_solve_queue(lanes, qops, qbs, width=min(widths), restart=args.restart, **qkw)
        tune = autotune.tune_queue(lanes, qops, qbs, sample=len(qops), widths=widths, lane_counts=(1, 2),
                                   restart=args.restart, restarts=restarts, basis=args.basis, run=run, **qkw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, qinf, _ = ddg.gmres_solve_queue(lanes[:tune["lanes"]], qops, qbs, width=tune["width"],
                                           restart=tune["restart"], **qkw)
        torch.cuda.synchronize()
        qdt = time.perf_counter() - t0
    finally:
        for c in lanes:
            c.close()
    single = [t[2] for t in tune["timings"] if t[0] == len(qops) and t[1] == 1 and t[3] == args.restart]
    return {"workload": f"{len(qops)} plain GMRES solves, 16 each of 128x128, 192x192, 256x256, 384x256 "
                        "(one design trajectory per size, queue in that order), c64 + FP64 refinement to 1e-6; "
                        f"restart autotuned <= {args.restart}",
            "value": round(sum(i["converged"] for i in qinf) / qdt, 2), "unit": "solves/s",
            "tuned": {"width": tune["width"], "lanes": tune["lanes"], "restart": tune["restart"]},
            "single_batch_value": round(single[0], 2) if single else None,
            "single_batch": f"one batch of {len(qops)}, GMRES({args.restart})",
            "tuning": [{"width": w, "lanes": l, "restart": m, "solves_per_s": round(v, 2)}
                       for w, l, v, m in tune["timings"]],
            "iters_mean": float(np.mean([i["iters"] for i in qinf])),
            "iters_max": int(max(i["iters"] for i in qinf)),
            "converged": int(sum(i["converged"] for i in qinf)),
            "worst_true_rel_residual": float(max(i["true_rel_residual"] for i in qinf))}


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
