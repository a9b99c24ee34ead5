"""Benchmark: FDFD solves/s to relative residual 1e-6 on one GB300, CNN-augmented
against plain GMRES, on the two-wavelength 256x256 design workload.

Workload (the default): 256x256 Yee grids (40 nm cells, 10-cell PML, line
source on column 20 with a Gaussian profile of 6 cells), every permittivity a
synthetic splitter-like device simulated at 1300 nm and at 1550 nm.  The
permittivities come from 272 design trajectories x 16 steps (trajectory t
seeded PCG64(3000 + t)): trajectories 0-253 (4064 permittivities, 8128
problems) train the predictors, trajectories 254-255 are the validation set
on which each variant's restart policy is chosen per wavelength, trajectories
256-271 (256 permittivities, 512 solves) are held out.

Set-up (not timed, the paper's convention): the library solves --n-pca
training problems per wavelength (plain GMRES(200), complex64 + FP64
refinement) and fits, per wavelength, the 20 leading principal components (the
PCA variant) and the k that offset the CNN's output; it then trains the
subspace CNN (k = 8 complex outputs, one network with the wavelength as an
input channel) with the residual loss (Eq. 6) on the 8128 training problems:
that loss needs only the right-hand sides, no solved fields.

One timed step = one held-out trajectory at both wavelengths (32 solves): CNN
prediction (orthonormalised on the device) into the subspace [PCA-20 of the
wavelength | CNN-8] and augmented GMRES(200) with the chosen restart policy,
complex64 Arnoldi with the basis stored in FP32 inside FP64 refinement, to true
relative residual 1e-6, iteration cap 5000.  Steps go round the 16 held-out
trajectories.  `value` counts converged solves per second with the inputs
resident in HBM; `e2e` runs the same step through fdfd_solve_host (host
permittivities in, host fields out, copies inside the call).  Plain and
PCA-augmented GMRES run one pass over the same 512 solves for the comparison.
Under torchrun every rank solves its own copy of the workload (weak scaling).

Other modes: --workload large1024 (1024x1024, 20 nm: 64 solves, CNN k = 16
against plain GMRES, and the FP32-only path to 1e-4) and --workload batched
(uneven grids 128x128 ... 384x256 through the solve queue: plain, PCA-20 and
CNN-8); --case solver|cnn are fixed-size runs for kernel profiling.
"""
from __future__ import annotations

import os

# the CPU oracle's BLAS uses every host core (set before numpy loads it)
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, str(os.cpu_count() or 1))

import argparse  # noqa: E402
import json  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import threading  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FDFD solves/s to rel-residual 1e-6 on 1 GB300: CNN-augmented vs plain GMRES"
WAVELENGTHS = (1300e-9, 1550e-9)
N_TRAIN_TRAJ, N_TEST_TRAJ, TRAJ_STEPS = 256, 16, 16
N_VAL_TRAJ = 2          # the last training trajectories, kept apart for choosing restart policies
# held-out trajectories per timed step: 2 x 16 permittivities x 2 wavelengths =
# 64 solves in one lock-step batch (a step of 32 leaves more of its time to
# the last few solves of its tail: 4.8 % fewer solves/s measured); 8 steps
# are one pass over the 512 held-out solves
TRAJ_PER_STEP = 2
N_STEPS_PASS = N_TEST_TRAJ // TRAJ_PER_STEP
POLICY_MARGIN = 0.03    # step saving a policy that keeps more columns must show to be chosen
SEED_CONFIG = 3          # trajectory t of this workload: PCG64(1000 * 3 + t)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="splitter256", choices=["splitter256", "large1024", "batched"])
    p.add_argument("--precision", default="c64", choices=["c64", "c128"])
    p.add_argument("--restart", type=int, default=200)
    p.add_argument("--maxit", type=int, default=5000)
    p.add_argument("--k", type=int, default=20, help="PCA components of the PCA variant")
    p.add_argument("--cnn-k", type=int, default=8)
    p.add_argument("--cnn-steps", type=int, default=1500)
    p.add_argument("--cnn-batch", type=int, default=16)
    p.add_argument("--cnn-lr", type=float, default=3e-4)
    p.add_argument("--n-pca", type=int, default=64, help="training problems solved per wavelength for the PCA bases")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--log-jsonl", default=None,
                   help="write one JSON line per solve of the headline workload's passes to this file")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-pca", action="store_true", help="skip the PCA variant's pass (profiling runs)")
    p.add_argument("--levers", action="store_true",
                   help="also measure the levers on the CNN's gain (restart policy, PCA + CNN, k, training size)")
    p.add_argument("--graphs", default="on", choices=["on", "off"],
                   help="run each batched solve's restart cycles as one CUDA graph launch")
    p.add_argument("--basis", default="f32", choices=["f32", "f16"],
                   help="storage of the Krylov basis (arithmetic stays FP32, the true residual FP64)")
    # fixed-size runs for kernel profiling (ncu) and quick timing; no JSON line
    p.add_argument("--case", default=None, choices=["solver", "cnn", "cnn-train", "stencil", "plain-steps"],
                   help="solver: --solves batched held-out problems with an iteration cap (every launch "
                        "sees the same basis sizes from run to run); cnn: the CNN forward of --solves problems")
    p.add_argument("--solves", type=int, default=64)
    p.add_argument("--n", type=int, default=128, help="grid side of --case runs")
    p.add_argument("--wavelength", type=float, default=1550e-9, help="--case runs")
    p.add_argument("--repeat", type=int, default=1)
    p.add_argument("--orth", default=None, choices=[None, "cgs2", "dcgs2"])
    p.add_argument("--profile", action="store_true", help="--case solver: per-kernel-class time and GB/s")
    p.add_argument("--tensor-cores", default="on", choices=["on", "off"])
    p.add_argument("--tma", default="on", choices=["on", "off"],
                   help="--case cnn|cnn-train: plain-input forward convolutions from TMA tiles")
    return p.parse_args()


# ------------------------------------------------------------------ fixed-size cases (profiling)
def case_problems(a):
    from paper_1902_00090_gb300 import inputs
    g = inputs.grid_for(a.n, a.n, wavelength=a.wavelength)
    cfg = 2 if a.n == 128 else SEED_CONFIG
    eps = inputs.trajectory_set(g, cfg, (a.solves + 15) // 16)[: a.solves]
    return g, eps


def case_solver(a):
    """Solves a.solves problems of the a.n x a.n trajectory set, batched, with
    an iteration cap.  Augmentation (a.k > 0) uses random vectors: the kernels'
    work does not depend on their quality."""
    import torch
    import paper_1902_00090_gb300 as ddg
    from paper_1902_00090_gb300 import inputs

    g, eps = case_problems(a)
    ops = [ddg.fdfd_operator(g, torch.as_tensor(e, device="cuda")) for e in eps]
    bs = [ddg.fdfd_source(op, g.i_src, g.sigma_src, g.j_src) for op in ops]
    ctx = ddg.Context(orthogonalization=a.orth)
    ctx.set_graphs(a.graphs == "on")
    ctx.set_basis_storage(a.basis)
    U = None
    if a.k > 0:
        U = torch.as_tensor(inputs.random_complex(g.D, 7, shape=(a.k, g.D)), device="cuda")
    for r in range(a.repeat):
        if a.profile and r == a.repeat - 1:
            ctx.profile_enable(True)
        torch.cuda.synchronize()
        t0 = time.time()
        if U is None:
            xs, infos, st = ddg.gmres_solve_batched(ctx, ops, bs, tol=1e-6, restart=a.restart, maxit=a.maxit,
                                                    precision=a.precision)
        else:
            xs, infos, st = ddg.augmented_gmres_solve_batched(ctx, ops, bs, [U] * len(ops), tol=1e-6,
                                                              restart=a.restart, maxit=a.maxit,
                                                              precision=a.precision)
        torch.cuda.synchronize()
        dt = time.time() - t0
        print(f"run {r}: {len(ops)} solves, {dt * 1e3:.1f} ms, iters mean "
              f"{np.mean([i['iters'] for i in infos]):.1f}, status {st}, launches {ctx.launches}")
    if a.profile:
        for name, (ms, by, n) in ctx.profile_read().items():
            if n:
                print(f"  {name:10s} {n:6d} launches {ms:9.2f} ms  {by / max(ms, 1e-9) / 1e6:8.1f} GB/s "
                      f" {ms * 1e3 / n:8.1f} us/launch")


def case_stencil(a):
    """The standalone operator application (fdfd_apply_c64 and fdfd_apply) on
    one a.n x a.n problem: a.repeat applications between CUDA events, GB/s of
    algorithmic bytes (x read, eps read, y written: 20 B per cell in complex64,
    40 B in complex128) against the measured copy bandwidth."""
    import torch
    import paper_1902_00090_gb300 as ddg
    from paper_1902_00090_gb300 import inputs

    g = inputs.grid_for(a.n, a.n, wavelength=a.wavelength)
    eps = inputs.trajectory_eps(g, SEED_CONFIG, 0, 1)[0]
    op = ddg.fdfd_operator(g, torch.as_tensor(eps, device="cuda"))
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs") \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else None
    for name, dt, fn, per_cell in (("c64", torch.complex64, ddg.fdfd_apply_c64, 20),
                                   ("c128", torch.complex128, ddg.fdfd_apply, 40)):
        x = torch.randn(g.D, dtype=dt, device="cuda")
        y = torch.empty_like(x)
        for _ in range(3):
            fn(op, x, y)
        _, ms = timed_call(torch, lambda: [fn(op, x, y) for _ in range(a.repeat)])
        gbs = per_cell * g.D * a.repeat / (ms / 1e3) / 1e9
        print(f"{name}: {a.n}x{a.n}, {ms * 1e3 / a.repeat:.1f} us per apply, {gbs:.0f} GB/s"
              + (f" = {gbs / peak:.3f} of the measured {peak:.0f} GB/s" if peak else ""))


def case_plain_steps(a):
    """Plain GMRES(200) step counts on the GPU (complex128 and complex64 +
    refinement, cap 20000) for the problems of the oracle's report
    (`python -m oracle.iterations_report --workload splitter256 --count 4`):
    permittivities 0 and 1 of held-out trajectory 256, at 1300 and 1550 nm."""
    import torch
    import paper_1902_00090_gb300 as ddg

    ctx = ddg.Context()
    rows = []
    for j in range(a.solves):
        g = splitter_grids()[j % 2]
        e = trajectory(N_TRAIN_TRAJ)[j // 2]
        op = ddg.fdfd_operator(g, torch.as_tensor(e, device="cuda"))
        b = ddg.fdfd_source(op, g.i_src, g.sigma_src, g.j_src)
        row = {"j": j, "problem": f"256x256 {int(round(g.wavelength * 1e9))} nm, step {j // 2}"}
        for prec in ("c128", "c64"):
            _, info, _ = ddg.gmres_solve(ctx, op, b, tol=1e-6, restart=200, maxit=20000, precision=prec)
            row[prec] = {"iters": info["iters"], "cycles": info["cycles"],
                         "true_rel_residual": info["true_rel_residual"]}
        rows.append(row)
        print(json.dumps(row), flush=True)


def case_cnn_train(a):
    """a.repeat residual-loss training steps of the default network (k =
    a.cnn_k) on a.solves problems of a.n x a.n, with the forward and backward
    convolutions on tcgen05 (--tensor-cores off: CUDA cores)."""
    import torch
    import paper_1902_00090_gb300 as ddg

    g, eps = case_problems(a)
    ops = [ddg.fdfd_operator(g, torch.as_tensor(e, device="cuda")) for e in eps]
    b = ddg.fdfd_source(ops[0], g.i_src, g.sigma_src, g.j_src)
    P = ddg.Predictor(k=a.cnn_k)
    P.init_he(seed=0)
    P.set_loss("residual")
    on = a.tensor_cores == "on"
    P.set_tensor_cores(on, backward=on, tma=a.tma == "on")
    src = (g.i_src, g.sigma_src, g.j_src)
    for r in range(a.repeat):
        torch.cuda.synchronize()
        t0 = time.time()
        loss = P.train_step(ops, src, [b] * len(ops), a.cnn_lr)
        torch.cuda.synchronize()
        print(f"step {r}: {a.solves} problems, {(time.time() - t0) * 1e3:.2f} ms, loss {loss:.5f}, "
              f"launches {P.launches}")


def case_cnn(a):
    """Predicts the subspaces of a.solves a.n x a.n problems with the default
    network (He-initialised weights: the kernels' work does not depend on them)."""
    import torch
    import paper_1902_00090_gb300 as ddg

    g, eps = case_problems(a)
    ops = [ddg.fdfd_operator(g, torch.as_tensor(e, device="cuda")) for e in eps]
    P = ddg.Predictor(k=a.cnn_k)
    P.init_he(seed=0)
    P.set_tensor_cores(a.tensor_cores == "on", tma=a.tma == "on")
    src = (g.i_src, g.sigma_src, g.j_src)
    U = [torch.empty((a.cnn_k, g.D), dtype=torch.complex128, device="cuda") for _ in ops]
    for r in range(a.repeat):
        torch.cuda.synchronize()
        t0 = time.time()
        P.predict(ops, src, U=U)
        torch.cuda.synchronize()
        print(f"run {r}: {a.solves} predictions, {(time.time() - t0) * 1e3:.2f} ms, launches {P.launches}")


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


# ------------------------------------------------------------------ workload
def splitter_grids():
    from paper_1902_00090_gb300 import inputs
    return [inputs.grid_for(256, 256, wavelength=lam) for lam in WAVELENGTHS]


def step_traj(st: int):
    """Held-out trajectories (offsets from the first held-out one) of timed step st."""
    return [TRAJ_PER_STEP * st + j for j in range(TRAJ_PER_STEP)]


def trajectory(t: int):
    """Permittivities of design trajectory t (16, 256, 256); the grid's
    wavelength does not enter the permittivity."""
    from paper_1902_00090_gb300 import inputs
    return inputs.trajectory_eps(splitter_grids()[0], SEED_CONFIG, t, TRAJ_STEPS)


def choose_policy(table, lam, margin=POLICY_MARGIN):
    """From [((cycles, keep), {wavelength: mean steps}), ...], the restart
    policy for `lam`: candidates in order of the columns they keep after the
    first cycle (then of the cycles with all of V); a later one replaces the
    choice only with fewer than (1 - margin) x the chosen one's steps."""
    order = sorted(table, key=lambda t: (t[0][1], t[0][0]))
    best, steps = order[0][0], order[0][1][lam]
    for cand, sc in order[1:]:
        if sc[lam] < (1.0 - margin) * steps:
            best, steps = cand, sc[lam]
    return best


def summarize(infos, wl_of=None):
    """Iterations, convergence and residuals of a list of solve infos; with
    wl_of (solve index -> wavelength in nm) also per wavelength."""
    def one(ii):
        its = [i["iters"] for i in ii]
        res = [i["true_rel_residual"] for i in ii]
        miss = [r for i, r in zip(ii, res) if not i["converged"]]
        fs = [i["first_step_rel_residual"] for i in ii if i["first_step_rel_residual"] == i["first_step_rel_residual"]]
        d = {"solves": len(ii), "converged": int(sum(i["converged"] for i in ii)),
             "iters_mean": round(float(np.mean(its)), 1), "iters_max": int(max(its)),
             "worst_true_rel_residual": float(max(res))}
        if fs:
            d["first_step_rel_residual_mean"] = round(float(np.mean(fs)), 5)
        if miss:
            d["not_converged_residual_median"] = float(np.median(miss))
        return d
    out = one(infos)
    if wl_of is not None:
        for wl in sorted(set(wl_of)):
            out[f"{wl}nm"] = one([i for i, w in zip(infos, wl_of) if w == wl])
    return out


def headline_config(args, world):
    """The `config` object of the headline workload (both arms print it)."""
    n_step = len(WAVELENGTHS) * TRAJ_PER_STEP * TRAJ_STEPS
    return {
        "workload": "splitter256: CNN-augmented GMRES(200) (subspace [PCA-20 | CNN-8], one network for both "
                    "wavelengths, residual-loss training on 8128 problems), 256x256 Yee grid at 40 nm, 1300 and "
                    "1550 nm, 512 held-out solves (16 trajectories x 16 steps x 2 wavelengths) to rel. residual "
                    "1e-6, cap 5000; plain and PCA-20 GMRES alongside",
        "grid": "256x256", "dx_nm": 40, "wavelengths_nm": [1300, 1550], "npml": 10,
        "restart": args.restart, "tol": 1e-6, "maxit": args.maxit, "solves_per_step": n_step,
        "step": f"{TRAJ_PER_STEP} held-out trajectories ({TRAJ_PER_STEP * TRAJ_STEPS} permittivities) at both "
                f"wavelengths, one batched solve; steps go round the {N_TEST_TRAJ} held-out trajectories "
                f"({N_STEPS_PASS} steps per pass)",
        "predictor": f"cnn k={args.cnn_k} (6 levels, 32-128 channels, bf16 weights and activations, FP32 "
                     "accumulation; inputs eps, wavelength, PML mask, source; output offset = the k leading PCs "
                     "of the solved training fields of each wavelength; output orthonormalised on the device)",
        "restart_policy": "per wavelength, chosen on two validation trajectories (fewest steps; a policy keeping "
                          "more columns must save 3 %) among: all 28 vectors in the first cycle then plain GMRES "
                          "/ then the PCA-20 columns kept / all kept (cnn.policy); V-only residual > 0.5 -> its "
                          "step, then plain",
        "precision": "complex64 Arnoldi and matvecs, FP64 true residual, Givens, least squares and x (refinement "
                     "every restart)" if args.precision == "c64" else "complex128",
        "krylov_basis_storage": {"f32": "FP32 (complex64)",
                                 "f16": "IEEE half (arithmetic FP32, true residual FP64)"}[args.basis],
        "training_problems": 2 * (N_TRAIN_TRAJ - N_VAL_TRAJ) * TRAJ_STEPS,
        "validation_problems": 2 * N_VAL_TRAJ * TRAJ_STEPS,
        "l2": f"no flush: the per-step working set ({n_step} Krylov bases of 105 MB) exceeds the 129 MB L2",
        "parallelism": f"replicas x{world}",
        "solve_loop": ("one CUDA graph launch per batched solve (restart cycles and Arnoldi steps under "
                       "device-side WHILE/IF nodes)") if args.graphs == "on" else "host-launched",
    }


def solve_records(variant, step_infos, per_step_ms, grids):
    """One dict per solve of the timed steps `step_infos` ([(step, infos)],
    infos in the step's order: wavelength, then trajectory, then permittivity)
    of the two-wavelength workload: which problem it was (held-out trajectory,
    permittivity, wavelength, the trajectory's seed), what the solve reported,
    and its step's wall time (the solves of a step share every launch)."""
    n_traj = TRAJ_PER_STEP * TRAJ_STEPS
    out = []
    for q, (st, infos) in enumerate(step_infos):
        for i, inf in enumerate(infos):
            w, rem = divmod(i, n_traj)
            t = N_TRAIN_TRAJ + step_traj(st)[rem // TRAJ_STEPS]
            g = grids[w]
            out.append({"workload": "splitter256", "variant": variant, "timed_step": q, "step": st,
                        "trajectory": t, "seed": f"PCG64({1000 * SEED_CONFIG + t})",
                        "permittivity": rem % TRAJ_STEPS, "wavelength_nm": int(round(g.wavelength * 1e9)),
                        "grid": f"{g.nx}x{g.ny}", "iterations": int(inf["iters"]),
                        "restart_cycles": int(inf["cycles"]), "converged": bool(inf["converged"]),
                        "true_rel_residual": float(inf["true_rel_residual"]),
                        "first_step_rel_residual": float(inf["first_step_rel_residual"]),
                        "fallback_used": bool(inf["fallback_used"]), "breakdown": bool(inf["breakdown"]),
                        "step_ms": round(float(per_step_ms[q]), 3), "solves_in_step": len(infos)})
    return out


def run_ours(args, rank, world):
    import torch
    import paper_1902_00090_gb300 as ddg

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    grids = splitter_grids()
    g0 = grids[0]
    src = (g0.i_src, g0.sigma_src, g0.j_src)
    D = g0.D
    ctx = ddg.Context()
    ctx.set_graphs(args.graphs == "on")
    ctx.set_basis_storage(args.basis)
    kw = dict(tol=1e-6, restart=args.restart, maxit=args.maxit, precision=args.precision)

    # --- problems: every permittivity at both wavelengths, operators resident
    t0 = time.time()
    train_ops = {lam: [] for lam in WAVELENGTHS}
    for t in range(N_TRAIN_TRAJ):
        for e in trajectory(t):
            ed = torch.as_tensor(e, device=dev)
            for g in grids:
                train_ops[g.wavelength].append(ddg.fdfd_operator(g, ed))
    test_eps = [trajectory(N_TRAIN_TRAJ + t) for t in range(N_TEST_TRAJ)]
    test_ops, test_b, test_wl = [], [], []
    for st in range(N_STEPS_PASS):    # step st: trajectories step_traj(st) at both wavelengths (64 solves)
        ops_t = [ddg.fdfd_operator(g, torch.as_tensor(e, device=dev))
                 for g in grids for t in step_traj(st) for e in test_eps[t]]
        test_ops.append(ops_t)
        test_b.append([ddg.fdfd_source(op, *src) for op in ops_t])
        test_wl.append([int(round(g.wavelength * 1e9)) for g in grids for t in step_traj(st) for _ in test_eps[t]])
    b_of = {lam: ddg.fdfd_source(train_ops[lam][0], *src) for lam in WAVELENGTHS}
    setup_s = time.time() - t0

    # the last N_VAL_TRAJ training trajectories are kept apart for choosing
    # the restart policies (neither the PCA fit nor the CNN's training sees
    # them); a validation step holds TRAJ_PER_STEP of them at both
    # wavelengths, in the order of a timed step
    n_val = N_VAL_TRAJ * TRAJ_STEPS
    val_steps = []
    for v0 in range(0, N_VAL_TRAJ, TRAJ_PER_STEP):
        lo = len(train_ops[WAVELENGTHS[0]]) - n_val + v0 * TRAJ_STEPS
        n_v = TRAJ_PER_STEP * TRAJ_STEPS
        ops_v = [op for lam in WAVELENGTHS for op in train_ops[lam][lo:lo + n_v]]
        val_steps.append((ops_v, [b_of[lam] for lam in WAVELENGTHS for _ in range(n_v)]))
    for lam in WAVELENGTHS:
        del train_ops[lam][-n_val:]

    # --- PCA bases per wavelength from solved training problems (evenly spread
    # over the training trajectories), the library's own solves
    t0 = time.time()
    U_pca, U_base, pca_info = {}, {}, {}
    n_tr = len(train_ops[WAVELENGTHS[0]])
    pick = np.linspace(0, n_tr - 1, args.n_pca).astype(int)
    for lam in WAVELENGTHS:
        ops_p = [train_ops[lam][i] for i in pick]
        xs, inf, _ = ddg.gmres_solve_batched(ctx, ops_p, [b_of[lam]] * len(ops_p), tol=1e-6, restart=200,
                                             maxit=20000, precision="c64")
        F = torch.stack(xs)
        U_pca[lam], _ = ddg.pca_fit(ctx, F, args.k)
        U_base[lam], sig = ddg.pca_fit(ctx, F, args.cnn_k)
        pca_info[f"{int(round(lam * 1e9))}nm"] = summarize(inf)
        del F, xs
    torch.cuda.synchronize()
    pca_s = time.time() - t0

    # --- CNN predictor (Sec. III): one network for both wavelengths, trained
    # with the residual loss (Eq. 6) on all 8192 training problems
    t0 = time.time()
    P = train_cnn(ddg, args, grids, train_ops, b_of, U_base, src, D)
    torch.cuda.synchronize()
    cnn_s = time.time() - t0
    train_losses = P.train_losses
    # levers (--levers): a k = 16 network (its offset: the 16 leading PCs of
    # each wavelength) and the k = 8 network trained on a quarter of the
    # training problems, with the same steps, batch and learning rate
    P16 = Pq = None
    if args.levers:
        n_all = sum(len(v) for v in train_ops.values())
        P16 = train_cnn(ddg, args, grids, train_ops, b_of, U_pca, src, D, k=16)
        Pq = train_cnn(ddg, args, grids, train_ops, b_of, U_base, src, D, n_problems=n_all // 4)
        Pq.n_problems = n_all // 4
    del train_ops

    n_step = len(test_ops[0])
    step_lams = [g.wavelength for g in grids for _ in range(n_step // len(grids))]
    xs = [torch.zeros(D, dtype=torch.complex128, device=dev) for _ in range(n_step)]
    # the headline's subspace per solve: [PCA-20 of its wavelength | CNN-8]
    # (the PCA rows are fixed, the CNN writes the rest each step)
    kc = args.k + args.cnn_k
    U_comb = [torch.empty((kc, D), dtype=torch.complex128, device=dev) for _ in range(n_step)]
    for u, lam in zip(U_comb, step_lams):
        u[:args.k].copy_(U_pca[lam])
    U_cnn_rows = [u[args.k:] for u in U_comb]
    U_cnn = [torch.empty((args.cnn_k, D), dtype=torch.complex128, device=dev) for _ in range(n_step)]
    U_pca_step = [U_pca[lam] for lam in step_lams]

    def solve_cnn(ops, bs):
        for x in xs:
            x.zero_()
        P.predict(ops, src, U=U_cnn_rows)
        return ddg.augmented_gmres_solve_batched(ctx, ops, bs, U_comb, x=xs, **kw)

    def solve_cnn8(ops, bs):
        for x in xs:
            x.zero_()
        P.predict(ops, src, U=U_cnn)
        return ddg.augmented_gmres_solve_batched(ctx, ops, bs, U_cnn, x=xs, **kw)

    def solve_pca(ops, bs):
        for x in xs:
            x.zero_()
        return ddg.augmented_gmres_solve_batched(ctx, ops, bs, U_pca_step, x=xs, **kw)

    def solve_plain(ops, bs):
        for x in xs:
            x.zero_()
        return ddg.gmres_solve_batched(ctx, ops, bs, x=xs, **kw)

    def set_policy(pol):
        for lam, (cyc, keep) in pol.items():
            ctx.set_augmented_policy(cyc, keep, wavelength=lam)

    def tune_policy(solve, candidates):
        """Per wavelength, the restart policy (cycles with all of V, then the
        leading `keep` columns) chosen on the validation trajectories by mean
        Krylov steps (a solve that misses the cap counts twice the cap).
        Candidates are taken in order of the columns they keep after the first
        cycle; one that keeps more replaces the choice only when it saves more
        than POLICY_MARGIN of the steps, since every kept column adds its bytes
        to every later Arnoldi step and the kept CNN vectors, nearly inside the
        PCA span, gained on one validation trajectory and lost on the held-out
        set.  (Charging the kept columns' bytes in full chose the first-cycle
        policy at 1300 nm, whose held-out solves then missed the cap more
        often: fewer steps with margin is the safer criterion.)"""
        table = []
        for cand in candidates:
            set_policy({lam: cand for lam in WAVELENGTHS})
            its = {lam: [] for lam in WAVELENGTHS}
            for ops_v, b_v in val_steps:
                _, inf, _ = solve(ops_v, b_v)
                for i, l2 in zip(inf, step_lams):
                    its[l2].append(i["iters"] if i["converged"] else 2 * args.maxit)
            table.append((cand, {lam: float(np.mean(its[lam])) for lam in WAVELENGTHS}))
        best = {lam: choose_policy(table, lam) for lam in WAVELENGTHS}
        report = {f"{int(round(lam * 1e9))}nm": {"chosen": {"cycles": best[lam][0], "keep": best[lam][1]},
                                                 "steps": {f"{c[0]}/{c[1]}": round(v[lam], 1) for c, v in table}}
                  for lam in WAVELENGTHS}
        return best, report

    t0 = time.time()
    every = 10**6
    pol_cnn, rep_cnn = tune_policy(solve_cnn, [(1, 0), (1, 8), (1, args.k), (every, kc)])
    pol_pca, rep_pca = tune_policy(solve_pca, [(1, 0), (1, 8), (every, args.k)])
    tune_s = time.time() - t0

    def step_cnn(t):
        return solve_cnn(test_ops[t], test_b[t])

    def step_pca(t):
        return solve_pca(test_ops[t], test_b[t])

    def step_plain(t):
        return solve_plain(test_ops[t], test_b[t])

    def timed(step, K, W, start=0, profile=False, clocks=False):
        """W untimed then K timed steps start, start+1, ... (mod N_STEPS_PASS, each
        TRAJ_PER_STEP held-out trajectories); CUDA events around the whole
        region and around each step."""
        seq = [(start + q) % N_STEPS_PASS for q in range(W + K)]
        for q in range(W):
            step(seq[q])
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(dev.index) if clocks else None
        if sampler:
            sampler.start()
        if profile:
            ctx.profile_enable(True)
        l0 = ctx.launches + P.launches
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
        infos, per_step = [], []
        torch.cuda.nvtx.range_push(f"timed_{step.__name__}")   # ncu --nvtx-include selects these launches
        ev[0].record()
        for q in range(K):
            _, inf, _ = step(seq[W + q])
            ev[q + 1].record()
            infos.append((seq[W + q], inf))
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        ms = ev[0].elapsed_time(ev[K])
        per_step = [ev[q].elapsed_time(ev[q + 1]) for q in range(K)]
        launches = ctx.launches + P.launches - l0
        prof = ctx.profile_read() if profile else None
        if profile:
            ctx.profile_enable(False)
        clk = sampler.stop() if sampler else None
        solved = int(sum(i["converged"] for _, inf in infos for i in inf))
        ms_all, solved_all = reduce_over_ranks(ms, solved, world, dev)
        return dict(ms=ms_all, solved=solved_all, infos=infos, per_step=per_step, launches=launches, prof=prof,
                    clocks=clk)

    def pass_of(r):
        """The first N_STEPS_PASS timed steps of r (every held-out trajectory
        once: the 512 solves): converged solves per second and the statistics
        per wavelength."""
        steps = r["infos"][:N_STEPS_PASS]
        assert sorted(t for t, _ in steps) == list(range(N_STEPS_PASS))
        ms = float(sum(r["per_step"][:N_STEPS_PASS]))
        flat = [i for _, inf in steps for i in inf]
        wl = [w for t, _ in steps for w in test_wl[t]]
        solved = int(sum(i["converged"] for i in flat))
        return {"value": round(solved / (ms / 1e3), 3), "unit": "solves/s", "seconds": round(ms / 1e3, 3),
                **summarize(flat, wl)}

    def one_pass(step):
        r = timed(step, N_STEPS_PASS, 1)
        return pass_of(r), r

    K, W = args.steps, args.warmup
    set_policy(pol_cnn)
    head = timed(step_cnn, K, W, start=0, clocks=True)
    value = head["solved"] / (head["ms"] / 1e3)
    # the same step with CUDA events around every launch (they order the
    # launches, and the step loop is host-driven): per-class kernel times
    prof = timed(step_cnn, 1, 0, start=0, profile=True)["prof"]
    # CNN inference of one step alone
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    P.predict(test_ops[0], src, U=U_cnn_rows)
    e1.record()
    torch.cuda.synchronize()
    predict_ms = e0.elapsed_time(e1)

    # the CNN's pass over the 512 held-out solves: the first N_STEPS_PASS
    # timed steps when there are that many (they start at step W mod
    # N_STEPS_PASS and go round)
    cnn_pass = pass_of(head) if K >= N_STEPS_PASS else one_pass(step_cnn)[0]
    pca_pass = pca_run = None
    if not args.no_pca:
        set_policy(pol_pca)
        pca_pass, pca_run = one_pass(step_pca)
    plain_pass = plain_run = None
    plain_sample = None
    if not args.no_plain:
        plain_pass, plain_run = one_pass(step_plain)
        # plain GMRES(200) without the cap on one held-out trajectory (context:
        # how far past the cap the 1300 nm solves go)
        for x in xs:
            x.zero_()
        _, inf_u, _ = ddg.gmres_solve_batched(ctx, test_ops[0], test_b[0], x=xs, tol=1e-6, restart=args.restart,
                                              maxit=20000, precision=args.precision)
        plain_sample = {"trajectories": [N_TRAIN_TRAJ + t for t in step_traj(0)], "maxit": 20000,
                        **summarize(inf_u, test_wl[0])}

    levers = None
    if args.levers:
        # what moves the CNN's gain: the CNN's vectors alone (each restart
        # policy), and the headline's subspace with each fixed policy
        levers = {}
        for name, solve, cands in (("cnn8", solve_cnn8, [(1, 0), (every, args.cnn_k)]),
                                   ("pca20_plus_cnn8", solve_cnn, [(1, 0), (1, args.k), (every, kc)])):
            for cand in cands:
                set_policy({lam: cand for lam in WAVELENGTHS})
                levers[f"{name}_cycles{min(cand[0], 99)}_keep{cand[1]}"] = one_pass(
                    lambda t, solve=solve: solve(test_ops[t], test_b[t]))[0]
        # k = 16: the CNN's 16 vectors alone, and [PCA-16 | CNN-16]
        U16 = [torch.empty((16, D), dtype=torch.complex128, device=dev) for _ in range(n_step)]
        U_comb16 = [torch.empty((32, D), dtype=torch.complex128, device=dev) for _ in range(n_step)]
        for u, lam in zip(U_comb16, step_lams):
            u[:16].copy_(U_pca[lam][:16])

        def solve_cnn16(ops, bs):
            for x in xs:
                x.zero_()
            P16.predict(ops, src, U=U16)
            return ddg.augmented_gmres_solve_batched(ctx, ops, bs, U16, x=xs, **kw)

        def solve_pca16_cnn16(ops, bs):
            for x in xs:
                x.zero_()
            P16.predict(ops, src, U=[u[16:] for u in U_comb16])
            return ddg.augmented_gmres_solve_batched(ctx, ops, bs, U_comb16, x=xs, **kw)

        for name, solve, cands in (("cnn16", solve_cnn16, [(1, 0), (every, 16)]),
                                   ("pca16_plus_cnn16", solve_pca16_cnn16, [(1, 0), (1, 16)])):
            for cand in cands:
                set_policy({lam: cand for lam in WAVELENGTHS})
                levers[f"{name}_cycles{min(cand[0], 99)}_keep{cand[1]}"] = one_pass(
                    lambda t, solve=solve: solve(test_ops[t], test_b[t]))[0]

        # training-set size: the headline's subspace and policy with the k = 8
        # network trained on a quarter of the problems
        def solve_cnn_quarter(ops, bs):
            for x in xs:
                x.zero_()
            Pq.predict(ops, src, U=U_cnn_rows)
            return ddg.augmented_gmres_solve_batched(ctx, ops, bs, U_comb, x=xs, **kw)

        set_policy(pol_cnn)
        levers[f"pca20_plus_cnn8_trained_on_{Pq.n_problems}"] = one_pass(
            lambda t: solve_cnn_quarter(test_ops[t], test_b[t]))[0]
        levers["train_loss_last"] = {"cnn8": round(float(np.mean(train_losses[-20:])), 5),
                                     "cnn16": round(float(np.mean(P16.train_losses[-20:])), 5),
                                     f"cnn8_{Pq.n_problems}": round(float(np.mean(Pq.train_losses[-20:])), 5)}
        set_policy(pol_cnn)

    # --- e2e: host permittivities in, host fields out, through fdfd_solve_host
    eps_host = [[torch.from_numpy(np.ascontiguousarray(e)).pin_memory() for e in test_eps[t]]
                for t in range(N_TEST_TRAJ)]
    x_host = [torch.empty(D, dtype=torch.complex128).pin_memory() for _ in range(n_step)]
    e2e_grids = [g for g in grids for _ in range(n_step // len(grids))]

    set_policy(pol_cnn)

    def step_e2e(st):
        ep = [eps_host[t][j] for _ in grids for t in step_traj(st) for j in range(TRAJ_STEPS)]
        inf, st_ = ddg.fdfd_solve_host(ctx, e2e_grids, ep, src, x_host, P=P, U_fixed=U_pca_step, **kw)
        return None, inf, st_

    eK = max(2, min(K, 4))
    e2 = timed(step_e2e, eK, 1, start=0)
    e2e = {"value": round(e2["solved"] / (e2["ms"] / 1e3), 3), "unit": "solves/s", "steps": eK,
           "h2d_bytes_per_step": int(n_step * D * 8), "d2h_bytes_per_step": int(n_step * D * 16),
           "call": "fdfd_solve_host (eps from pinned host memory; operators, sources, CNN prediction, "
                   "solve; fields copied back to pinned host memory)"}

    roof = roofline(args, prof)
    flat = [i for _, inf in head["infos"] for i in inf]
    wl = [w for t, _ in head["infos"] for w in test_wl[t]]
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "solves/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": round(head["ms"] / K, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64+f64" if args.precision == "c64" else "c128",
        "data": "synthetic",
        "config": headline_config(args, world),
        "cnn": {**summarize(flat, wl), "subspace": f"[PCA-{args.k} of the wavelength | CNN-{args.cnn_k}]",
                "policy": rep_cnn, "pass": cnn_pass, "predict_ms_per_step": round(predict_ms, 2),
                "train_s": round(cnn_s, 1), "loss": "Eq. 6 (residual)", "train_steps": args.cnn_steps,
                "batch": args.cnn_batch, "lr": args.cnn_lr,
                "train_loss_first": round(float(np.mean(train_losses[:20])), 5),
                "train_loss_last": round(float(np.mean(train_losses[-20:])), 5)},
        "pca": {"k": args.k, "policy": rep_pca, **pca_pass} if pca_pass else None,
        "plain": plain_pass,
        "plain_uncapped_sample": plain_sample,
        "speedup_vs_plain": round(cnn_pass["value"] / plain_pass["value"], 3) if plain_pass else None,
        "pca_speedup_vs_plain": round(pca_pass["value"] / plain_pass["value"], 3) if plain_pass and pca_pass else None,
        "speedup_note": "same 512 held-out solves, one pass each; solves/s counts converged solves only "
                        "(non-converged ones count in the time); plain GMRES(200) misses the 5000 cap on most "
                        "1300 nm solves (its iterations-to-cap and residual reached are in plain.1300nm)",
        "setup": {"operators_s": round(setup_s, 1), "pca_fields_s": round(pca_s, 1), "pca_fields": pca_info,
                  "policy_tuning_s": round(tune_s, 1),
                  "n_pca_per_wavelength": args.n_pca},
        "levers": levers,
        "roofline": roof, "e2e": e2e, "gpu_launches": int(head["launches"]), "clocks": head["clocks"],
    }
    line["_oracle_sample"] = oracle_sample_spec(P, U_base, test_eps, grids, flat, wl, head["infos"],
                                                U_pca=U_pca, policy=pol_cnn)
    if args.log_jsonl and rank == 0:
        recs = solve_records("cnn", head["infos"], head["per_step"], grids)
        for name, run in (("pca", pca_run), ("plain", plain_run)):
            if run is not None:
                recs += solve_records(name, run["infos"], run["per_step"], grids)
        with open(args.log_jsonl, "w") as f:
            for r in recs:
                f.write(json.dumps(r) + "\n")
    return line


def train_cnn(ddg, args, grids, train_ops, b_of, U_base, src, D, steps=None, n_problems=None, k=None, seed=0):
    """The subspace CNN: He-initialised, zero head, output offset = the k
    leading PCs of each wavelength (scaled to O(1) entries), trained with the
    residual loss on random batches of the training problems (both
    wavelengths)."""
    k = k or args.cnn_k
    P = ddg.Predictor(k=k)
    P.init_he(seed=seed)
    P.set_tensor_cores(True, backward=True)      # forward and backward convolutions on tcgen05
    for g in grids:
        P.set_output_base(U_base[g.wavelength][:k], g.nx, g.ny, scale=float(np.sqrt(D)), wavelength=g.wavelength)
    P.zero_head()
    P.set_loss("residual")
    pool = [(lam, i) for lam in WAVELENGTHS for i in range(len(train_ops[lam]))]
    if n_problems is not None:
        pool = pool[: n_problems // 2] + pool[len(pool) // 2: len(pool) // 2 + n_problems // 2]
    rng = np.random.default_rng(seed)
    losses = []
    for _ in range(steps or args.cnn_steps):
        idx = rng.choice(len(pool), args.cnn_batch, replace=False)
        ops = [train_ops[pool[i][0]][pool[i][1]] for i in idx]
        losses.append(P.train_step(ops, src, [b_of[pool[i][0]] for i in idx], args.cnn_lr))
    P.train_losses = losses
    return P


def roofline(args, prof):
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
    # DRAM bytes over algorithmic bytes of the same kernels, from one ncu
    # capture per basis storage (dram__bytes_read.sum + dram__bytes_write.sum
    # of one launch at Arnoldi step 101: FP32 basis, 32 solves of 256x256;
    # half basis, 64 solves of 128x128); the summaries are in profiles/.  The
    # half-basis k_dots2 has changed since its capture (alpha and gamma partials
    # formed before the stage loop), so it has no ratio until it is taken again.
    ratio = ({"update": 1.02} if args.basis == "f16" else {"dots": 1.01, "update": 1.02}).get(dom)
    return {"kernel": {"dots": "k_dots2", "update": "k_update2"}.get(dom, f"k_{dom}"), "bound": "hbm",
            "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "traffic": round(ratio * d_bytes / d_n) if ratio else None,
            "traffic_source": ("ncu dram bytes / algorithmic bytes = %.2f for this kernel, times the mean "
                               "algorithmic bytes per launch" % ratio) if ratio else None,
            "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)",
            "timing": "CUDA events around every launch on the solver's stream, profiled pass of one timed step",
            "launches": d_n, "avg_launch_us": round(d_ms * 1e3 / max(1, d_n), 2),
            "algorithmic_bytes_per_launch": round(d_bytes / max(1, d_n)),
            "share_of_kernel_time": round(d_ms / total_ms, 4),
            "classes": {c: {"ms": round(v[0], 2), "GBps": round(v[1] / max(v[0], 1e-9) / 1e6, 1),
                            "launches": v[2]} for c, v in prof.items()}}


# ------------------------------------------------------------------ other workloads
def timed_call(torch, fn):
    """One call between CUDA events on the current stream: (result, ms)."""
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    r = fn()
    e1.record()
    torch.cuda.synchronize()
    return r, e0.elapsed_time(e1)


def run_large(args, rank, world):
    """The large grid: 1024x1024 at 20 nm (about 1M unknowns), 1550 nm,
    20-cell PML; 64 held-out solves (4 trajectories x 16 steps, seeds
    PCG64(5000 + t), t < 4); the CNN (k = 16) trained with the residual loss on
    256 problems of trajectories 4-19, its output offset the 16 leading PCs of
    16 approximate training fields (plain GMRES(200), 2000 steps: restarted
    GMRES does not converge on this grid).  Plain and CNN-augmented GMRES(200)
    in complex64 + FP64 refinement to 1e-6, and the FP32-only path to 1e-4, all
    capped at --maxit; a solve that misses its tolerance reports the steps run
    and the residual reached."""
    import torch
    import paper_1902_00090_gb300 as ddg
    from paper_1902_00090_gb300 import inputs

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    g = inputs.grid_1024()
    src = (g.i_src, g.sigma_src, g.j_src)
    k = 16
    t0 = time.time()
    test_ops = [ddg.fdfd_operator(g, torch.as_tensor(e, device=dev)) for t in range(4)
                for e in inputs.trajectory_eps(g, 5, t)]
    train_ops = [ddg.fdfd_operator(g, torch.as_tensor(e, device=dev)) for t in range(4, 20)
                 for e in inputs.trajectory_eps(g, 5, t)]
    b = ddg.fdfd_source(test_ops[0], *src)
    ctx = ddg.Context()
    ctx.set_graphs(args.graphs == "on")
    ctx.set_basis_storage(args.basis)
    pick = list(range(0, len(train_ops), len(train_ops) // 16))[:16]
    xs, inf_f, _ = ddg.gmres_solve_batched(ctx, [train_ops[i] for i in pick], [b] * len(pick), tol=1e-6,
                                           restart=200, maxit=2000, precision="c64")
    U_base, _ = ddg.pca_fit(ctx, torch.stack(xs), k)
    del xs
    P = ddg.Predictor(k=k)
    P.init_he(seed=0)
    P.set_tensor_cores(True, backward=True)
    P.set_output_base(U_base, g.nx, g.ny, scale=float(np.sqrt(g.D)))
    P.zero_head()
    P.set_loss("residual")
    rng = np.random.default_rng(0)
    batch = 4
    losses = [P.train_step([train_ops[i] for i in rng.choice(len(train_ops), batch, replace=False)], src,
                           [b] * batch, args.cnn_lr) for _ in range(args.cnn_steps)]
    setup_s = time.time() - t0
    n = len(test_ops)
    bs = [b] * n
    x = [torch.zeros(g.D, dtype=torch.complex128, device=dev) for _ in range(n)]
    U = [torch.empty((k, g.D), dtype=torch.complex128, device=dev) for _ in range(n)]
    out = {}
    for name, tol, prec in (("c64_refine_1e-6", 1e-6, "c64"), ("fp32_only_1e-4", 1e-4, "c64_only")):
        for variant, pol in (("plain", None), ("cnn_first_cycle", (1, 0)), ("cnn_kept", (10**6, k))):
            for v in x:
                v.zero_()
            if pol:
                ctx.set_augmented_policy(*pol)
            if variant == "plain":
                (_, inf, st), ms = timed_call(torch, lambda: ddg.gmres_solve_batched(
                    ctx, test_ops, bs, x=x, tol=tol, restart=args.restart, maxit=args.maxit, precision=prec))
            else:
                def go():
                    for c0 in range(0, n, 16):     # prediction in chunks: activations of 16 grids of 1M cells
                        P.predict(test_ops[c0:c0 + 16], src, U=U[c0:c0 + 16])
                    return ddg.augmented_gmres_solve_batched(ctx, test_ops, bs, U, x=x, tol=tol,
                                                             restart=args.restart, maxit=args.maxit, precision=prec)
                (_, inf, st), ms = timed_call(torch, go)
            conv = sum(i["converged"] for i in inf)
            out[f"{variant}_{name}"] = {"value": round(conv / (ms / 1e3), 4), "unit": "solves/s",
                                        "seconds": round(ms / 1e3, 2), "tol": tol, **summarize(inf)}
    # HBM fraction of the Arnoldi kernels at this size: a short profiled run
    ctx.profile_enable(True)
    for v in x:
        v.zero_()
    ddg.gmres_solve_batched(ctx, test_ops, bs, x=x, tol=1e-6, restart=args.restart, maxit=2 * args.restart,
                            precision="c64")
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    roof = roofline(args, prof)
    roof["timing"] = "CUDA events around every launch, two restart cycles of the 64 plain solves"
    best = max(("cnn_first_cycle", "cnn_kept"), key=lambda v: out[f"{v}_c64_refine_1e-6"]["value"])
    return {"metric": METRIC, "workload": "large1024", "value": out[f"{best}_c64_refine_1e-6"]["value"],
            "unit": "solves/s", "n_gpus": world, "higher_is_better": True, "dtype": "c64+f64", "data": "synthetic",
            "config": {"workload": "large1024: 1024x1024 Yee grid at 20 nm (1,048,576 unknowns), 1550 nm, "
                                   "20-cell PML, 64 held-out solves (4 trajectories x 16), CNN k=16 against plain "
                                   "GMRES(200); complex64 + FP64 refinement to 1e-6 and FP32-only to 1e-4",
                       "restart": args.restart, "maxit": args.maxit,
                       "krylov_basis_storage": args.basis, "basis_bytes": n * (args.restart + 1) * g.D * 8,
                       "cnn_train_steps": args.cnn_steps, "cnn_batch": batch,
                       "restart_policy": "cnn_first_cycle: the 16 vectors in the first cycle, then plain GMRES; "
                                         "cnn_kept: the 16 vectors in every cycle; value = the better one",
                       "value_variant": best},
            "runs": out, "offset_fields": summarize(inf_f),
            "cnn_train_loss_first": round(float(np.mean(losses[:10])), 5),
            "cnn_train_loss_last": round(float(np.mean(losses[-10:])), 5), "setup_s": round(setup_s, 1),
            "roofline": roof}


BATCH_SIZES = ((128, 128), (192, 192), (256, 256), (384, 256))


def run_batched(args, rank, world):
    """The batched-solves workload: 1024 correlated solves from 64 design
    trajectories (16 per grid size: 128x128, 192x192, 256x256, 384x256; 40 nm,
    1550 nm; seeds PCG64(4000 + t), trajectories 32 s + 16 .. 32 s + 31 of size
    s held out, 32 s .. 32 s + 15 for training), run through the solve queue
    (group width and lanes autotuned) as three variants: plain GMRES, PCA-20
    and CNN-8 (PCA and CNN fitted and trained per grid size), plus the CNN
    with recycling along the trajectories (gmres_solve_trajectories).
    Complex64 + FP64 refinement to 1e-6, cap --maxit."""
    import torch
    import paper_1902_00090_gb300 as ddg
    from paper_1902_00090_gb300 import autotune, inputs

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    t0 = time.time()
    lanes = []
    for _ in range(2):
        c = ddg.Context()
        c.set_graphs(args.graphs == "on")
        c.set_basis_storage(args.basis)
        c.set_augmented_policy(1, 0)      # the subspace in the first cycle, then plain GMRES
        lanes.append(c)
    ctx = lanes[0]
    ops, bs, U_pca, U_cnn, per_size = [], [], [], [], {}
    traj_ops = {}
    for si, (nx, ny) in enumerate(BATCH_SIZES):
        g = inputs.grid_for(nx, ny)
        src = (g.i_src, g.sigma_src, g.j_src)
        tr_ops = [ddg.fdfd_operator(g, torch.as_tensor(e, device=dev)) for t in range(16)
                  for e in inputs.trajectory_eps(g, 4, 32 * si + t)]
        b = ddg.fdfd_source(tr_ops[0], *src)
        pick = list(range(0, len(tr_ops), len(tr_ops) // args.n_pca))[: args.n_pca]
        xs, inf, _ = ddg.gmres_solve_batched(ctx, [tr_ops[i] for i in pick], [b] * len(pick), tol=1e-6,
                                             restart=200, maxit=20000, precision="c64")
        F = torch.stack(xs)
        up, _ = ddg.pca_fit(ctx, F, args.k)
        ub, _ = ddg.pca_fit(ctx, F, args.cnn_k)
        del F, xs
        P = ddg.Predictor(k=args.cnn_k)
        P.init_he(seed=si)
        P.set_tensor_cores(True, backward=True)
        P.set_output_base(ub, nx, ny, scale=float(np.sqrt(g.D)))
        P.zero_head()
        P.set_loss("residual")
        rng = np.random.default_rng(si)
        for _ in range(args.cnn_steps):
            idx = rng.choice(len(tr_ops), args.cnn_batch, replace=False)
            P.train_step([tr_ops[i] for i in idx], src, [b] * args.cnn_batch, args.cnn_lr)
        del tr_ops
        te = [[ddg.fdfd_operator(g, torch.as_tensor(e, device=dev)) for e in inputs.trajectory_eps(g, 4, 32 * si + 16 + t)]
              for t in range(16)]
        traj_ops[(nx, ny)] = (te, b)
        flat = [op for tr in te for op in tr]
        ops += flat
        bs += [b] * len(flat)
        U_pca += [up] * len(flat)
        per_size[(nx, ny)] = (P, src, flat)
    setup_s = time.time() - t0
    n = len(ops)
    kw = dict(tol=1e-6, maxit=args.maxit, precision=args.precision)

    def run(ln, A, b, U, w, nl, tol, m, maxit, prec):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        _, infos, _ = ddg.gmres_solve_queue(ln[:nl], A, b, U=U, width=w, tol=tol, restart=m, maxit=maxit,
                                            precision=prec)
        torch.cuda.synchronize()
        return sum(1 for i in infos if i["converged"]) / (time.perf_counter() - t1)

    tune = autotune.tune_queue(lanes, ops, bs, sample=64, widths=(32, 64, 128), lane_counts=(1, 2),
                               restart=args.restart, basis=args.basis, run=run, repeats=1, **kw)
    width, nl = tune["width"], tune["lanes"]
    out = {}

    def predict_all():
        Us = []
        for (nx, ny), (P, src, flat) in per_size.items():
            Us += P.predict(flat, src)
        return Us

    for variant in ("plain", "pca20", "cnn8"):
        def go():
            U = None if variant == "plain" else (U_pca if variant == "pca20" else predict_all())
            return ddg.gmres_solve_queue(lanes[:nl], ops, bs, U=U, width=width, restart=args.restart, **kw)
        (_, inf, st), ms = timed_call(torch, go)
        conv = sum(i["converged"] for i in inf)
        sizes = [f"{o.nx}x{o.ny}" for o in ops]
        d = {"value": round(conv / (ms / 1e3), 3), "unit": "solves/s", "seconds": round(ms / 1e3, 2),
             **summarize(inf)}
        for sz in sorted(set(sizes)):
            d[sz] = summarize([i for i, z in zip(inf, sizes) if z == sz])
        out[variant] = d

    # the CNN with recycling along the trajectories (subspace [CNN-8 |
    # previous solution]) through the queue over trajectories: groups of 8
    # trajectories of one grid size on 4 lanes
    rl = lanes + [ddg.Context() for _ in range(2)]
    for c in rl[2:]:
        c.set_graphs(args.graphs == "on")
        c.set_basis_storage(args.basis)
        c.set_augmented_policy(1, 0)

    def recycle():
        A, B, Ut = [], [], []
        for (nx, ny), (te, b) in traj_ops.items():
            P, src, flat = per_size[(nx, ny)]
            Us = P.predict(flat, src)
            A += te
            B += [[b] * 16 for _ in range(16)]
            Ut += [Us[16 * r:16 * (r + 1)] for r in range(16)]
        _, inf, _ = ddg.gmres_solve_queue_trajectories(rl, A, B, Ut, traj_per_group=8, restart=args.restart, **kw)
        return [i for tr in inf for i in tr]
    inf_r, ms = timed_call(torch, recycle)
    out["cnn8_recycle"] = {"value": round(sum(i["converged"] for i in inf_r) / (ms / 1e3), 3), "unit": "solves/s",
                           "seconds": round(ms / 1e3, 2), **summarize(inf_r),
                           "note": "gmres_solve_queue_trajectories: groups of 8 trajectories (one grid size) on 4 "
                                   "lanes, step t of a group's trajectories in one batch"}
    for c in rl:
        c.close()
    return {"metric": METRIC, "workload": "batched", "value": out["cnn8"]["value"], "unit": "solves/s",
            "n_gpus": world, "higher_is_better": True, "dtype": "c64+f64", "data": "synthetic",
            "config": {"workload": "batched: 1024 correlated solves from 64 trajectories, 256 each of 128x128, "
                                   "192x192, 256x256 and 384x256 (40 nm, 1550 nm), through the solve queue; plain, "
                                   "PCA-20 and CNN-8 (fitted and trained per grid size)",
                       "restart": args.restart, "maxit": args.maxit, "queue": {"width": width, "lanes": nl},
                       "tuning": [{"width": t[0], "lanes": t[1], "solves_per_s": round(t[2], 2)}
                                  for t in tune["timings"]],
                       "krylov_basis_storage": args.basis, "cnn_train_steps": args.cnn_steps,
                       "restart_policy": "the subspace in the first cycle, then plain GMRES"},
            "variants": out, "speedup_cnn_vs_plain": round(out["cnn8"]["value"] / out["plain"]["value"], 3),
            "setup_s": round(setup_s, 1)}


# ------------------------------------------------------------------ oracle (CPU)
def oracle_sample_spec(P, U_base, test_eps, grids, flat, wl, step_infos, U_pca=None, policy=None, per_wl=8):
    """What the CPU baseline needs from the GPU run: the trained weights, the
    output offset, PCA rows and restart policy of each wavelength, and the
    sampled problems (the first `per_wl` permittivities of the first timed
    step at each wavelength) with the restart cycles and steps their GPU
    solves needed, to scale the sample."""
    st0, inf0 = step_infos[0]
    t0 = step_traj(st0)[0]
    n_wl = TRAJ_PER_STEP * len(test_eps[0])      # solves of one wavelength in a step (1300 nm first)
    spec = {"theta": P.get_params(), "channels": P.channels, "k": P.k,
            "base": {g.wavelength: U_base[g.wavelength][: P.k].cpu().numpy() for g in grids},
            "problems": [{"eps": test_eps[t0][j], "grid": g, "gpu_cycles": int(inf0[w * n_wl + j]["cycles"]),
                          "gpu_iters": int(inf0[w * n_wl + j]["iters"])}
                         for w, g in enumerate(grids) for j in range(per_wl)]}
    if U_pca is not None:
        spec["pca"] = {g.wavelength: U_pca[g.wavelength].cpu().numpy() for g in grids}   # (k_pca, D) each
    if policy is not None:
        spec["policy"] = {g.wavelength: tuple(int(v) for v in policy[g.wavelength]) for g in grids}
    return spec


def oracle_cnn_subspace(spec, prob):
    """The headline variant's subspace for one sampled problem, computed by the
    oracle: [PCA rows of its wavelength | its fp64 forward pass of the trained
    weights plus the offset] (the CNN part alone without PCA rows in the spec)."""
    from oracle import cnn as ocnn
    g = prob["grid"]
    cfg = ocnn.CNNConfig(cin=4, channels=tuple(spec["channels"]), k=spec["k"])
    x = ocnn.input_channels(prob["eps"], g.wavelength, g.npml, g.i_src, g.sigma_src, g.j_src)[None]
    y = ocnn.forward(cfg, spec["theta"].astype(np.float64), x)
    V = ocnn.to_complex_fields(y)[0]                       # (D, k)
    V = V + np.sqrt(g.D) * spec["base"][g.wavelength].T
    if "pca" in spec:
        V = np.concatenate([spec["pca"][g.wavelength].T, V], axis=1)
    return V


def _oracle_job(job):
    """One sampled problem in a worker process: the oracle's subspace and
    `cycles` restart cycles of its augmented GMRES; (prediction s, solve s,
    cycles run, first-step residual)."""
    from oracle import fdfd, gmres
    spec, prob, restart, cycles = job
    g = prob["grid"]
    A = fdfd.operator_for(g, prob["eps"])
    b = fdfd.source_for(g)
    t0 = time.time()
    V = oracle_cnn_subspace(spec, prob)
    t_pred = time.time() - t0
    cyc, keep = spec.get("policy", {}).get(g.wavelength, (10**6, V.shape[1]))
    t0 = time.time()
    _, info = gmres.augmented_gmres(A, b, V, tol=1e-6, restart=restart, maxit=cycles * restart,
                                    aug_cycles=cyc, aug_keep=keep)
    return t_pred, time.time() - t0, int(info.cycles), float(info.first_step_rel_residual)


def cpu_baseline(args, spec, cycles=1, procs=None):
    """The oracle (numpy/scipy complex128) on every host core, on a bounded
    sample: the sampled held-out problems of the headline variant (the
    subspace [PCA rows | CNN-k] from the oracle's own fp64 forward pass of the
    trained weights, the restart policy of each problem's wavelength), each in
    a process of its own with one BLAS thread, all at once; each runs its
    first `cycles` restart cycles, scaled to a whole solve by the restart
    cycles its GPU solve needed.  Solves/s = processes / mean seconds per
    solve (each core working through solves one after another).  The pool is
    started with spawn (this process has a CUDA context)."""
    import multiprocessing as mp
    probs = spec["problems"]
    nproc = max(1, min(len(probs), procs or os.cpu_count() or 1))
    shared = {k: v for k, v in spec.items() if k != "problems"}
    jobs = [({**shared, "base": {p["grid"].wavelength: shared["base"][p["grid"].wavelength]},
              **({"pca": {p["grid"].wavelength: shared["pca"][p["grid"].wavelength]}} if "pca" in shared else {})},
             p, args.restart, cycles) for p in probs]
    saved = {v: os.environ.get(v) for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
    for v in saved:
        os.environ[v] = "1"      # inherited by the spawned workers before they load numpy
    try:
        t0 = time.time()
        with mp.get_context("spawn").Pool(nproc) as pool:
            res = pool.map(_oracle_job, jobs, chunksize=1)
        wall = time.time() - t0
    finally:
        for v, val in saved.items():
            if val is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = val
    sec = [tp + ts / max(1, c) * p["gpu_cycles"] for (tp, ts, c, _), p in zip(res, probs)]
    mean_sec = float(np.mean(sec))
    per_cycle = float(np.mean([ts / max(1, c) for _, ts, c, _ in res]))
    n_wl = len({p["grid"].wavelength for p in probs})
    sub = (f"[PCA-{next(iter(spec['pca'].values())).shape[0]} | CNN-{spec['k']}]" if "pca" in spec
           else f"CNN-{spec['k']}")
    pol = "; ".join(f"{int(round(l * 1e9))} nm: all columns for {c} cycle(s), then {k} kept"
                    for l, (c, k) in sorted(spec.get("policy", {}).items()))
    return {"value": round(nproc / mean_sec, 6), "unit": "solves/s", "cores": nproc, "kind": "oracle",
            "sample": f"{len(probs)} held-out {probs[0]['grid'].nx}x{probs[0]['grid'].ny} solves "
                      f"({len(probs) // n_wl} per wavelength, the first permittivities of the first timed step), "
                      f"augmented GMRES({args.restart}) with the headline's subspace {sub} (the trained network's "
                      f"fp64 forward pass) and restart policy ({pol}), {cycles} restart cycle(s) each "
                      f"({per_cycle:.1f} s per cycle on average, complex128 numpy/scipy), scaled to the "
                      f"{np.mean([p['gpu_cycles'] for p in probs]):.1f} cycles "
                      f"({np.mean([p['gpu_iters'] for p in probs]):.0f} steps) their GPU solves needed on "
                      f"average; {nproc} spawned processes with one BLAS thread each, all at once "
                      f"({wall:.1f} s wall); solves/s = processes / mean seconds per solve",
            "oracle_first_step_rel_residual": round(float(np.mean([r[3] for r in res])), 5)}


def run_reference(args, rank, world):
    """The oracle timed on the host cores, on the same workload and metric.
    Each step is one GMRES(200) restart cycle of a held-out 1550 nm solve
    augmented by the k leading PCs of 8 oracle-solved training fields (set-up
    untimed; the trained CNN exists only on the GPU side, so the oracle runs
    the PCA variant), the cycles of consecutive steps continuing one solve (a
    converged solve starts the next from zero).  Solves/s = 1 / (mean cycle
    time x cycles the oracle needed for that solve; when it did not converge
    within the run, the cycles extrapolated from its residual reduction)."""
    if rank != 0:
        return None
    import scipy.sparse.linalg as spla
    from oracle import fdfd, gmres, pca
    g = splitter_grids()[1]
    b = fdfd.source_for(g)
    train = [trajectory(t)[0] for t in range(0, N_TRAIN_TRAJ, N_TRAIN_TRAJ // 8)]
    F = np.column_stack([spla.spsolve(fdfd.operator_for(g, e).tocsc(), b) for e in train])
    U, _ = pca.pca_basis(F, args.k)
    A = fdfd.operator_for(g, trajectory(N_TRAIN_TRAJ)[0])
    x = np.zeros(g.D, dtype=np.complex128)
    times, cycles, conv_at, res = [], 0, None, 1.0
    for q in range(args.warmup + args.steps):
        t0 = time.time()
        x, info = gmres.augmented_gmres(A, b, U, x0=x, tol=1e-6, restart=args.restart, maxit=args.restart)
        dt = time.time() - t0
        cycles += 1
        res = info.true_rel_residual
        if q >= args.warmup:
            times.append(dt)
        if info.converged:
            conv_at = conv_at or cycles
            x = np.zeros(g.D, dtype=np.complex128)
            cycles = 0
    per_cycle = float(np.mean(times))
    if conv_at:
        need, how = conv_at, "measured"
    else:
        need = int(np.ceil(cycles * np.log(1e-6) / np.log(max(res, 1e-300)))) if res < 1 else args.maxit // args.restart
        need, how = min(need, args.maxit // args.restart), f"extrapolated from residual {res:.2e} after {cycles} cycles"
    v = 1.0 / (per_cycle * need)
    cb = {"value": round(v, 6), "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
          "sample": f"each step: one GMRES({args.restart}) restart cycle of a held-out 256x256 1550 nm solve "
                    f"augmented by k={args.k} PCs of 8 oracle-solved training fields (the workload's PCA variant: "
                    f"the trained CNN exists only in the GPU arm's run; complex128 numpy/scipy, "
                    f"{per_cycle:.2f} s per cycle), scaled by {need} cycles per solve ({how}); BLAS threads = "
                    f"os.cpu_count() = {os.cpu_count()}"}
    return {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per_cycle * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": headline_config(args, world),
            "cpu_baseline": cb,
            "e2e": {"value": round(v, 6), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.case is not None:
        {"solver": case_solver, "cnn": case_cnn, "cnn-train": case_cnn_train, "stencil": case_stencil,
         "plain-steps": case_plain_steps}[args.case](args)
        return
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
    line = {"splitter256": run_ours, "large1024": run_large, "batched": run_batched}[args.workload](args, rank, world)
    spec = line.pop("_oracle_sample", None)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline and spec is not None:
            line["cpu_baseline"] = cpu_baseline(args, spec)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
