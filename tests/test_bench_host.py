"""Host logic of bench.py that needs no GPU: the clock record taken during the
timed region (parsing of nvidia-smi samples) and the restart-policy choice."""
import os
import sys
import threading

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def sampler_with(lines):
    c = bench.ClockSampler(0)
    c.proc = FakeProc()
    c.t = threading.Thread(target=lambda: None)
    c.t.start()
    c.lines = list(lines)
    return c


def test_clock_record_median_max_and_reasons():
    lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    r = sampler_with(lines).stop()
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_record_flags_throttling_and_missing_samples():
    r = sampler_with(["0, 1500, 2070, 1400, 0x40, Not Active, Active, Not Active, Not Active"]).stop()
    assert r["reasons"] == ["hw_thermal_slowdown"] and r["sm_mhz"] == 1500.0
    assert sampler_with([]).stop()["reasons"] == ["no samples"]
    c = bench.ClockSampler(0)
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_policy_choice_needs_a_margin_to_keep_more_columns():
    every = 10**6
    # mean steps per wavelength as a validation pass reports them
    table = [((1, 0), {1: 3932.3, 2: 2534.9}), ((1, 8), {1: 4041.4, 2: 3170.2}),
             ((1, 20), {1: 3371.6, 2: 3210.0}), ((every, 28), {1: 3327.3, 2: 3390.0})]
    # 1300 nm: 1/20 saves 14 % over 1/0; all 28 kept saves only 1.3 % more
    assert bench.choose_policy(table, 1) == (1, 20)
    assert bench.choose_policy(table, 1, margin=0.0) == (every, 28)
    # 1550 nm: the first-cycle policy has the fewest steps
    assert bench.choose_policy(table, 2) == (1, 0)
    # the order of the table does not matter
    assert bench.choose_policy(table[::-1], 1) == (1, 20)
    # a large saving still buys more columns
    big = [((1, 0), {1: 5000.0}), ((every, 20), {1: 3400.0})]
    assert bench.choose_policy(big, 1) == (every, 20)


def test_cpu_baseline_runs_the_headline_subspace_and_policy():
    # The CPU baseline's oracle sample uses the headline variant's subspace
    # [PCA rows | CNN-k] and the restart policy of each problem's wavelength
    # (a tiny network on a 32x32 grid), one spawned single-thread process per
    # sampled problem.
    import numpy as np
    from types import SimpleNamespace
    from oracle import cnn as ocnn
    from paper_1902_00090_gb300 import inputs
    grids = [inputs.Grid(nx=32, ny=32, npml=4, i_src=6, sigma_src=3.0, slab_cells=2, wavelength=lam)
             for lam in (1300e-9, 1550e-9)]
    channels, k = (4, 4, 4, 4, 4, 4), 2
    cfg = ocnn.CNNConfig(cin=4, channels=channels, k=k)
    n = ocnn.num_params(cfg)
    rng = np.random.default_rng(0)
    D = grids[0].D
    pca = {g.wavelength: np.linalg.qr(rng.standard_normal((D, 3)) + 1j * rng.standard_normal((D, 3)))[0].T
           for g in grids}
    spec = {"theta": 0.1 * rng.standard_normal(n).astype(np.float32), "channels": channels, "k": k,
            "base": {g.wavelength: np.zeros((k, D), dtype=np.complex128) for g in grids},
            "pca": pca, "policy": {1300e-9: (10**6, 3), 1550e-9: (1, 0)},
            "problems": [{"eps": inputs.bernoulli_eps(g, j), "grid": g, "gpu_cycles": 3, "gpu_iters": 90}
                         for g in grids for j in range(2)]}
    V = bench.oracle_cnn_subspace(spec, spec["problems"][2])
    assert V.shape == (D, 3 + k) and np.array_equal(V[:, :3], pca[1550e-9].T)
    r = bench.cpu_baseline(SimpleNamespace(restart=30), spec, cycles=2, procs=2)
    assert r["kind"] == "oracle" and r["value"] > 0 and r["cores"] == 2
    assert "[PCA-3 | CNN-2]" in r["sample"] and "1550 nm: all columns for 1 cycle(s), then 0 kept" in r["sample"]
    assert "4 held-out 32x32 solves (2 per wavelength" in r["sample"]


def test_timed_steps_cover_the_held_out_set_once_per_pass():
    # one pass of timed steps holds every held-out trajectory exactly once
    trajs = [t for st in range(bench.N_STEPS_PASS) for t in bench.step_traj(st)]
    assert sorted(trajs) == list(range(bench.N_TEST_TRAJ))
    assert len(bench.step_traj(0)) == bench.TRAJ_PER_STEP


def test_headline_config_names_the_step_it_times():
    import sys
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        args = bench.parse()
    finally:
        sys.argv = argv
    cfg = bench.headline_config(args, 1)
    n = len(bench.WAVELENGTHS) * bench.TRAJ_PER_STEP * bench.TRAJ_STEPS
    assert cfg["solves_per_step"] == n and f"{n} Krylov bases" in cfg["l2"]
    assert cfg["restart"] == 200 and cfg["tol"] == 1e-6 and cfg["maxit"] == 5000
    assert cfg["krylov_basis_storage"] == "FP32 (complex64)"
    assert bench.headline_config(args, 2)["parallelism"] == "replicas x2"


def test_oracle_sample_takes_the_first_problems_of_each_wavelength():
    # The CPU baseline samples the first permittivities of the first timed
    # step at each wavelength (1300 nm solves come first in a step) and keeps
    # the GPU's restart cycles of exactly those solves.
    import numpy as np
    import torch
    from types import SimpleNamespace
    from paper_1902_00090_gb300 import inputs
    grids = [inputs.Grid(nx=8, ny=8, npml=2, i_src=2, sigma_src=1.0, slab_cells=2, wavelength=lam)
             for lam in bench.WAVELENGTHS]
    test_eps = [np.full((bench.TRAJ_STEPS, 8, 8), float(t)) + np.arange(bench.TRAJ_STEPS)[:, None, None] / 100
                for t in range(bench.N_TEST_TRAJ)]
    n_step = len(grids) * bench.TRAJ_PER_STEP * bench.TRAJ_STEPS
    infos = [{"cycles": i, "iters": 10 * i} for i in range(n_step)]
    P = SimpleNamespace(get_params=lambda: np.zeros(3, np.float32), channels=(4,) * 6, k=2)
    U = {g.wavelength: torch.zeros((5, 64), dtype=torch.complex128) for g in grids}
    st0 = 3
    spec = bench.oracle_sample_spec(P, U, test_eps, grids, None, None, [(st0, infos)], U_pca=U,
                                    policy={g.wavelength: (1, 0) for g in grids}, per_wl=4)
    probs = spec["problems"]
    assert len(probs) == 8
    t0 = bench.step_traj(st0)[0]
    n_wl = bench.TRAJ_PER_STEP * bench.TRAJ_STEPS
    for w, g in enumerate(grids):
        for j in range(4):
            p = probs[w * 4 + j]
            assert p["grid"].wavelength == g.wavelength
            assert p["gpu_cycles"] == w * n_wl + j and p["gpu_iters"] == 10 * (w * n_wl + j)
            assert np.array_equal(p["eps"], test_eps[t0][j])
    assert spec["base"][grids[0].wavelength].shape == (2, 64) and spec["pca"][grids[1].wavelength].shape == (5, 64)


def test_solve_records_name_each_problem():
    # The per-solve log (--log-jsonl): solve i of a timed step is wavelength
    # i // (TRAJ_PER_STEP * TRAJ_STEPS), then trajectory, then permittivity.
    import json
    from paper_1902_00090_gb300 import inputs
    grids = [inputs.Grid(nx=8, ny=8, npml=2, i_src=2, sigma_src=1.0, slab_cells=2, wavelength=lam)
             for lam in bench.WAVELENGTHS]
    n_step = len(grids) * bench.TRAJ_PER_STEP * bench.TRAJ_STEPS
    infos = [{"iters": i, "cycles": 1, "converged": 1, "true_rel_residual": 1e-7,
              "first_step_rel_residual": 0.05, "fallback_used": 0, "breakdown": 0} for i in range(n_step)]
    recs = bench.solve_records("cnn", [(5, infos), (6, infos)], [100.0, 200.0], grids)
    assert len(recs) == 2 * n_step
    r = recs[bench.TRAJ_STEPS + 3]       # first wavelength, the step's second trajectory, permittivity 3
    t = bench.N_TRAIN_TRAJ + bench.step_traj(5)[1]
    assert (r["trajectory"], r["permittivity"], r["wavelength_nm"], r["iterations"]) == (t, 3, 1300,
                                                                                         bench.TRAJ_STEPS + 3)
    assert r["seed"] == f"PCG64({1000 * bench.SEED_CONFIG + t})" and r["step_ms"] == 100.0
    last = recs[-1]
    assert last["wavelength_nm"] == 1550 and last["timed_step"] == 1 and last["step"] == 6
    assert last["permittivity"] == bench.TRAJ_STEPS - 1 and last["solves_in_step"] == n_step
    json.dumps(recs)                      # every field serialises
