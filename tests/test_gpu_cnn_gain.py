"""What the trained network gains over the method without it (the paper's
claim for the CNN predictor, Sec. III and Fig. 3; measured here on held-out
problems of the 128x128 trajectory set).

The predictor starts as its output offset alone (the 8 leading principal
components of solved training fields, zero head) and is trained with the
residual loss (Eq. 6) on the training problems' right-hand sides.  On 32
held-out problems (two trajectories the training never saw), data-driven
GMRES(200) with the trained network's subspace in its first restart cycle
must (a) cut the first-step residual (Eq. 6's minimum over the subspace) well
below what the untrained offset gives, (b) take fewer Krylov steps than plain
GMRES, and (c) no more steps than the offset alone.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1902_00090_gb300 as ddg  # noqa: E402
from paper_1902_00090_gb300 import inputs  # noqa: E402


def test_trained_network_beats_plain_gmres_and_its_offset():
    g = inputs.grid_128()
    src = (g.i_src, g.sigma_src, g.j_src)
    eps = inputs.trajectory_set(g, 2, 32)
    train, test = eps[:448], eps[-32:]
    ops_tr = [ddg.fdfd_operator(g, torch.as_tensor(e, device="cuda")) for e in train]
    ops_te = [ddg.fdfd_operator(g, torch.as_tensor(e, device="cuda")) for e in test]
    b = ddg.fdfd_source(ops_tr[0], *src)
    ctx = ddg.Context()
    ctx.set_augmented_policy(1, keep=0)      # the subspace in the first cycle, then plain GMRES
    xs, inf, st = ddg.gmres_solve_batched(ctx, ops_tr[::14], [b] * 32, tol=1e-6, restart=200, maxit=5000,
                                          precision="c64")
    assert st == 0
    U8, _ = ddg.pca_fit(ctx, torch.stack(xs), 8)
    P = ddg.Predictor(k=8)
    P.init_he(seed=0)
    P.set_output_base(U8, g.nx, g.ny, scale=float(np.sqrt(g.D)))
    P.zero_head()
    P.set_loss("residual")

    def solve_with(U):
        _, infos, st = ddg.augmented_gmres_solve_batched(ctx, ops_te, [b] * len(ops_te), U, tol=1e-6, restart=200,
                                                         maxit=5000, precision="c64")
        assert st == 0
        return (float(np.mean([i["iters"] for i in infos])),
                float(np.mean([i["first_step_rel_residual"] for i in infos])))

    it_off, fs_off = solve_with(P.predict(ops_te, src))          # the offset alone (untrained)
    rng = np.random.default_rng(0)
    for _ in range(600):
        idx = rng.choice(len(ops_tr), 16, replace=False)
        P.train_step([ops_tr[i] for i in idx], src, [b] * 16, 3e-4)
    it_cnn, fs_cnn = solve_with(P.predict(ops_te, src))
    _, inf_p, st = ddg.gmres_solve_batched(ctx, ops_te, [b] * len(ops_te), tol=1e-6, restart=200, maxit=5000,
                                           precision="c64")
    it_plain = float(np.mean([i["iters"] for i in inf_p]))
    print(f"held-out steps: plain {it_plain:.1f}, offset {it_off:.1f} (first step {fs_off:.4f}), "
          f"trained {it_cnn:.1f} (first step {fs_cnn:.4f})")
    assert fs_cnn <= 0.8 * fs_off
    assert it_cnn < 0.9 * it_plain
    assert it_cnn <= it_off
