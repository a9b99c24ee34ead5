"""GPU parity of the subspace-predicting CNN against the oracle (oracle/cnn.py).

The GPU network stores weights and activations in bfloat16 and accumulates in
FP32.  Bars: (1) against the oracle with the same bfloat16 storage (weights
and every stored activation rounded to nearest-even bfloat16): output within
2e-3 relative L2, loss within 1e-4, gradient cosine >= 0.9999; (2) against the
pure fp64 oracle on the same FP32 weights: output within 3e-2 relative L2,
loss within 2 %, gradient cosine >= 0.98 (what bfloat16 storage itself gives);
Adam by its formula applied to the GPU's own gradient (FP32 round-off).
"""
import dataclasses
import os
import tempfile

import numpy as np
import pytest

from oracle import cnn as ocnn
from oracle import fdfd
from paper_1902_00090_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1902_00090_gb300 as ddg  # noqa: E402

SMALL = dict(k=2, channels=(8, 16, 16))


def small_problems(n=2, N=32, seed=0):
    g = inputs.Grid(nx=N, ny=N, npml=4, i_src=6, sigma_src=3.0, slab_cells=4)
    eps = inputs.trajectory_set(g, 2, 1, steps=n) if seed == 0 else \
        inputs.trajectory_set(g, 2, seed + 1, steps=n)[-n:]
    ops = [ddg.fdfd_operator(g, torch.as_tensor(e, device="cuda")) for e in eps]
    return g, eps, ops


def oracle_inputs(g, eps):
    return np.stack([ocnn.input_channels(e, g.wavelength, g.npml, g.i_src, g.sigma_src, g.j_src) for e in eps])


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_layer_order_matches_oracle():
    cfg = ocnn.CNNConfig(cin=4, channels=SMALL["channels"], k=SMALL["k"])
    assert [s[1:] for s in ocnn.layer_shapes(cfg)] == \
        [s[1:] for s in ddg.binding.predictor_layer_shapes(SMALL["channels"], SMALL["k"])]
    P = ddg.Predictor(**SMALL)
    assert P.nparams == ocnn.num_params(cfg)


def test_forward_matches_oracle():
    g, eps, ops = small_problems()
    P = ddg.Predictor(**SMALL)
    P.init_he(seed=3)
    theta = P.get_params().astype(np.float64)
    y = P.forward(ops, (g.i_src, g.sigma_src, g.j_src)).cpu().numpy()
    cfg = ocnn.CNNConfig(cin=4, channels=SMALL["channels"], k=SMALL["k"])
    x = oracle_inputs(g, eps)
    yo = ocnn.forward(cfg, theta, x)
    assert y.shape == yo.shape
    assert rel(y, yo) <= 3e-2
    # same storage precision as the GPU (bfloat16 weights and activations)
    yb = ocnn.forward(cfg, ocnn.round_weights(cfg, theta, ocnn.bf16_round), ocnn.bf16_round(x),
                      store=ocnn.bf16_round)
    assert rel(y, yb) <= 2e-3


def sin_largest_angle(Q, U):
    """Sine of the largest principal angle between span(Q) and span(U) (Q
    orthonormal, U orthonormal columns): ||(I - Q Q^H) U||_2."""
    return np.linalg.norm(U - Q @ (Q.conj().T @ U), 2)


def test_predict_is_orthonormal_and_keeps_the_span():
    # K13: subspace_predict returns the network's k vectors made orthonormal on
    # the device (Cholesky QR twice, FP64); the span is that of the raw output
    g, eps, ops = small_problems()
    P = ddg.Predictor(**SMALL)
    P.init_he(seed=4)
    src = (g.i_src, g.sigma_src, g.j_src)
    y = P.forward(ops, src).cpu().numpy()
    U = P.predict(ops, src)
    cfg = ocnn.CNNConfig(cin=4, channels=SMALL["channels"], k=SMALL["k"])
    theta = P.get_params().astype(np.float64)
    yb = ocnn.forward(cfg, ocnn.round_weights(cfg, theta, ocnn.bf16_round), ocnn.bf16_round(oracle_inputs(g, eps)),
                      store=ocnn.bf16_round)
    for s in range(len(ops)):
        Us = U[s].cpu().numpy().T                     # (D, k): column c = v_c
        assert np.max(np.abs(Us.conj().T @ Us - np.eye(SMALL["k"]))) <= 1e-10
        Q, _ = np.linalg.qr(ocnn.to_complex_fields(y[s:s + 1])[0].astype(np.complex128))
        assert sin_largest_angle(Q, Us) <= 1e-6
        # and the span of the oracle's forward pass (same bfloat16 storage)
        Qo, _ = np.linalg.qr(ocnn.to_complex_fields(yb[s:s + 1])[0])
        assert sin_largest_angle(Qo, Us) <= 2e-2


def test_predict_drops_a_dependent_vector():
    # with a zero head the output is the offset alone: v_3 = v_1 + v_2 is
    # spanned by the first two, so it comes out as a zero vector and the
    # others stay orthonormal with the span of {v_1, v_2}
    g, eps, ops = small_problems()
    P = ddg.Predictor(k=3, channels=SMALL["channels"])
    P.init_he(seed=14)
    P.zero_head()
    a, b = inputs.random_complex(g.D, 21), inputs.random_complex(g.D, 22)
    P.set_output_base(torch.as_tensor(np.stack([a, b, a + b]), device="cuda"), g.nx, g.ny)
    U = P.predict(ops, (g.i_src, g.sigma_src, g.j_src))
    Q, _ = np.linalg.qr(np.stack([a, b], axis=1))
    for Ut in U:
        Us = Ut.cpu().numpy().T
        assert not np.any(Us[:, 2])
        assert np.max(np.abs(Us[:, :2].conj().T @ Us[:, :2] - np.eye(2))) <= 1e-10
        assert sin_largest_angle(Q, Us[:, :2]) <= 1e-6


def test_loss_and_gradient_match_oracle():
    g, eps, ops = small_problems()
    P = ddg.Predictor(**SMALL)
    P.init_he(seed=5)
    theta = P.get_params().astype(np.float64)
    fields = [inputs.random_complex(g.D, 10 + s) for s in range(len(ops))]
    src = (g.i_src, g.sigma_src, g.j_src)
    loss, grad = P.loss_grad(ops, src, [torch.as_tensor(f, device="cuda") for f in fields])
    cfg = ocnn.CNNConfig(cin=4, channels=SMALL["channels"], k=SMALL["k"])
    x = oracle_inputs(g, eps)
    gg = grad.cpu().numpy().astype(np.float64)
    assert 0.0 <= loss <= 1.0
    # (1) the oracle with bfloat16 storage, as the GPU network: tight
    lb, gb = ocnn.batch_loss_and_grad(cfg, ocnn.round_weights(cfg, theta, ocnn.bf16_round), ocnn.bf16_round(x),
                                      np.stack(fields), store=ocnn.bf16_round)
    assert abs(loss - lb) <= 1e-4
    assert gg @ gb / (np.linalg.norm(gg) * np.linalg.norm(gb)) >= 0.9999
    assert rel(gg, gb) <= 1e-2
    # (2) the fp64 oracle: bfloat16 storage (8 significant bits) perturbs a
    # near-unit loss's small gradient by ~15 % here (the emulation above gives
    # the same cosine, 0.988, to eight digits)
    lo, go = ocnn.batch_loss_and_grad(cfg, theta, x, np.stack(fields))
    assert abs(loss - lo) <= 2e-2 * max(lo, 1e-3)
    assert gg @ go / (np.linalg.norm(gg) * np.linalg.norm(go)) >= 0.98


def test_adam_step_matches_formula():
    g, eps, ops = small_problems()
    P = ddg.Predictor(**SMALL)
    P.init_he(seed=6)
    theta0 = P.get_params().astype(np.float64)
    fields = [torch.as_tensor(inputs.random_complex(g.D, 20 + s), device="cuda") for s in range(len(ops))]
    src = (g.i_src, g.sigma_src, g.j_src)
    st = ocnn.AdamState(m=np.zeros_like(theta0), v=np.zeros_like(theta0))
    th = theta0.copy()
    for it in range(3):
        _, grad = P.loss_grad(ops, src, fields)
        P.adam_step(1e-3)
        th = ocnn.adam_step(th, grad.cpu().numpy().astype(np.float64), st, lr=1e-3)
        got = P.get_params().astype(np.float64)
        assert np.max(np.abs(got - th)) <= 1e-6 + 1e-5 * np.max(np.abs(th))


def test_checkpoint_round_trip_and_corruption():
    P = ddg.Predictor(**SMALL)
    P.init_he(seed=7)
    g, eps, ops = small_problems()
    fields = [torch.as_tensor(inputs.random_complex(g.D, 30 + s), device="cuda") for s in range(len(ops))]
    P.train_step(ops, (g.i_src, g.sigma_src, g.j_src), fields, 1e-3)
    theta = P.get_params()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "p.bin")
        P.save(path)
        Q = ddg.Predictor(**SMALL)
        Q.load_file(path)
        assert np.array_equal(Q.get_params(), theta)
        raw = bytearray(open(path, "rb").read())
        raw[200] ^= 0xFF
        open(path, "wb").write(bytes(raw))
        with pytest.raises(ddg.DdgError):
            Q.load_file(path)
        R = ddg.Predictor(k=3, channels=SMALL["channels"])
        P.save(path)
        with pytest.raises(ddg.DdgError):
            R.load_file(path)


def test_training_reduces_loss_and_helps_the_solver():
    # Solved training fields (the library's own solver), a few hundred Adam steps,
    # then the trained predictor's subspace must capture much more of held-out
    # solutions than the untrained one (Eq. 5 on held-out fields, and the
    # V-only residual of Eq. 6 reported by the augmented solver).
    N = 64
    g = inputs.grid_for(N, N)
    eps_tr = inputs.trajectory_set(g, 2, 6, steps=8)
    eps_te = inputs.trajectory_eps(g, 2, 30, steps=4)
    ctx = ddg.Context()
    ctx.set_fallback(2.0)    # compare the two subspaces inside the augmented method
    src = (g.i_src, g.sigma_src, g.j_src)

    def solve(eps_set):
        ops = [ddg.fdfd_operator(g, torch.as_tensor(e, device="cuda")) for e in eps_set]
        bs = [ddg.fdfd_source(op, *src) for op in ops]
        xs, infos, st = ddg.gmres_solve_batched(ctx, ops, bs, tol=1e-6, restart=100, maxit=20000, precision="c64")
        assert st == 0
        return ops, bs, xs

    ops_tr, _, f_tr = solve(eps_tr)
    ops_te, bs_te, f_te = solve(eps_te)
    P = ddg.Predictor(k=4, channels=(16, 32, 32, 48))
    P.init_he(seed=1)
    l_te0, _ = P.loss_grad(ops_te, src, f_te, want_grad=False)
    U0 = P.predict(ops_te, src)
    rng = np.random.default_rng(0)
    losses = []
    for it in range(300):
        idx = rng.choice(len(ops_tr), 8, replace=False)
        losses.append(P.train_step([ops_tr[i] for i in idx], src, [f_tr[i] for i in idx], 2e-3))
    assert np.mean(losses[-20:]) < 0.5 * np.mean(losses[:5])
    l_te1, _ = P.loss_grad(ops_te, src, f_te, want_grad=False)
    assert l_te1 < 0.5 * l_te0, (l_te0, l_te1)
    U1 = P.predict(ops_te, src)
    r0 = [ddg.augmented_gmres_solve(ctx, op, b, U, tol=1e-6, restart=100, maxit=20000, precision="c64")[1]
          for op, b, U in zip(ops_te, bs_te, U0)]
    r1 = [ddg.augmented_gmres_solve(ctx, op, b, U, tol=1e-6, restart=100, maxit=20000, precision="c64")[1]
          for op, b, U in zip(ops_te, bs_te, U1)]
    assert all(i["converged"] for i in r0 + r1)
    first0 = np.mean([i["first_step_rel_residual"] for i in r0])
    first1 = np.mean([i["first_step_rel_residual"] for i in r1])
    assert first1 < 0.7 * first0, (first0, first1)


def test_full_size_network_runs_at_128():
    g = inputs.grid_128()
    eps = inputs.trajectory_set(g, 2, 1, steps=2)
    ops = [ddg.fdfd_operator(g, torch.as_tensor(e, device="cuda")) for e in eps]
    P = ddg.Predictor(k=8)
    P.init_he(seed=0)
    y = P.forward(ops, (g.i_src, g.sigma_src, g.j_src))
    assert y.shape == (2, 128, 128, 16) and torch.isfinite(y).all()


def test_residual_loss_and_gradient_match_oracle():
    g, eps, ops = small_problems()
    P = ddg.Predictor(**SMALL)
    P.init_he(seed=8)
    P.set_loss("residual")
    theta = P.get_params().astype(np.float64)
    src = (g.i_src, g.sigma_src, g.j_src)
    bs = [ddg.fdfd_source(op, *src) for op in ops]
    loss, grad = P.loss_grad(ops, src, bs)
    cfg = ocnn.CNNConfig(cin=4, channels=SMALL["channels"], k=SMALL["k"])
    x = oracle_inputs(g, eps)
    As = [fdfd.operator_for(g, e) for e in eps]
    rhs = [b.cpu().numpy() for b in bs]
    gg = grad.cpu().numpy().astype(np.float64)
    assert 0.0 <= loss <= 1.0
    lb, gb = ocnn.batch_residual_loss_and_grad(cfg, ocnn.round_weights(cfg, theta, ocnn.bf16_round),
                                               ocnn.bf16_round(x), As, rhs, store=ocnn.bf16_round)
    assert abs(loss - lb) <= 1e-3 * max(lb, 1e-2)
    assert gg @ gb / (np.linalg.norm(gg) * np.linalg.norm(gb)) >= 0.999
    lo, go = ocnn.batch_residual_loss_and_grad(cfg, theta, x, As, rhs)
    assert abs(loss - lo) <= 2e-2 * max(lo, 1e-2)
    assert gg @ go / (np.linalg.norm(gg) * np.linalg.norm(go)) >= 0.98


TC = dict(k=2, channels=(16, 32, 48))   # every 3x3 layer but the first takes the tensor-core path


def test_tensor_core_convolutions_match_oracle():
    # channel counts that are multiples of 16: the forward 3x3 convolutions run
    # on tcgen05 (BF16 x BF16, FP32 in tensor memory); same bars as the CUDA-core
    # forward against the bfloat16-emulated and the fp64 oracle
    g, eps, ops = small_problems(n=3)
    P = ddg.Predictor(**TC)
    P.init_he(seed=11)
    theta = P.get_params().astype(np.float64)
    y = P.forward(ops, (g.i_src, g.sigma_src, g.j_src)).cpu().numpy()
    cfg = ocnn.CNNConfig(cin=4, channels=TC["channels"], k=TC["k"])
    x = oracle_inputs(g, eps)
    yb = ocnn.forward(cfg, ocnn.round_weights(cfg, theta, ocnn.bf16_round), ocnn.bf16_round(x),
                      store=ocnn.bf16_round)
    assert rel(y, yb) <= 2e-3
    assert rel(y, ocnn.forward(cfg, theta, x)) <= 3e-2


def test_tensor_core_forward_equals_cuda_core_forward():
    # the full-size network at 128x128 on both convolution paths: equal up to
    # FP32 summation order (and the BF16 roundings it flips)
    g = inputs.grid_128()
    eps = inputs.trajectory_set(g, 2, 1, steps=3)
    ops = [ddg.fdfd_operator(g, torch.as_tensor(e, device="cuda")) for e in eps]
    P = ddg.Predictor(k=8)
    P.init_he(seed=2)
    src = (g.i_src, g.sigma_src, g.j_src)
    y_tc = P.forward(ops, src).cpu().numpy()
    P.set_tensor_cores(False)
    y_cc = P.forward(ops, src).cpu().numpy()
    P.set_tensor_cores(True)
    y_tc2 = P.forward(ops, src).cpu().numpy()
    assert np.array_equal(y_tc, y_tc2)          # deterministic
    assert rel(y_tc, y_cc) <= 1e-2


def test_tma_tile_forward_equals_gather_forward():
    # the full-size network at 128x128: the plain-input layers of levels 0-3
    # (Ci, Co of 32, 48, 64, 96) load their tiles by TMA and read the taps by
    # descriptor offsets; the others keep the gather.  Same K order as the
    # gather path, so the same FP32 accumulation up to the tensor core's own
    # order; checked against the gather-only forward, twice for determinism.
    g = inputs.grid_128()
    eps = inputs.trajectory_set(g, 2, 1, steps=5)
    ops = [ddg.fdfd_operator(g, torch.as_tensor(e, device="cuda")) for e in eps]
    P = ddg.Predictor(k=8)
    P.init_he(seed=4)
    src = (g.i_src, g.sigma_src, g.j_src)
    y_tma = P.forward(ops, src).cpu().numpy()
    y_tma2 = P.forward(ops, src).cpu().numpy()
    P.set_tensor_cores(True, tma=False)
    y_g = P.forward(ops, src).cpu().numpy()
    assert np.array_equal(y_tma, y_tma2)
    print(f"TMA-tile forward vs gather: bitwise equal {np.array_equal(y_tma, y_g)}, rel {rel(y_tma, y_g):.2e}")
    assert rel(y_tma, y_g) <= 1e-6


def test_input_field_network_matches_oracle():
    # a network with the approximate-field input (6 channels): forward against
    # the bfloat16-emulated oracle given the same field; without the field set,
    # the call is refused
    g, eps, ops = small_problems()
    P = ddg.Predictor(input_field=True, **SMALL)
    P.init_he(seed=12)
    src = (g.i_src, g.sigma_src, g.j_src)
    with pytest.raises(ddg.DdgError):
        P.forward(ops, src)
    f = inputs.random_complex(g.D, 77)
    P.set_input_field(torch.as_tensor(f, device="cuda"), g.nx, g.ny)
    theta = P.get_params().astype(np.float64)
    y = P.forward(ops, src).cpu().numpy()
    cfg = ocnn.CNNConfig(cin=6, channels=SMALL["channels"], k=SMALL["k"])
    assert P.nparams == ocnn.num_params(cfg)
    x = np.stack([ocnn.input_channels(e, g.wavelength, g.npml, g.i_src, g.sigma_src, g.j_src, field=f) for e in eps])
    yb = ocnn.forward(cfg, ocnn.round_weights(cfg, theta, ocnn.bf16_round), ocnn.bf16_round(x),
                      store=ocnn.bf16_round)
    assert rel(y, yb) <= 2e-3
    # a checkpoint of this network does not load into one without the field input
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "p.bin")
        P.save(path)
        Q = ddg.Predictor(**SMALL)
        with pytest.raises(ddg.DdgError):
            Q.load_file(path)


def test_output_base_is_added():
    # the fixed output offset: y = scale * base + network output (output layout
    # [pixel][2k], channel 2c / 2c + 1 = Re / Im of vector c); with a zero head
    # the output is the base alone, and removing the base restores the network
    g, eps, ops = small_problems()
    P = ddg.Predictor(**SMALL)
    P.init_he(seed=13)
    src = (g.i_src, g.sigma_src, g.j_src)
    y0 = P.forward(ops, src).cpu().numpy()
    k = SMALL["k"]
    Uh = inputs.random_complex(g.D, 5, shape=(k, g.D))
    P.set_output_base(torch.as_tensor(Uh, device="cuda"), g.nx, g.ny, scale=3.0)
    y1 = P.forward(ops, src).cpu().numpy()
    base = np.zeros((g.ny, g.nx, 2 * k), dtype=np.float32)
    base[..., 0::2] = (3.0 * Uh.real.T).reshape(g.ny, g.nx, k)
    base[..., 1::2] = (3.0 * Uh.imag.T).reshape(g.ny, g.nx, k)
    assert np.max(np.abs(y1 - (y0 + base[None]))) <= 1e-6 * np.max(np.abs(y0) + np.abs(base))
    P.zero_head()
    assert np.array_equal(P.forward(ops, src).cpu().numpy(), np.broadcast_to(base, y1.shape))
    P.set_output_base(None, g.nx, g.ny)
    assert not np.any(P.forward(ops, src).cpu().numpy())


def test_output_base_per_wavelength():
    # offsets keyed by wavelength serve the problems at that wavelength; an
    # offset for every wavelength serves the rest; a problem with neither is
    # refused
    g, eps, _ = small_problems()
    g2 = dataclasses.replace(g, wavelength=1300e-9)
    ops = [ddg.fdfd_operator(g, torch.as_tensor(eps[0], device="cuda")),
           ddg.fdfd_operator(g2, torch.as_tensor(eps[1], device="cuda"))]
    P = ddg.Predictor(**SMALL)
    P.init_he(seed=15)
    P.zero_head()
    k = SMALL["k"]
    U13 = inputs.random_complex(g.D, 31, shape=(k, g.D))
    Uany = inputs.random_complex(g.D, 32, shape=(k, g.D))
    src = (g.i_src, g.sigma_src, g.j_src)
    P.set_output_base(torch.as_tensor(U13, device="cuda"), g.nx, g.ny, wavelength=1300e-9)
    with pytest.raises(ddg.DdgError):
        P.forward(ops, src)          # the 1550 nm problem has no offset
    P.set_output_base(torch.as_tensor(Uany, device="cuda"), g.nx, g.ny)

    def layout(Uh):
        base = np.zeros((g.ny, g.nx, 2 * k), dtype=np.float32)
        base[..., 0::2] = Uh.real.T.reshape(g.ny, g.nx, k)
        base[..., 1::2] = Uh.imag.T.reshape(g.ny, g.nx, k)
        return base

    y = P.forward(ops, src).cpu().numpy()
    assert np.array_equal(y[0], layout(Uany)) and np.array_equal(y[1], layout(U13))



def test_tensor_core_backward_matches_oracle():
    # the backward convolutions (data and weight gradients) on tcgen05
    # (predictor_set_tensor_cores bit 2): the masked output gradient enters
    # both products in bfloat16.  Against the oracle with the same storage
    # (activations and, in every layer but the first, whose weight gradient
    # stays on CUDA cores, the masked gradient rounded to bfloat16), and
    # against the CUDA-core backward pass of the same network.
    chans = (16, 32, 32)
    g, eps, ops = small_problems()
    P = ddg.Predictor(k=2, channels=chans)
    P.init_he(seed=17)
    theta = P.get_params().astype(np.float64)
    fields = [inputs.random_complex(g.D, 40 + s) for s in range(len(ops))]
    src = (g.i_src, g.sigma_src, g.j_src)
    fd = [torch.as_tensor(f, device="cuda") for f in fields]
    P.set_tensor_cores(True)
    loss_cc, grad_cc = P.loss_grad(ops, src, fd)
    P.set_tensor_cores(True, backward=True)
    loss_tc, grad_tc = P.loss_grad(ops, src, fd)
    assert loss_tc == loss_cc                       # the forward pass is the same
    cfg = ocnn.CNNConfig(cin=4, channels=chans, k=2)
    x = oracle_inputs(g, eps)
    lb, gb = ocnn.batch_loss_and_grad(cfg, ocnn.round_weights(cfg, theta, ocnn.bf16_round), ocnn.bf16_round(x),
                                      np.stack(fields), store=ocnn.bf16_round,
                                      gstore=lambda name, gg: gg if name == "enc0a" else ocnn.bf16_round(gg))
    gt = grad_tc.cpu().numpy().astype(np.float64)
    gc = grad_cc.cpu().numpy().astype(np.float64)
    assert abs(loss_tc - lb) <= 1e-4
    assert gt @ gb / (np.linalg.norm(gt) * np.linalg.norm(gb)) >= 0.9999
    assert rel(gt, gb) <= 1e-2
    assert gt @ gc / (np.linalg.norm(gt) * np.linalg.norm(gc)) >= 0.999
