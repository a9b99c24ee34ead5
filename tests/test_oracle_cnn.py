"""Pins of the oracle CNN, projection loss (Eq. 5) and Adam."""
import numpy as np
import pytest
import scipy.signal

from oracle import cnn, losses


def test_conv3x3_matches_library_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 7, 9, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = cnn.conv3x3(x, w, b)
    for bb in range(2):
        for co in range(4):
            ref = b[co] + sum(scipy.signal.correlate2d(x[bb, :, :, ci], w[co, ci], mode="same")
                              for ci in range(3))
            assert np.allclose(y[bb, :, :, co], ref, atol=1e-12)


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 8, 6, 3))
    g = rng.standard_normal((2, 4, 3, 3))
    assert np.isclose(np.sum(cnn.avgpool2(x) * g), np.sum(x * cnn.avgpool2_backward(g)))
    u = rng.standard_normal((2, 4, 3, 3))
    G = rng.standard_normal((2, 8, 6, 3))
    assert np.isclose(np.sum(cnn.upsample2(u) * G), np.sum(u * cnn.upsample2_backward(G)))


def test_conv_backward_is_adjoint_and_gradient():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 5, 6, 3))
    w = rng.standard_normal((2, 3, 3, 3))
    b = rng.standard_normal(2)
    gy = rng.standard_normal((1, 5, 6, 2))
    gx, gw, gb = cnn.conv3x3_backward(x, w, gy)
    # <conv(x) - b, gy> is linear in x and in w
    f = lambda xx, ww: np.sum((cnn.conv3x3(xx, ww, 0 * b)) * gy)
    assert np.isclose(f(x, w), np.sum(x * gx))
    assert np.isclose(f(x, w), np.sum(w * gw))
    assert np.allclose(gb, gy.sum(axis=(0, 1, 2)))


def small_cfg():
    return cnn.CNNConfig(cin=4, channels=(4, 6, 5), k=2)


def test_network_gradient_finite_differences():
    cfg = small_cfg()
    rng = np.random.default_rng(3)
    theta = 0.3 * rng.standard_normal(cnn.num_params(cfg))
    x = rng.standard_normal((2, 8, 8, 4))
    gy = rng.standard_normal((2, 8, 8, 2 * cfg.k))
    y, cache = cnn.forward(cfg, theta, x, keep=True)
    g, _ = cnn.backward(cfg, theta, cache, gy)
    L = lambda th: np.sum(cnn.forward(cfg, th, x) * gy)
    for idx in rng.choice(theta.size, 25, replace=False):
        e = np.zeros_like(theta)
        e[idx] = 1e-6
        fd = (L(theta + e) - L(theta - e)) / 2e-6
        assert abs(fd - g[idx]) <= 1e-5 * max(1.0, abs(fd)), (idx, fd, g[idx])


def test_projection_loss_value_and_gradient():
    rng = np.random.default_rng(4)
    D, k = 40, 3
    V = rng.standard_normal((D, k)) + 1j * rng.standard_normal((D, k))
    f = rng.standard_normal(D) + 1j * rng.standard_normal(D)
    l, gr, gi = cnn.projection_loss_and_grad(V, f)
    assert abs(l - losses.projection_loss(V, f)) <= 1e-12     # Eq. 5 by lstsq
    for _ in range(10):
        r, c = rng.integers(D), rng.integers(k)
        for part, g in ((1.0, gr), (1j, gi)):
            dV = np.zeros_like(V)
            dV[r, c] = 1e-7 * part
            fd = (cnn.projection_loss_and_grad(V + dV, f)[0] - cnn.projection_loss_and_grad(V - dV, f)[0]) / 2e-7
            assert abs(fd - g[r, c]) <= 1e-6 * max(1.0, abs(fd))


def test_batch_loss_gradient_finite_differences():
    cfg = small_cfg()
    rng = np.random.default_rng(5)
    theta = 0.3 * rng.standard_normal(cnn.num_params(cfg))
    x = rng.standard_normal((2, 8, 8, 4))
    fields = rng.standard_normal((2, 64)) + 1j * rng.standard_normal((2, 64))
    l, g = cnn.batch_loss_and_grad(cfg, theta, x, fields)
    assert 0.0 <= l <= 1.0
    for idx in rng.choice(theta.size, 15, replace=False):
        e = np.zeros_like(theta)
        e[idx] = 1e-6
        fd = (cnn.batch_loss_and_grad(cfg, theta + e, x, fields)[0]
              - cnn.batch_loss_and_grad(cfg, theta - e, x, fields)[0]) / 2e-6
        assert abs(fd - g[idx]) <= 1e-5 * max(1e-2, abs(fd)), (idx, fd, g[idx])


def test_adam_three_steps_by_hand():
    theta = np.array([1.0, -2.0])
    st = cnn.AdamState(m=np.zeros(2), v=np.zeros(2))
    gs = [np.array([0.5, -1.0]), np.array([0.1, 2.0]), np.array([-0.3, 0.0])]
    th = theta.copy()
    m = np.zeros(2)
    v = np.zeros(2)
    for t, g in enumerate(gs, start=1):
        th_o = cnn.adam_step(theta, g, st, lr=0.01)
        theta = th_o
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g * g
        th = th - 0.01 * (m / (1 - 0.9 ** t)) / (np.sqrt(v / (1 - 0.999 ** t)) + 1e-8)
        assert np.allclose(theta, th, rtol=0, atol=1e-15)
    # first step moves every coordinate with non-zero gradient by ~lr
    st2 = cnn.AdamState(m=np.zeros(2), v=np.zeros(2))
    t1 = cnn.adam_step(np.zeros(2), np.array([3.0, -7.0]), st2, lr=0.01)
    assert np.allclose(t1, [-0.01, 0.01], atol=1e-9)


def test_layer_shapes_and_param_count():
    cfg = cnn.CNNConfig()
    names = [s[0] for s in cnn.layer_shapes(cfg)]
    assert names[0] == "enc0a" and names[-1] == "head" and len(names) == 23
    d = dict((s[0], s[1:]) for s in cnn.layer_shapes(cfg))
    assert d["dec4a"] == (128, 256, 3) and d["dec0a"] == (32, 80, 3) and d["head"] == (16, 32, 1)


def test_bf16_rounding_definition():
    # bfloat16 keeps 8 significant bits; ties go to even
    assert cnn.bf16_round(1.0) == 1.0
    assert cnn.bf16_round(1.0 + 2.0 ** -8) == 1.0            # tie -> even (1.0)
    assert cnn.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6   # tie -> even mantissa
    assert cnn.bf16_round(1.0 + 2.0 ** -7) == 1.0 + 2.0 ** -7
    x = np.random.default_rng(0).standard_normal(1000)
    r = cnn.bf16_round(x)
    assert np.max(np.abs(r - x) / np.abs(x)) <= 2.0 ** -8


def test_residual_loss_value_and_gradient():
    from oracle import fdfd
    from paper_1902_00090_gb300 import inputs
    g = inputs.Grid(nx=12, ny=10, npml=3, i_src=3, sigma_src=2.0, slab_cells=2)
    rng = np.random.default_rng(6)
    A = fdfd.operator_for(g, inputs.background_eps(g) + rng.random((g.ny, g.nx)))
    b = fdfd.source_for(g)
    V = rng.standard_normal((g.D, 3)) + 1j * rng.standard_normal((g.D, 3))
    l, gr, gi = cnn.residual_loss_and_grad(A, V, b)
    assert abs(l - losses.residual_loss(A, V, b)) <= 1e-12          # Eq. 6 by lstsq
    for _ in range(12):
        r, c = rng.integers(g.D), rng.integers(3)
        for part, gg in ((1.0, gr), (1j, gi)):
            dV = np.zeros_like(V)
            dV[r, c] = 1e-7 * part
            fd = (cnn.residual_loss_and_grad(A, V + dV, b)[0] - cnn.residual_loss_and_grad(A, V - dV, b)[0]) / 2e-7
            assert abs(fd - gg[r, c]) <= 1e-6 * max(1.0, abs(fd))


def test_input_field_channels():
    # the approximate-field input: two more channels, Re and Im of the field
    # divided by its largest magnitude; the first four unchanged
    rng = np.random.default_rng(3)
    eps = 2.1 + 10.15 * rng.random((16, 12))
    f = rng.standard_normal(16 * 12) + 1j * rng.standard_normal(16 * 12)
    x4 = cnn.input_channels(eps, 1.55e-6, 2, 3, 2.0, 8.0)
    x6 = cnn.input_channels(eps, 1.55e-6, 2, 3, 2.0, 8.0, field=f)
    assert x6.shape == (16, 12, 6) and np.array_equal(x6[..., :4], x4)
    g = f.reshape(16, 12) / np.max(np.abs(f))
    assert np.array_equal(x6[..., 4], g.real) and np.array_equal(x6[..., 5], g.imag)
    assert np.isclose(np.max(np.hypot(x6[..., 4], x6[..., 5])), 1.0)


def test_gradient_storage_hook_replaces_the_product_operand_only():
    # gstore(name, g) replaces the masked output gradient in that layer's input
    # and weight gradients, not in its bias gradient: the identity gives the
    # plain backward pass bitwise; zeroing it at the first layer the backward
    # pass meets (dec0b) zeroes every gradient below that layer and its own
    # weights' gradient, and leaves its bias gradient and the head's unchanged
    cfg = small_cfg()
    rng = np.random.default_rng(7)
    theta = rng.standard_normal(cnn.num_params(cfg)) * 0.3
    x = rng.standard_normal((2, 8, 8, cfg.cin))
    y, cache = cnn.forward(cfg, theta, x, keep=True)
    gy = rng.standard_normal(y.shape)
    g0, _ = cnn.backward(cfg, theta, cache, gy)
    g1, _ = cnn.backward(cfg, theta, cache, gy, gstore=lambda name, g: g)
    assert np.array_equal(g0, g1)
    g2, _ = cnn.backward(cfg, theta, cache, gy,
                         gstore=lambda name, g: np.zeros_like(g) if name == "dec0b" else g)
    off = 0
    for name, co, ci, kk in cnn.layer_shapes(cfg):
        nw = co * ci * kk * kk
        if name == "head":
            assert np.array_equal(g2[off:off + nw + co], g0[off:off + nw + co])
        elif name == "dec0b":
            assert not np.any(g2[off:off + nw])
            assert np.array_equal(g2[off + nw:off + nw + co], g0[off + nw:off + nw + co])
        else:
            assert not np.any(g2[off:off + nw + co]), name
        off += nw + co
