"""Oracle subspace-predicting CNN, projection loss and Adam (fp64 numpy).

TEST INFRASTRUCTURE ONLY.

Sec. III ("Convolutional neural network", Fig. 3a): a convolutional network
maps the permittivity (plus cheap input channels) to N vectors v_1..v_N that
span the predicted subspace; complex quantities are carried as pairs of real
channels (Methods).  The paper does not give the architecture; this is the
encoder-decoder used throughout the library:

  * `levels` resolutions; at level l two 3x3 convolutions (zero padding) with
    bias, each followed by ReLU, `ch[l]` output channels;
  * between encoder levels a 2x2 average pool; in the decoder a nearest 2x
    upsampling whose output is concatenated (upsampled channels first) with the
    encoder output of the same level, then two 3x3 convolutions + ReLU;
  * a final 1x1 convolution with bias to 2k channels; channel pair (2c, 2c+1)
    is (Re, Im) of v_c.

Tensors are NHWC: (batch, ny, nx, channels).  Conv weights are (Cout, Cin, 3, 3)
with w[co, ci, dy+1, dx+1] multiplying x[y+dy, x+dx, ci]; biases (Cout,).

Projection loss (Eq. 5) of one sample with V (D x k complex) and field f:
    l = min over z of ||V z - f||^2 / ||f||^2 = 1 - a^H G^-1 a / ||f||^2,
    a = V^H f, G = V^H V.
Its Wirtinger gradient is dl/d(conj V) = -(f - V z) z^H / ||f||^2 with
z = G^-1 a, so dl/dRe V = 2 Re(.), dl/dIm V = 2 Im(.).

Adam (Kingma & Ba, 2015, Algorithm 1) with bias correction.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


# ---------------------------------------------------------------- layers
def conv3x3(x, w, b):
    """x (B, H, W, Ci), w (Co, Ci, 3, 3), b (Co,) -> (B, H, W, Co); zero padding."""
    B, H, W, Ci = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    out = np.zeros((B, H, W, w.shape[0]))
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, dy:dy + H, dx:dx + W, :]
            out += patch @ w[:, :, dy, dx].T
    return out + b


def conv3x3_backward(x, w, gout, gout_stored=None):
    """Gradients of conv3x3 w.r.t. x, w and b given d loss / d out.
    gout_stored (optional) replaces gout in the gradients w.r.t. x and w (a
    storage emulation, e.g. gout rounded to bfloat16); the bias gradient
    always sums gout itself."""
    B, H, W, Ci = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    gw = np.zeros_like(w)
    gxp = np.zeros_like(xp)
    gd = gout if gout_stored is None else gout_stored
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, dy:dy + H, dx:dx + W, :]
            gw[:, :, dy, dx] = np.einsum("bhwo,bhwi->oi", gd, patch)
            gxp[:, dy:dy + H, dx:dx + W, :] += gd @ w[:, :, dy, dx]
    gb = gout.sum(axis=(0, 1, 2))
    return gxp[:, 1:-1, 1:-1, :], gw, gb


def conv1x1(x, w, b):
    """x (B, H, W, Ci), w (Co, Ci), b (Co,)."""
    return x @ w.T + b


def avgpool2(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def avgpool2_backward(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) / 4.0


def upsample2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample2_backward(g):
    B, H, W, C = g.shape
    return g.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def relu(x):
    return np.maximum(x, 0.0)


def bf16_round(x):
    """Round to the nearest bfloat16 (the upper 16 bits of an IEEE binary32,
    round to nearest, ties to even); returns float64.  Used to emulate a
    network that stores weights and activations in bfloat16."""
    a = np.ascontiguousarray(x, dtype=np.float32).copy()
    u = a.view(np.uint32)
    r = ((u + np.uint32(0x7FFF) + ((u >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def round_weights(cfg, theta, rnd):
    """theta with every weight (not the biases) passed through rnd."""
    out = np.array(theta, dtype=np.float64)
    off = 0
    for _, co, ci, kk in layer_shapes(cfg):
        nw = co * ci * kk * kk
        out[off:off + nw] = rnd(out[off:off + nw])
        off += nw + co
    return out


# ---------------------------------------------------------------- network
@dataclass
class CNNConfig:
    cin: int = 4
    channels: tuple = (32, 48, 64, 96, 128, 128)
    k: int = 8                       # complex output fields

    @property
    def levels(self):
        return len(self.channels)


def layer_shapes(cfg: CNNConfig):
    """(name, Cout, Cin, kernel) in the canonical parameter order: encoder
    levels 0..L-1 (a, b), decoder levels L-2..0 (a, b), head."""
    ch = cfg.channels
    L = cfg.levels
    shapes = []
    for l in range(L):
        shapes.append((f"enc{l}a", ch[l], cfg.cin if l == 0 else ch[l - 1], 3))
        shapes.append((f"enc{l}b", ch[l], ch[l], 3))
    for l in range(L - 2, -1, -1):
        shapes.append((f"dec{l}a", ch[l], ch[l + 1] + ch[l], 3))
        shapes.append((f"dec{l}b", ch[l], ch[l], 3))
    shapes.append(("head", 2 * cfg.k, ch[0], 1))
    return shapes


def num_params(cfg: CNNConfig) -> int:
    n = 0
    for _, co, ci, kk in layer_shapes(cfg):
        n += co * ci * kk * kk + co
    return n


def unpack_params(cfg: CNNConfig, theta: np.ndarray):
    """Flat vector -> dict name -> (w, b).  Order per layer: weights (Co, Ci, k, k)
    row-major, then bias (Co,)."""
    out = {}
    off = 0
    for name, co, ci, kk in layer_shapes(cfg):
        nw = co * ci * kk * kk
        w = theta[off:off + nw].reshape(co, ci, kk, kk) if kk == 3 else theta[off:off + nw].reshape(co, ci)
        off += nw
        b = theta[off:off + co]
        off += co
        out[name] = (w, b)
    assert off == theta.size
    return out


def forward(cfg: CNNConfig, theta, x, keep=False, store=None):
    """x (B, H, W, cin) -> output (B, H, W, 2k); with keep, also the cache.
    store (optional) is applied to every stored activation (e.g. bf16_round)."""
    st = store if store is not None else (lambda z: z)
    P = unpack_params(cfg, theta)
    L = cfg.levels
    cache = {"x": x}
    h = x
    skips = []
    for l in range(L):
        if l > 0:
            h = st(avgpool2(h))
        cache[f"in_enc{l}a"] = h
        h = st(relu(conv3x3(h, *P[f"enc{l}a"])))
        cache[f"out_enc{l}a"] = h
        h = st(relu(conv3x3(h, *P[f"enc{l}b"])))
        cache[f"out_enc{l}b"] = h
        skips.append(h)
    for l in range(L - 2, -1, -1):
        u = upsample2(h)
        cat = np.concatenate([u, skips[l]], axis=-1)
        cache[f"in_dec{l}a"] = cat
        h = st(relu(conv3x3(cat, *P[f"dec{l}a"])))
        cache[f"out_dec{l}a"] = h
        h = st(relu(conv3x3(h, *P[f"dec{l}b"])))
        cache[f"out_dec{l}b"] = h
    cache["in_head"] = h
    y = conv1x1(h, *P["head"])
    return (y, cache) if keep else y


def backward(cfg: CNNConfig, theta, cache, gy, gstore=None):
    """Gradient of the loss w.r.t. the flat parameter vector given dL/dy.
    gstore (optional): gstore(layer name, g) is the value of the masked output
    gradient g that enters that 3x3 layer's input and weight gradients (a
    storage emulation; the bias gradient always sums g itself)."""
    gs = gstore if gstore is not None else (lambda name, g: g)

    def conv_back(x, name, g):
        return conv3x3_backward(x, P[name][0], g, gs(name, g))

    P = unpack_params(cfg, theta)
    L = cfg.levels
    grads = {}
    wh, bh = P["head"]
    h = cache["in_head"]
    grads["head"] = (np.einsum("bhwo,bhwi->oi", gy, h), gy.sum(axis=(0, 1, 2)))
    gh = gy @ wh
    gskips = [None] * L
    # walk the decoder backwards: the forward order was l = L-2 ... 0
    for l in range(0, L - 1):
        gh = gh * (cache[f"out_dec{l}b"] > 0)
        gx, gw, gb = conv_back(cache[f"out_dec{l}a"], f"dec{l}b", gh)
        grads[f"dec{l}b"] = (gw, gb)
        gh = gx * (cache[f"out_dec{l}a"] > 0)
        gx, gw, gb = conv_back(cache[f"in_dec{l}a"], f"dec{l}a", gh)
        grads[f"dec{l}a"] = (gw, gb)
        cu = cfg.channels[l + 1]
        gskips[l] = gx[..., cu:]
        gh = upsample2_backward(gx[..., :cu])
    # encoder backwards: bottleneck level L-1 receives gh (from the decoder)
    for l in range(L - 1, -1, -1):
        if l < L - 1:
            gh = gh + gskips[l]
        gh = gh * (cache[f"out_enc{l}b"] > 0)
        gx, gw, gb = conv_back(cache[f"out_enc{l}a"], f"enc{l}b", gh)
        grads[f"enc{l}b"] = (gw, gb)
        gh = gx * (cache[f"out_enc{l}a"] > 0)
        gx, gw, gb = conv_back(cache[f"in_enc{l}a"], f"enc{l}a", gh)
        grads[f"enc{l}a"] = (gw, gb)
        gh = avgpool2_backward(gx) if l > 0 else gx
    flat = []
    for name, co, ci, kk in layer_shapes(cfg):
        gw, gb = grads[name]
        flat.append(gw.reshape(-1))
        flat.append(gb.reshape(-1))
    return np.concatenate(flat), gh


def to_complex_fields(y):
    """(B, H, W, 2k) -> (B, D, k) complex."""
    B, H, W, C = y.shape
    y = y.reshape(B, H * W, C)
    return y[..., 0::2] + 1j * y[..., 1::2]


# ---------------------------------------------------------------- loss
def projection_loss_and_grad(V: np.ndarray, f: np.ndarray):
    """Eq. 5 for one sample: V (D, k) complex, f (D,) complex ->
    (loss, dl/dRe V, dl/dIm V)."""
    a = V.conj().T @ f
    G = V.conj().T @ V
    z = np.linalg.solve(G, a)
    F = np.vdot(f, f).real
    loss = 1.0 - np.vdot(a, z).real / F
    wb = -np.outer(f - V @ z, z.conj()) / F        # dl / d conj(V)
    return loss, 2.0 * wb.real, 2.0 * wb.imag


def batch_loss_and_grad(cfg: CNNConfig, theta, x, fields, store=None, gstore=None):
    """Mean projection loss over the batch and its gradient w.r.t. theta."""
    y, cache = forward(cfg, theta, x, keep=True, store=store)
    V = to_complex_fields(y)
    B = x.shape[0]
    gy = np.zeros_like(y)
    tot = 0.0
    for s in range(B):
        l, gr, gi = projection_loss_and_grad(V[s], fields[s])
        tot += l
        g = np.zeros((V.shape[1], 2 * cfg.k))
        g[:, 0::2] = gr
        g[:, 1::2] = gi
        gy[s] = g.reshape(y.shape[1:]) / B
    gtheta, _ = backward(cfg, theta, cache, gy, gstore=gstore)
    return tot / B, gtheta


# ---------------------------------------------------------------- Adam
@dataclass
class AdamState:
    m: np.ndarray
    v: np.ndarray
    t: int = 0


def adam_step(theta, g, st: AdamState, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    st.t += 1
    st.m = b1 * st.m + (1 - b1) * g
    st.v = b2 * st.v + (1 - b2) * g * g
    mh = st.m / (1 - b1 ** st.t)
    vh = st.v / (1 - b2 ** st.t)
    return theta - lr * mh / (np.sqrt(vh) + eps)


# ---------------------------------------------------------------- inputs
def input_channels(eps: np.ndarray, wavelength: float, npml: int, src_col: int, sigma: float, j_c: float,
                   field: np.ndarray = None):
    """Network input (ny, nx, 4): normalised permittivity, wavelength, PML mask,
    source profile; with `field` (an approximate field of the grid, ny*nx
    complex) two more channels, its real and imaginary parts divided by its
    largest magnitude (ny, nx, 6)."""
    ny, nx = eps.shape
    x = np.zeros((ny, nx, 4 if field is None else 6))
    if field is not None:
        f = np.asarray(field, dtype=np.complex128).reshape(ny, nx)
        f = f / np.max(np.abs(f))
        x[..., 4] = f.real
        x[..., 5] = f.imag
    x[..., 0] = (eps - 2.1) / 10.15
    x[..., 1] = (wavelength - 1.3e-6) / 0.25e-6
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    inside = (i >= npml) & (i < nx - npml) & (j >= npml) & (j < ny - npml)
    x[..., 2] = np.where(inside, 0.0, 1.0)
    x[..., 3][:, src_col] = np.exp(-((np.arange(ny) - j_c) ** 2) / (2 * sigma * sigma))
    return x


# ---------------------------------------------------------------- residual loss (Eq. 6)
def residual_loss_and_grad(A, V: np.ndarray, b: np.ndarray):
    """Eq. 6 for one sample: l = min over z of ||A V z - b||^2 / ||b||^2.
    With W = A V it is Eq. 5's expression with (W, b) in place of (V, f), so
    dl/d(conj V) = A^H dl/d(conj W).  Returns (loss, dl/dRe V, dl/dIm V)."""
    W = np.column_stack([A @ V[:, c] for c in range(V.shape[1])])
    loss, gr, gi = projection_loss_and_grad(W, b)
    gw = 0.5 * (gr + 1j * gi)                       # dl / d conj(W)
    AH = A.conj().T
    gv = np.column_stack([AH @ gw[:, c] for c in range(V.shape[1])])
    return loss, 2.0 * gv.real, 2.0 * gv.imag


def batch_residual_loss_and_grad(cfg: CNNConfig, theta, x, ops, rhs, store=None, gstore=None):
    """Mean Eq. 6 loss over the batch (ops: sparse A per sample, rhs: b per
    sample) and its gradient w.r.t. theta."""
    y, cache = forward(cfg, theta, x, keep=True, store=store)
    V = to_complex_fields(y)
    B = x.shape[0]
    gy = np.zeros_like(y)
    tot = 0.0
    for s in range(B):
        l, gr, gi = residual_loss_and_grad(ops[s], V[s], rhs[s])
        tot += l
        g = np.zeros((V.shape[1], 2 * cfg.k))
        g[:, 0::2] = gr
        g[:, 1::2] = gi
        gy[s] = g.reshape(y.shape[1:]) / B
    gtheta, _ = backward(cfg, theta, cache, gy, gstore=gstore)
    return tot / B, gtheta
