"""FP64 reference of the warm-start network (numpy, plain and slow).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg are the only callers.  The paper has no network; this module
restates, from its written description, the BF16 U-Net that predicts a
relaxed spin configuration from a random one (the warm start of the
velocity-projection minimiser of Appendix D), with every step in float64 and
every gradient derived by hand, so the CUDA kernels' forward pass, data and
weight gradients and Adam step can be compared with it.  It shares no code
with the CUDA library.

Definitions (NHWC arrays, periodic lattice):
* conv3x3: out[b,y,x,o] = bias[o] + sum_{t,i} W[o,t,i] in[b,(y+dy)%H,(x+dx)%W,i]
  with tap t = 3(dy+1) + (dx+1);
* ReLU after every 3x3 convolution; 2x2 mean pooling; nearest upsampling by
  2; channel concatenation [upsampled | skip];
* widths w = (32, 64, 128, 256): e1a, e1b at L; e2a, e2b at L/2; e3a, e3b at
  L/4; b4a, b4b at L/8; d3a, d3b; d2a, d2b; d1a, d1b back up; head
  y = Wh a + bh (32 -> 3), prediction m = y/|y|;
* input channels: n (3), the 4 per-system features, zeros up to 32;
* loss = mean over pixels of 1 - m . m_target;
* flat parameters: per convolution W [Cout][9][Cin] then bias, then Wh
  [3][32], bh [3];
* Adam (Kingma & Ba, 2015) with bias-corrected moments.

Pins (tests/test_oracle_pins.py): the convolution against a brute-force
loop, every backward function against central finite differences of the
forward, the whole network's gradient against finite differences of its loss,
and Adam's first step against its closed form.
"""
import numpy as np

IN_CH = 32
N_FEATURES = 4


def architecture(widths=(32, 64, 128, 256), in_ch=IN_CH):
    """(name, cin, cout, level) of the 14 convolutions, in parameter order."""
    w1, w2, w3, w4 = widths
    return [("e1a", in_ch, w1, 0), ("e1b", w1, w1, 0), ("e2a", w1, w2, 1), ("e2b", w2, w2, 1),
            ("e3a", w2, w3, 2), ("e3b", w3, w3, 2), ("b4a", w3, w4, 3), ("b4b", w4, w4, 3),
            ("d3a", w4 + w3, w3, 2), ("d3b", w3, w3, 2), ("d2a", w3 + w2, w2, 1), ("d2b", w2, w2, 1),
            ("d1a", w2 + w1, w1, 0), ("d1b", w1, w1, 0)]


def unpack(flat, widths=(32, 64, 128, 256), in_ch=IN_CH):
    """Split the flat parameter vector into {name: (W, b)} and the head."""
    flat = np.asarray(flat, dtype=np.float64)
    out, k = {}, 0
    for name, cin, cout, _ in architecture(widths, in_ch):
        nw = cout * 9 * cin
        out[name] = (flat[k:k + nw].reshape(cout, 9, cin), flat[k + nw:k + nw + cout])
        k += nw + cout
    w1 = widths[0]
    out["head"] = (flat[k:k + 3 * w1].reshape(3, w1), flat[k + 3 * w1:k + 3 * w1 + 3])
    k += 3 * w1 + 3
    if k != flat.size:
        raise ValueError("parameter vector has %d entries, architecture needs %d" % (flat.size, k))
    return out


def pack(params, widths=(32, 64, 128, 256), in_ch=IN_CH):
    parts = []
    for name, _, _, _ in architecture(widths, in_ch):
        W, b = params[name]
        parts += [np.asarray(W).ravel(), np.asarray(b).ravel()]
    parts += [np.asarray(params["head"][0]).ravel(), np.asarray(params["head"][1]).ravel()]
    return np.concatenate(parts)


# ------------------------------------------------------------------ layers
TAPS = [(t // 3 - 1, t % 3 - 1) for t in range(9)]


def shifted(x, dy, dx):
    """s[b, y, x] = x[b, (y+dy)%H, (x+dx)%W]."""
    return np.roll(x, shift=(-dy, -dx), axis=(1, 2))


def conv3x3(x, W, b):
    out = np.zeros(x.shape[:3] + (W.shape[0],)) + b
    for t, (dy, dx) in enumerate(TAPS):
        out += shifted(x, dy, dx) @ W[:, t, :].T
    return out


def conv3x3_backward(x, W, dz):
    """(dx, dW, db) of conv3x3 for the output gradient dz."""
    dxs = np.zeros_like(x)
    dW = np.zeros_like(W)
    for t, (dy, dx) in enumerate(TAPS):
        s = shifted(x, dy, dx)
        dW[:, t, :] = np.einsum("bhwo,bhwi->oi", dz, s)
        # out[p] reads x[p + off]: the gradient flows back to x[q] from dz[q - off]
        dxs += shifted(dz @ W[:, t, :], -dy, -dx)
    return dxs, dW, dz.sum(axis=(0, 1, 2))


def relu(z):
    return np.maximum(z, 0.0)


def pool(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool_backward(dp):
    return np.repeat(np.repeat(dp, 2, axis=1), 2, axis=2) / 4.0


def upsample(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample_backward(du):
    B, H, W, C = du.shape
    return du.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def network_input(spins, features, L, in_ch=IN_CH):
    """spins [B, L*L, >=3], features [B, 4] -> [B, L, L, in_ch]."""
    spins = np.asarray(spins, dtype=np.float64)
    features = np.asarray(features, dtype=np.float64)
    B = spins.shape[0]
    x = np.zeros((B, L, L, in_ch))
    x[..., :3] = spins[:, :, :3].reshape(B, L, L, 3)
    x[..., 3:3 + N_FEATURES] = features[:, None, None, :]
    return x


# ------------------------------------------------------------------ network
ENCODER = ["e1a", "e1b", "e2a", "e2b", "e3a", "e3b", "b4a", "b4b"]


def forward(params, x):
    """Activations of every layer (post-ReLU), the pools and the head output."""
    a = {}
    h = x
    pools = []
    for i, name in enumerate(ENCODER):
        W, b = params[name]
        h = relu(conv3x3(h, W, b))
        a[name] = h
        if i in (1, 3, 5):
            h = pool(h)
            pools.append(h)
    for name_a, name_b, skip in (("d3a", "d3b", "e3b"), ("d2a", "d2b", "e2b"), ("d1a", "d1b", "e1b")):
        cat = np.concatenate([upsample(h), a[skip]], axis=-1)
        W, b = params[name_a]
        h = relu(conv3x3(cat, W, b))
        a[name_a] = h
        W, b = params[name_b]
        h = relu(conv3x3(h, W, b))
        a[name_b] = h
    Wh, bh = params["head"]
    y = h @ Wh.T + bh
    return a, pools, y


def loss_of(y, target):
    """Mean of 1 - m . m_target with m = y/|y|; target [B, L, L, 3]."""
    m = y / np.linalg.norm(y, axis=-1, keepdims=True)
    return float(np.mean(1.0 - np.sum(m * target, axis=-1)))


def predict(params, x):
    _, _, y = forward(params, x)
    return y / np.linalg.norm(y, axis=-1, keepdims=True)


def loss_and_gradient(params, x, target):
    """Loss and {name: (dW, db)} for one batch, by reverse-mode differentiation
    written out layer by layer."""
    a, pools, y = forward(params, x)
    P = y.shape[0] * y.shape[1] * y.shape[2]
    ny = np.linalg.norm(y, axis=-1, keepdims=True)
    m = y / ny
    c = np.sum(m * target, axis=-1, keepdims=True)
    loss = float(np.mean(1.0 - c))
    # d(1 - m.t)/dy = -(t - (m.t) m) / |y|
    dy = -(target - c * m) / ny / P
    grads = {}
    Wh, bh = params["head"]
    h = a["d1b"]
    grads["head"] = (np.einsum("bhwo,bhwi->oi", dy, h), dy.sum(axis=(0, 1, 2)))
    da = dy @ Wh
    skip_grad = {}

    def through(name, inp, da_out):
        dz = da_out * (a[name] > 0)
        W, _ = params[name]
        dx, dW, db = conv3x3_backward(inp, W, dz)
        grads[name] = (dW, db)
        return dx

    inputs_dec = {"d3a": ("b4b", "e3b"), "d2a": ("d3b", "e2b"), "d1a": ("d2b", "e1b")}
    for name_a, name_b in (("d1a", "d1b"), ("d2a", "d2b"), ("d3a", "d3b")):
        da = through(name_b, a[name_a], da)
        coarse, skip = inputs_dec[name_a]
        cat = np.concatenate([upsample(a[coarse]), a[skip]], axis=-1)
        dcat = through(name_a, cat, da)
        C0 = a[coarse].shape[-1]
        skip_grad[skip] = dcat[..., C0:]
        da = upsample_backward(dcat[..., :C0])
    # bottom and encoder, from b4b down; pools[k] = pool(a[e(k+1)b])
    order = [("b4b", "b4a"), ("b4a", 2), ("e3b", "e3a"), ("e3a", 1), ("e2b", "e2a"), ("e2a", 0), ("e1b", "e1a"),
             ("e1a", None)]
    for name, src in order:
        if isinstance(src, str):
            inp = a[src]
        elif src is None:
            inp = x
        else:
            inp = pools[src]
        dx = through(name, inp, da)
        if isinstance(src, int):  # dx is the pool's gradient; add the skip path
            skip = {2: "e3b", 1: "e2b", 0: "e1b"}[src]
            da = pool_backward(dx) + skip_grad[skip]
        else:
            da = dx
    return loss, grads


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step; returns the new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
