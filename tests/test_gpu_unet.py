"""GPU parity of the warm-start network's kernels against the FP64 oracle.

Inputs and weights are drawn as BF16-representable values, so both sides see
the same numbers.  Tolerances:
* convolution outputs are FP32 sums of K = 9 * Cin products rounded to BF16:
  |gpu - ref| <= 2^-8 |ref| + 2 K 2^-24 S, with S the same sum over absolute
  values (the worst-case bound of a length-K FP32 sum, doubled);
* weight gradients are FP32 sums over P pixels (no final rounding):
  |gpu - ref| <= 2 (P + splits) 2^-24 S;
* the whole network stores every activation and activation gradient in
  BF16, so its loss and gradients are compared as relative L2 errors per
  layer.  The gradient test uses a uniform +z target: with random targets
  every weight gradient is a sum of terms of random sign that nearly cancel,
  and BF16 storage alone then moves it by 3-14%; with the +z target the
  same storage rounding, emulated in float64, moves no layer's gradient by
  more than 0.8%, and the test allows 3%.
"""
import numpy as np
import pytest
import torch

from oracle import unet as U
from paper_1901_11350_gb300 import inputs as I

pytestmark = pytest.mark.gpu

UN = pytest.importorskip("paper_1901_11350_gb300.unet")


def bf(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).cuda()


def f64(t):
    return t.float().cpu().numpy().astype(np.float64)


def rand_bf(rng, shape, scale=1.0):
    t = bf(rng.standard_normal(shape) * scale)
    return t, f64(t)


@pytest.fixture(params=["mma", "tcgen05", "tcgen05_ws", "tcgen05_halo"])
def kernel(request):
    old = UN.conv_kernel()
    UN.set_conv_kernel(request.param)
    yield request.param
    UN.check_device_error()
    UN.set_conv_kernel(old)


def virtual_input(x0, x1, up0):
    x = U.upsample(x0) if up0 else x0
    return x if x1 is None else np.concatenate([x, x1], axis=-1)


CONV_CASES = [
    # B, H, W, C0, up0, C1, Cout
    (2, 16, 16, 32, 0, 0, 32),
    (2, 16, 16, 64, 1, 32, 32),
    (1, 16, 16, 128, 0, 0, 256),
    (8, 8, 8, 256, 1, 128, 128),
    (2, 16, 16, 32, 0, 0, 96),
    (2, 8, 24, 64, 0, 0, 192),
    # rows of 64 and 128 pixels: the halo tiles of kernel 3
    (1, 8, 64, 32, 0, 0, 32),
    (1, 8, 64, 64, 1, 32, 64),
    (1, 4, 128, 64, 1, 32, 32),
]


@pytest.mark.parametrize("case", CONV_CASES)
@pytest.mark.parametrize("relu", [False, True])
def test_conv_forward(case, relu, kernel):
    B, H, W, C0, up0, C1, Cout = case
    rng = np.random.default_rng(hash(case) % 2**32)
    h0, w0 = (H // 2, W // 2) if up0 else (H, W)
    s0, x0 = rand_bf(rng, (B, h0, w0, C0))
    s1, x1 = rand_bf(rng, (B, H, W, C1)) if C1 else (None, None)
    Wt, Wn = rand_bf(rng, (Cout, 9, C0 + C1), 1.0 / np.sqrt(9 * (C0 + C1)))
    bias = rng.standard_normal(Cout).astype(np.float32)
    out = UN.conv3x3_forward(s0, Wt, torch.from_numpy(bias).cuda(), relu=relu, src1=s1, up0=bool(up0))
    x = virtual_input(x0, x1, up0)
    ref = U.conv3x3(x, Wn, bias.astype(np.float64))
    S = U.conv3x3(np.abs(x), np.abs(Wn), np.abs(bias.astype(np.float64)))
    if relu:
        ref = np.maximum(ref, 0)
    K = 9 * (C0 + C1)
    tol = 2.0 ** -8 * np.abs(ref) + 2 * K * 2.0 ** -24 * S
    err = np.abs(f64(out) - ref)
    assert np.all(err <= tol), float(np.max(err - tol))


@pytest.mark.parametrize("case", [(2, 16, 16, 96, 32), (2, 8, 8, 256, 256), (4, 16, 16, 32, 64), (1, 8, 64, 32, 64)])
def test_conv_data_gradient(case, kernel):
    # the data gradient is the forward kernel with transposed weights and the
    # input's ReLU mask
    B, H, W, Cin, Cout = case
    rng = np.random.default_rng(Cin * 1000 + Cout)
    Wt, Wn = rand_bf(rng, (Cout, 9, Cin), 1.0 / np.sqrt(9 * Cin))
    dzt, dz = rand_bf(rng, (B, H, W, Cout))
    at, a = rand_bf(rng, (B, H, W, Cin))
    WT = UN.conv3x3_transpose(Wt)
    assert torch.equal(WT.cpu(), torch.flip(Wt.cpu().permute(2, 1, 0), dims=[1]))
    out = UN.conv3x3_forward(dzt, WT, None, relu=False, mask=at)
    dx, _, _ = U.conv3x3_backward(np.zeros((B, H, W, Cin)), Wn, dz)
    ref = dx * (a > 0)
    # S: the same sums over absolute values
    Sx, _, _ = U.conv3x3_backward(np.zeros((B, H, W, Cin)), np.abs(Wn), np.abs(dz))
    K = 9 * Cout
    tol = 2.0 ** -8 * np.abs(ref) + 2 * K * 2.0 ** -24 * Sx
    err = np.abs(f64(out) - ref)
    assert np.all(err <= tol), float(np.max(err - tol))


@pytest.mark.parametrize("case", [
    (2, 16, 16, 32, 0, 0, 32),
    (2, 16, 16, 64, 1, 32, 32),
    (8, 8, 8, 256, 1, 128, 128),
    (1, 16, 16, 128, 0, 0, 256),
    (16, 32, 32, 32, 0, 0, 64),
    (1, 16, 16, 32, 0, 0, 288),  # the bias sum takes channels in slices of 256
])
def test_conv_weight_gradient(case, kernel):
    B, H, W, C0, up0, C1, Cout = case
    rng = np.random.default_rng(7 + C0 + Cout + B)
    h0, w0 = (H // 2, W // 2) if up0 else (H, W)
    s0, x0 = rand_bf(rng, (B, h0, w0, C0))
    s1, x1 = rand_bf(rng, (B, H, W, C1)) if C1 else (None, None)
    dzt, dz = rand_bf(rng, (B, H, W, Cout))
    dW, db = UN.conv3x3_wgrad(s0, dzt, src1=s1, up0=bool(up0))
    x = virtual_input(x0, x1, up0)
    _, rW, rb = U.conv3x3_backward(x, np.zeros((Cout, 9, x.shape[-1])), dz)
    _, SW, Sb = U.conv3x3_backward(np.abs(x), np.zeros((Cout, 9, x.shape[-1])), np.abs(dz))
    P = B * H * W
    gW, gb = dW.cpu().numpy().astype(np.float64), db.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(gW - rW) <= 2 * (P + 1024) * 2.0 ** -24 * SW)
    assert np.all(np.abs(gb - rb) <= 2 * (P + 1024) * 2.0 ** -24 * Sb)
    # deterministic: a second call gives the same bits
    dW2, db2 = UN.conv3x3_wgrad(s0, dzt, src1=s1, up0=bool(up0))
    assert torch.equal(dW, dW2) and torch.equal(db, db2)


def _net_case(L=32, B=8, seed=3, target="random"):
    rng = np.random.default_rng(seed)
    flat = I.unet_init(seed)
    # small random biases so no layer starts exactly at the ReLU kink
    for l in range(14):
        co, _, _, bo = UN.layer(l)
        flat[bo:bo + co] = rng.uniform(0.0, 0.05, co)
    spins = np.stack([I.random_spins(L * L, seed * 100 + b) for b in range(B)])
    if target == "random":
        target = np.stack([I.random_spins(L * L, seed * 100 + 50 + b) for b in range(B)])
    else:
        target = np.zeros((B, L * L, 3))
        target[..., 2] = 1.0
    feats = rng.uniform(0, 1, (B, 4)).astype(np.float32)
    rec = lambda a: torch.from_numpy(np.concatenate([a, np.zeros(a.shape[:2] + (1,))], -1).astype(np.float32)).cuda()  # noqa: E731
    return flat, rec(spins), torch.from_numpy(feats).cuda(), rec(target)


def _oracle_view(flat, spins, feats, target, L):
    """The oracle's inputs as the GPU sees them: BF16 convolution weights and
    network input, FP32 biases and head."""
    p = flat.astype(np.float64).copy()
    for l in range(14):
        co, ci, wo, bo = UN.layer(l)
        p[wo:bo] = f64(bf(flat[wo:bo]))
    params = U.unpack(p)
    B = spins.shape[0]
    x = U.network_input(f64(bf(spins.cpu().numpy()[..., :3])), f64(bf(feats.cpu().numpy())), L)
    t = target.cpu().numpy()[..., :3].astype(np.float64).reshape(B, L, L, 3)
    return params, x, t


def test_network_loss_and_gradient_match_oracle(kernel):
    L, B = 32, 8
    flat, spins, feats, target = _net_case(L, B, target="+z")
    net = UN.UNet(L, B, flat)
    grad = torch.empty(net.n_params, dtype=torch.float32, device="cuda")
    loss = net.loss_grad(spins, feats, target, grad).item()
    params, x, t = _oracle_view(flat, spins, feats, target, L)
    rloss, rgrads = U.loss_and_gradient(params, x, t)
    assert abs(loss - rloss) <= 2e-3 * abs(rloss)
    g = grad.cpu().numpy().astype(np.float64)
    names = [a[0] for a in U.architecture()] + ["head"]
    for l, name in enumerate(names):
        co, ci, wo, bo = UN.layer(l)
        for k, (lo, hi) in enumerate(((wo, bo), (bo, bo + co))):
            ref = rgrads[name][k].ravel()
            got = g[lo:hi]
            rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert rel < 3e-2, (name, k, rel)


def test_network_predict_and_adam(kernel):
    L, B = 32, 8
    flat, spins, feats, target = _net_case(L, B, seed=5)
    net = UN.UNet(L, B, flat)
    pred = net.predict(spins, feats)
    p = pred.cpu().numpy()
    assert np.allclose(np.linalg.norm(p[..., :3], axis=-1), 1.0, atol=1e-6) and np.all(p[..., 3] == 0)
    params, x, t = _oracle_view(flat, spins, feats, target, L)
    ref = U.predict(params, x).reshape(B, L * L, 3)
    cos = np.sum(p[..., :3] * ref, axis=-1)
    assert np.mean(cos) > 0.9999 and np.min(cos) > 0.99
    # Adam on the GPU's own gradient against the oracle's update (FP32 arithmetic)
    grad = torch.empty(net.n_params, dtype=torch.float32, device="cuda")
    net.loss_grad(spins, feats, target, grad)
    net.adam(1e-3)
    got = net.get_params().astype(np.float64)
    g = grad.cpu().numpy().astype(np.float64)
    exp, _, _ = U.adam_step(flat.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, 1e-3)
    assert np.max(np.abs(got - exp)) <= 1e-6 * 1e-3 + 2e-7 * np.max(np.abs(flat))


def test_network_training_lowers_the_loss():
    # learn the identity map on one batch: 40 Adam steps must cut the loss
    L, B = 32, 8
    flat, spins, feats, _ = _net_case(L, B, seed=9)
    net = UN.UNet(L, B, flat)
    first = net.loss_grad(spins, feats, spins).item()
    net.adam(1e-3)
    for _ in range(39):
        net.train_step(spins, feats, spins, 1e-3)
    last = net.loss_grad(spins, feats, spins).item()
    assert last < 0.5 * first, (first, last)


def test_network_rejects_bad_batches():
    net = UN.UNet(32, 8)
    s = torch.zeros((3, 1024, 4), dtype=torch.float32, device="cuda")
    f = torch.zeros((3, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(Exception):
        net.predict(s, f)  # 3 * 16 bottom pixels is not a multiple of 128
    s = torch.zeros((16, 1024, 4), dtype=torch.float32, device="cuda")
    f = torch.zeros((16, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(Exception):
        net.predict(s, f)  # more than batch_max


def test_conv_pipeline_wait_that_runs_out_reports_and_leaves_the_device_usable():
    """With a wait limit of zero every CTA of the tcgen05 convolution gives up
    its first pipeline wait: it drains the MMAs it issued, frees its tensor
    memory and writes nothing, and the device flag reports SP_ERR_TIMEOUT.
    With the default limit restored the same call is correct again."""
    old = UN.conv_kernel()
    UN.set_conv_kernel("tcgen05")
    UN.check_device_error()
    B, H, W, C0, Cout = 2, 16, 16, 64, 64  # 18 K steps: the pipeline wait is reached
    rng = np.random.default_rng(11)
    s0, x0 = rand_bf(rng, (B, H, W, C0))
    Wt, Wn = rand_bf(rng, (Cout, 9, C0), 1.0 / np.sqrt(9 * C0))
    lib = UN.lib
    try:
        UN.set_wait_limit(0)
        out = torch.full((B, H, W, Cout), 7.0, dtype=torch.bfloat16, device="cuda")
        rc = lib().sp_conv3x3_forward(s0.data_ptr(), C0, 0, None, 0, Wt.data_ptr(), None, 0, None, B, H, W, Cout,
                                      out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert rc == 0
        assert lib().sp_unet_device_error() == -5  # SP_ERR_TIMEOUT
        assert bool(torch.all(out == 7.0)), "a CTA whose wait ran out wrote outputs"
    finally:
        UN.set_wait_limit()
    out = UN.conv3x3_forward(s0, Wt)
    assert lib().sp_unet_device_error() == 0
    ref = U.conv3x3(x0, Wn, np.zeros(Cout))
    S = U.conv3x3(np.abs(x0), np.abs(Wn), np.zeros(Cout))
    tol = 2.0 ** -8 * np.abs(ref) + 2 * 9 * C0 * 2.0 ** -24 * S
    assert np.all(np.abs(f64(out) - ref) <= tol)
    # the weight gradient's pipeline: 16 x 32 x 32 pixels give every split
    # more stages than the pipeline holds, so its wait is reached
    s0, x0 = rand_bf(rng, (16, 32, 32, C0))
    dzt, dz = rand_bf(rng, (16, 32, 32, Cout))
    try:
        UN.set_wait_limit(0)
        UN.conv3x3_wgrad(s0, dzt)
        assert lib().sp_unet_device_error() == -5
    finally:
        UN.set_wait_limit()
    dW, _ = UN.conv3x3_wgrad(s0, dzt)
    assert lib().sp_unet_device_error() == 0
    _, rW, _ = U.conv3x3_backward(x0, np.zeros((Cout, 9, C0)), dz)
    _, SW, _ = U.conv3x3_backward(np.abs(x0), np.zeros((Cout, 9, C0)), np.abs(dz))
    assert np.all(np.abs(dW.cpu().numpy() - rW) <= 2 * (16 * 32 * 32 + 1024) * 2.0 ** -24 * SW)
    UN.set_conv_kernel(old)



def test_halo_conv_wait_that_runs_out_reports_and_leaves_the_device_usable():
    """The halo-tile kernel waits for a chunk's MMAs before it refills the
    chunk's buffers: with a wait limit of zero every CTA of a two-chunk
    convolution gives up there, drains the MMAs it issued, frees its tensor
    memory and writes nothing, and the device flag reports SP_ERR_TIMEOUT;
    with the default limit restored the same call is correct."""
    old = UN.conv_kernel()
    UN.set_conv_kernel("tcgen05_halo")
    UN.check_device_error()
    B, H, W, C0, Cout = 2, 8, 64, 64, 64  # rows of 64 pixels, two chunks of 32 input channels
    rng = np.random.default_rng(13)
    s0, x0 = rand_bf(rng, (B, H, W, C0))
    Wt, Wn = rand_bf(rng, (Cout, 9, C0), 1.0 / np.sqrt(9 * C0))
    lib = UN.lib
    try:
        UN.set_wait_limit(0)
        out = torch.full((B, H, W, Cout), 7.0, dtype=torch.bfloat16, device="cuda")
        rc = lib().sp_conv3x3_forward(s0.data_ptr(), C0, 0, None, 0, Wt.data_ptr(), None, 0, None, B, H, W, Cout,
                                      out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert rc == 0
        assert lib().sp_unet_device_error() == -5  # SP_ERR_TIMEOUT
        assert bool(torch.all(out == 7.0)), "a CTA whose wait ran out wrote outputs"
    finally:
        UN.set_wait_limit()
    out = UN.conv3x3_forward(s0, Wt)
    assert lib().sp_unet_device_error() == 0
    UN.set_conv_kernel(old)
    ref = U.conv3x3(x0, Wn, np.zeros(Cout))
    S = U.conv3x3(np.abs(x0), np.abs(Wn), np.zeros(Cout))
    tol = 2.0 ** -8 * np.abs(ref) + 2 * 9 * C0 * 2.0 ** -24 * S
    assert np.all(np.abs(f64(out) - ref) <= tol)