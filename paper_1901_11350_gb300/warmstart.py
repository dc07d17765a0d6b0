"""Learned warm start for energy minimisation.

The velocity-projection minimiser (Appendix D) relaxes a spin configuration
to a local energy minimum.  This module trains the BF16 U-Net of
``unet.py`` on relaxations the minimiser itself produces and measures what a
predicted starting point saves.  The minimiser always finishes the job: a
prediction is only a start, and every reported result is the minimiser's own
final state, judged by its energy and max torque.

Workload (``inputs.warmstart_draw``): L x L periodic hexagonal monolayers,
J = 1 meV, interfacial D ~ U[0.1, 0.5] meV, K ~ U[0, 0.2] meV (z),
B ~ U[0, 3] T (z), random initial spins.

* generate: batched FP32 relaxations of the random starts (labels).
* train: Adam on mean(1 - m . m_label) with random lattice translations.
* evaluate, on held-out systems, three arms that all end with FP64 max torque
  below `tol`:
    unaided   FP64 velocity projection from the random start, the plain
              method (batched here; each system's iterates are bit-identical
              to the one-system loop, which is timed on a sample);
    batched   the same start, FP32 relaxation to `fp32_tol`, then FP64;
    warm      network prediction, FP32 relaxation to `fp32_tol`, then FP64;
    uniform   the trivial guess -- the +z ferromagnet tilted by 0.05 rad
              random noise -- relaxed like the warm arm, to show what the
              network adds over it.
  Systems whose final energies agree with the unaided arm's to 1e-8 relative
  are "matched"; the others ended in a different local minimum and are
  counted as lower or higher.  Where the unaided arm hit its iteration cap,
  its last energy is the comparison.  Final states whose energy equals the
  +z ferromagnet's (1e-8) are counted as ferromagnetic.
"""
import argparse
import json
import math
import time

import numpy as np
import torch

from . import binding as B
from . import inputs as I
from . import unet as UN

VP_DT = 0.2          # velocity-projection time step (mass 1)
LABEL_TOL = 1e-4     # FP32 label relaxations stop at this max torque (meV)
FP32_TOL = 1e-4      # FP32 stage of the batched and warm arms
TOL = 1e-6           # final max torque (meV) of every evaluated relaxation
MATCH_RTOL = 1e-8    # same final energy


def _records(spins, dtype=torch.float32):
    """[n, N, 3] numpy -> [n, N, 4] CUDA records."""
    n, N, _ = spins.shape
    out = torch.zeros((n, N, 4), dtype=dtype, device="cuda")
    out[..., :3] = torch.from_numpy(np.ascontiguousarray(spins)).to(device="cuda", dtype=dtype)
    return out


def _features(draws):
    return torch.from_numpy(np.stack([I.warmstart_features(d) for d in draws])).cuda()


class _Timer:
    """Device time between two events on the current stream, in seconds."""

    def __enter__(self):
        self.a = torch.cuda.Event(enable_timing=True)
        self.b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        self.a.record()
        return self

    def __exit__(self, *exc):
        self.b.record()
        torch.cuda.synchronize()
        self.seconds = self.a.elapsed_time(self.b) / 1e3


def relax(ctxs, spins, tol, max_iter, check_every=256, dt=VP_DT):
    """Batched minimisation of spins [n, N, 4] in place; one context per
    system.  Returns (iterations, max torque, device seconds)."""
    n, N, _ = spins.shape
    flat = spins.view(n * N, 4)
    vel = torch.zeros_like(flat)
    with _Timer() as t:
        it, mt = B.minimise_batch(ctxs, flat, vel, [k * N for k in range(n)], dt=dt, mass=1.0, tol=tol,
                                  max_iter=max_iter, check_every=check_every)
    return it, mt, t.seconds


def energies(ctxs, spins):
    return np.array([c.energy(spins[k])[0].item() for k, c in enumerate(ctxs)])


def _contexts(draws, prec):
    return [B.Context(d["geometry"], d["hamiltonian"], prec) for d in draws]


def _close(ctxs):
    for c in ctxs:
        c.close()


def unet_flops(L):
    """Forward multiply-add FLOPs of the network per L x L sample: 2 x pixels
    x 9 x Cin x Cout per 3x3 convolution (the head and pointwise steps are
    not counted)."""
    levels = [0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0]
    return float(sum(2 * (L >> lv) ** 2 * 9 * ci * co for (ci, co), lv in zip(I.UNET_LAYERS, levels)))


def save_params(path, flat):
    """Trained parameters: convolution weights as BF16 bit patterns (the
    precision the kernels use), biases and the head in FP32."""
    flat = np.asarray(flat, dtype=np.float32)
    mask = np.zeros(flat.size, dtype=bool)
    k = 0
    for ci, co in I.UNET_LAYERS:
        mask[k:k + co * 9 * ci] = True
        k += co * 9 * ci + co
    w = torch.from_numpy(flat[mask]).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.savez_compressed(path, conv_bf16=w, other_f32=flat[~mask], n=np.int64(flat.size))


def load_params(path):
    d = np.load(path)
    n = int(d["n"])
    mask = np.zeros(n, dtype=bool)
    k = 0
    for ci, co in I.UNET_LAYERS:
        mask[k:k + co * 9 * ci] = True
        k += co * 9 * ci + co
    flat = np.empty(n, dtype=np.float32)
    flat[mask] = torch.from_numpy(d["conv_bf16"].view(np.int16)).view(torch.bfloat16).float().numpy()
    flat[~mask] = d["other_f32"]
    return flat


# ------------------------------------------------------------------ data
def generate(seed, n, L=128, chunk=1024, max_iter=20000, tol=LABEL_TOL, log=print):
    """Labelled relaxations: dict of CUDA tensors init/label [n, L*L, 4],
    feat [n, 4] and numpy iters/torque [n]."""
    init = torch.empty((n, L * L, 4), dtype=torch.float32, device="cuda")
    label = torch.empty_like(init)
    feat = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    iters, torque = np.zeros(n, dtype=np.int64), np.zeros(n)
    seconds = 0.0
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        draws = [I.warmstart_draw(seed, i, L) for i in range(c0, c1)]
        x = _records(np.stack([d["spins"] for d in draws]))
        init[c0:c1] = x
        feat[c0:c1] = _features(draws)
        ctxs = _contexts(draws, "f32")
        it, mt, sec = relax(ctxs, x, tol, max_iter)
        _close(ctxs)
        label[c0:c1] = x
        iters[c0:c1], torque[c0:c1] = it, mt
        seconds += sec
        log("generate %d-%d: %.1f s, median iterations %d, converged %d/%d"
            % (c0, c1, sec, int(np.median(it)), int((mt < tol).sum()), c1 - c0))
    return dict(init=init, label=label, feat=feat, iters=iters, torque=torque, seconds=seconds, L=L)


# ------------------------------------------------------------------ training
def train(data, epochs, batch=64, lr=1e-3, lr_min=3e-5, seed=0, log=print, net=None):
    """Adam with a cosine learning-rate schedule; every sample is shifted by
    a random lattice translation (the Hamiltonian is translation invariant on
    the periodic lattice).  Returns (net, history)."""
    L = data["L"]
    n = data["init"].shape[0]
    if net is None:
        net = UN.UNet(L, batch, I.unet_init(seed))
    rng = np.random.default_rng(seed + 1)
    steps = epochs * (n // batch)
    history = []
    k = 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).cuda()
        acc = torch.zeros(1, dtype=torch.float64, device="cuda")
        nb = n // batch
        for j in range(nb):
            idx = perm[j * batch:(j + 1) * batch]
            sy, sx = (int(v) for v in rng.integers(0, L, 2))
            s = torch.roll(data["init"][idx].view(batch, L, L, 4), (sy, sx), (1, 2)).reshape(batch, L * L, 4)
            t = torch.roll(data["label"][idx].view(batch, L, L, 4), (sy, sx), (1, 2)).reshape(batch, L * L, 4)
            rate = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * k / max(1, steps)))
            acc += net.train_step(s.contiguous(), data["feat"][idx].contiguous(), t.contiguous(), rate)
            k += 1
        mean = acc.item() / nb
        history.append(mean)
        log("epoch %d: loss %.5f (%.1f s)" % (ep + 1, mean, time.perf_counter() - t0))
    return net, history


def predict(net, spins, feat):
    """Network prediction for spins [n, N, 4] in batches of net.batch_max."""
    out = torch.empty_like(spins)
    bm = net.batch_max
    for c0 in range(0, spins.shape[0], bm):
        c1 = min(spins.shape[0], c0 + bm)
        out[c0:c1] = net.predict(spins[c0:c1].contiguous(), feat[c0:c1].contiguous())
    return out


def mean_loss(net, data, batch=None):
    """Mean loss of the network on a data set (no update)."""
    bm = batch or net.batch_max
    n = data["init"].shape[0] // bm * bm
    tot = 0.0
    for c0 in range(0, n, bm):
        tot += net.loss_grad(data["init"][c0:c0 + bm].contiguous(), data["feat"][c0:c0 + bm].contiguous(),
                             data["label"][c0:c0 + bm].contiguous()).item()
    return tot / max(1, n // bm)


# ------------------------------------------------------------------ evaluation
def evaluate(net, seed, n, L=128, max_iter=30000, polish_max_iter=5000, fp32_tol=FP32_TOL, tol=TOL, chunk=500,
             per_system=8, log=print):
    """Three-arm comparison on held-out systems (see the module docstring).
    The unaided arm and the FP32 stages get max_iter iterations, the FP64
    stage after FP32 polish_max_iter more."""
    draws = [I.warmstart_draw(seed, i, L) for i in range(n)]
    init_np = np.stack([d["spins"] for d in draws])
    feat = _features(draws)
    arms = ("unaided", "batched", "warm", "uniform")
    res = {k: dict(iters=np.zeros(n, np.int64), iters32=np.zeros(n, np.int64), torque=np.zeros(n),
                   energy=np.zeros(n), seconds=0.0) for k in arms}
    res["warm"]["net_seconds"] = 0.0
    e_fm = np.zeros(n)
    uniform_np = np.stack([I.perturbed(I.ferromagnet(L * L), 0.05, 1000 + i) for i in range(n)])
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        sl = slice(c0, c1)
        d = draws[c0:c1]
        c64, c32 = _contexts(d, "f64"), _contexts(d, "f32")
        x = _records(init_np[sl], torch.float64)
        it, mt, sec = relax(c64, x, tol, max_iter)
        r = res["unaided"]
        r["iters"][sl], r["torque"][sl], r["energy"][sl] = it, mt, energies(c64, x)
        r["seconds"] += sec
        fm = _records(np.stack([I.ferromagnet(L * L)] * (c1 - c0)), torch.float64)
        e_fm[sl] = energies(c64, fm)
        for arm in ("batched", "warm", "uniform"):
            r = res[arm]
            x32 = _records(uniform_np[sl] if arm == "uniform" else init_np[sl])
            if arm == "warm":
                with _Timer() as t:
                    x32 = predict(net, x32, feat[sl])
                r["net_seconds"] += t.seconds
                r["seconds"] += t.seconds
            it32, _, s32 = relax(c32, x32, fp32_tol, max_iter)
            x64 = x32.double()
            it64, mt64, s64 = relax(c64, x64, tol, polish_max_iter)
            r["iters32"][sl] = it32
            r["iters"][sl] = it32 + it64
            r["torque"][sl], r["energy"][sl] = mt64, energies(c64, x64)
            r["seconds"] += s32 + s64
        _close(c64)
        _close(c32)
        log("evaluate %d-%d: unaided %.1f s, batched %.1f s, warm %.1f s" %
            (c0, c1, res["unaided"]["seconds"], res["batched"]["seconds"], res["warm"]["seconds"]))
    # the unaided method as a one-system loop, timed on a sample
    sample = []
    for i in range(min(per_system, n)):
        c = B.Context(draws[i]["geometry"], draws[i]["hamiltonian"], "f64")
        x = c.spins(init_np[i])
        v = c.spins(np.zeros_like(init_np[i]))
        with _Timer() as t:
            it, mt = c.minimise(x, v, dt=VP_DT, tol=tol, max_iter=max_iter, check_every=256)
        assert it == res["unaided"]["iters"][i], "one-system loop differs from the batched iterate"
        sample.append((int(it), t.seconds))
        c.close()
    out = summarise(res, draws, sample, max_iter, tol, e_fm)
    out["polish_max_iter"] = polish_max_iter
    return out


def summarise(res, draws, sample, max_iter, tol, e_fm):
    U, out = res["unaided"], {}
    conv_u = U["torque"] < tol
    is_fm = lambda e: np.abs(e - e_fm) <= MATCH_RTOL * np.abs(e_fm)  # noqa: E731
    per_iter = sum(s for _, s in sample) / max(1, sum(i for i, _ in sample))
    out["unaided_per_system_loop"] = dict(sample_systems=len(sample), sample_iterations=[i for i, _ in sample],
                                          sample_seconds=[s for _, s in sample], seconds_per_iteration=per_iter,
                                          est_seconds_all=float(per_iter * U["iters"].sum()))
    for arm in res:
        r = res[arm]
        conv = r["torque"] < tol
        both = conv & conv_u
        rel = np.abs(r["energy"] - U["energy"]) / np.abs(U["energy"])
        match = both & (rel <= MATCH_RTOL)
        o = dict(converged=int(conv.sum()), n=len(conv), batched_seconds=r["seconds"],
                 median_iterations=float(np.median(r["iters"])), mean_iterations=float(np.mean(r["iters"])),
                 ferromagnetic_final=int(is_fm(r["energy"]).sum()))
        if arm != "unaided":
            cap = conv & ~conv_u
            o.update(matched=int(match.sum()), lower=int((both & ~match & (r["energy"] < U["energy"])).sum()),
                     higher=int((both & ~match & (r["energy"] > U["energy"])).sum()),
                     matched_iterations=int(r["iters"][match].sum()),
                     unaided_matched_iterations=int(U["iters"][match].sum()),
                     fp32_iterations_median=float(np.median(r["iters32"])),
                     unaided_capped=dict(n=int(cap.sum()), lower=int((cap & (r["energy"] < U["energy"])).sum()),
                                         higher=int((cap & (r["energy"] > U["energy"])).sum())))
            if arm == "warm":
                o["network_seconds"] = r["net_seconds"]
        out[arm] = o
    out["max_iter"] = max_iter
    out["tol"] = tol
    return out


# ------------------------------------------------------------------ command line
def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--train-n", type=int, default=20000)
    ap.add_argument("--eval-n", type=int, default=1000)
    ap.add_argument("--L", type=int, default=128)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--label-max-iter", type=int, default=20000)
    ap.add_argument("--eval-max-iter", type=int, default=30000)
    ap.add_argument("--polish-max-iter", type=int, default=5000)
    ap.add_argument("--chunk", type=int, default=1024)
    ap.add_argument("--out", default=None, help="write parameters (.npz) and the report (.json) with this prefix")
    ap.add_argument("--params", default=None, help="evaluate these trained parameters (.npz), no training")
    a = ap.parse_args(argv)
    log = lambda s: print(s, flush=True)  # noqa: E731
    t0 = time.perf_counter()
    if a.params:
        net = UN.UNet(a.L, a.batch, load_params(a.params))
        report = dict(params=a.params)
    else:
        data = generate(I.WARMSTART_SEEDS["train"], a.train_n, a.L, a.chunk, a.label_max_iter, log=log)
        net, hist = train(data, a.epochs, a.batch, a.lr, log=log)
        report = dict(train_n=a.train_n, epochs=a.epochs, batch=a.batch, loss_history=hist,
                      label_seconds=data["seconds"], label_converged=int((data["torque"] < LABEL_TOL).sum()))
        del data
        torch.cuda.empty_cache()
    report["evaluation"] = evaluate(net, I.WARMSTART_SEEDS["heldout"], a.eval_n, a.L, a.eval_max_iter, a.polish_max_iter,
                                    log=log)
    report["wall_seconds"] = time.perf_counter() - t0
    if a.out:
        save_params(a.out + ".npz", net.get_params())
        with open(a.out + ".json", "w") as f:
            json.dump(report, f, indent=1)
    log(json.dumps(report["evaluation"], indent=1))


if __name__ == "__main__":
    main()
