"""Learned warm start for the geodesic nudged elastic band (Sec. GNEB).

The network of ``unet.py`` (the same BF16 U-Net and kernels as the
minimiser's warm start) predicts the images of a converged skyrmion-collapse
path: from the relaxed skyrmion endpoint (3 channels) and four broadcast
features -- the reaction coordinate s = v / (M - 1) of the image and the
Hamiltonian's D / 0.5, K / 0.2, B / 3 (J = 1 meV throughout, so its channel
carries s) -- to image v of the minimum energy path.  Unlike a relaxation
from random spins, the converged path is a function of its endpoints, so
there is something to learn.  GNEB always finishes the job: a predicted
path is only a start, and every reported result is the chain GNEB itself
converges to max force < tol, judged by its barrier.

Workload (``inputs.gneb_draw`` with 128 x 128 periodic hexagonal lattices):
chains of M = 16 images from the ferromagnet (image 0) to a relaxed Neel
skyrmion (image M - 1), J = 1, D ~ U[0.25, 0.4], K ~ U[0.05, 0.1] meV,
B ~ U[0.5, 2] T, radius ~ U{3..8}; training seed 7, held-out seed 8.

* generate: converged FP32 chains (batched GNEB, climbing image) -> samples
  (endpoint, features, image v) for v = 1 .. M - 2.
* train: ``warmstart.train`` (Adam, random lattice translations).
* evaluate on held-out chains, three arms, each converged by the batched
  FP32 GNEB to max force < tol:
    geodesic  the method's own initial path (great-circle interpolation);
    ansatz    a trivial physical guess: Neel profiles whose radius shrinks
              linearly from the relaxed skyrmion's to zero;
    network   the predicted interior images (endpoints kept exactly).
  Reported: iterations, device seconds (the network's own time included) and
  the barrier of each converged chain (its highest image re-evaluated by an
  FP64 context) against the geodesic arm's.
All arithmetic runs in the library's kernels; this module orchestrates.
"""
import argparse
import json
import math
import time

import numpy as np
import torch

from . import binding as B
from . import gneb_batch as G
from . import inputs as I
from . import unet as UN
from . import warmstart as W

M_IMAGES = 16
L_SIDE = 128
GNEB_DT = 0.2
TOL = 1e-5
SEEDS = I.GNEB_WARMSTART_SEEDS


def features(draw, s):
    """(s, D/0.5, K/0.2, B/3): the reaction coordinate in the channel the
    minimiser's warm start gives J (1 meV in every GNEB draw)."""
    h = draw["hamiltonian"]
    return np.array([s, h["D"][0] / 0.5, h["K"][0] / 0.2, h["B"][2] / 3.0], dtype=np.float32)


def chains(seed, n, log=None):
    return G.prepare(n_chains=n, seed=seed, precision="f32", sizes=(L_SIDE,), images=(M_IMAGES, M_IMAGES), log=log)


def converge(chs, starts=None, tol=TOL, chunk=50, max_iter=100000):
    """Batched FP32 GNEB of the chains from their slerp paths, or from
    `starts` (list of [M, N, 4] CUDA tensors).  Returns (state, seconds)."""
    if starts is not None:
        for ch, s in zip(chs, starts):
            ch.chain0 = s[..., :3].double().cpu().numpy()
    return G.run_batched(chs, dt=GNEB_DT, k_spring=1.0, tol=tol, chunk=chunk, max_iter=max_iter)


def samples(chs, state):
    """Training samples of converged chains: init = the skyrmion endpoint,
    feat = features(s), label = interior image v."""
    L = L_SIDE
    n = sum(ch.M - 2 for ch in chs)
    init = torch.empty((n, L * L, 4), dtype=torch.float32, device="cuda")
    label = torch.empty_like(init)
    feat = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    k = 0
    for j, ch in enumerate(chs):
        x = state[j]["x"].view(ch.M, ch.N, 4).float()
        for v in range(1, ch.M - 1):
            init[k] = x[ch.M - 1]
            label[k] = x[v]
            feat[k] = torch.from_numpy(features(ch.draw, v / (ch.M - 1.0)))
            k += 1
    return dict(init=init, label=label, feat=feat, L=L)


def predicted_paths(net, chs):
    """Network paths: endpoints exact, interior images predicted (one batch
    of all interior images of all chains)."""
    data = samples(chs, {j: dict(x=ch.ctx.spins(ch.chain0).reshape(-1, 4)) for j, ch in enumerate(chs)})
    pred = W.predict(net, data["init"], data["feat"])
    out, k = [], 0
    for ch in chs:
        x = ch.ctx.spins(ch.chain0).float().clone()
        for v in range(1, ch.M - 1):
            x[v] = pred[k]
            k += 1
        out.append(x)
    return out


def ansatz_paths(chs):
    """Trivial guess: Neel profiles theta(r) = pi (1 - r / R_v) of the
    skyrmion's helicity, R_v shrinking linearly from the relaxed skyrmion's
    radius (where its n_z changes sign) to zero along the chain."""
    out = []
    for ch in chs:
        g = ch.draw["geometry"]
        r = I.site_positions(g)
        c = r.mean(axis=0)
        sk = ch.chain0[-1]
        d = np.linalg.norm(r - c, axis=1)
        core = d[sk[:, 2] < 0]
        R = float(core.max()) + 0.5 if core.size else float(ch.draw["radius"])
        # the path runs from the ferromagnet (image 0) to the skyrmion (image M-1)
        x = np.array(ch.chain0, copy=True)
        for v in range(1, ch.M - 1):
            Rv = R * v / (ch.M - 1.0)
            x[v] = I.neel_skyrmion(r, c, Rv, I.SKYRMION_HELICITY) if Rv > 0.5 else I.ferromagnet(ch.N)
        out.append(ch.ctx.spins(x))
    return out


def barrier(ch, x):
    """FP64 barrier of a converged chain: highest image minus image 0."""
    c64 = B.Context(ch.draw["geometry"], ch.draw["hamiltonian"], "f64")
    xs = x.view(ch.M, ch.N, 4).double()
    E = np.array([c64.energy(xs[m].contiguous())[0].item() for m in range(ch.M)])
    c64.close()
    return float(E.max() - E[0])


def evaluate(net, n, seed=SEEDS["heldout"], log=print):
    chs = chains(seed, n)
    orig = [np.array(ch.chain0, copy=True) for ch in chs]
    res = {}
    for arm in ("geodesic", "ansatz", "network"):
        for ch, o in zip(chs, orig):
            ch.chain0 = np.array(o, copy=True)
        net_s = 0.0
        starts = None
        if arm == "ansatz":
            starts = ansatz_paths(chs)
        elif arm == "network":
            with W._Timer() as t:
                starts = predicted_paths(net, chs)
            net_s = t.seconds
        state, sec = converge(chs, starts)
        its = np.array([state[k]["iters"] for k in range(len(chs))])
        bars = np.array([barrier(ch, state[k]["x"]) for k, ch in enumerate(chs)])
        res[arm] = dict(seconds=sec + net_s, network_seconds=net_s, mean_iterations=float(its.mean()),
                        max_iterations=int(its.max()), converged=int(sum(state[k]["fmax"] < TOL for k in state)),
                        barriers=bars, iters=its)
        log("%s: %.2f s, mean iterations %.0f" % (arm, sec + net_s, its.mean()))
    # a chain "matches" when its barrier equals the geodesic arm's to 1e-4
    # relative (FP32 chains converged to 1e-5 meV/rad agree to ~1e-5); the
    # others converged onto another saddle (e.g. a collapse off the
    # lattice-symmetric centre) and are counted as lower or higher
    ref = res["geodesic"]["barriers"]
    ref_it = res["geodesic"].pop("iters")
    for arm in res:
        b = res[arm].pop("barriers")
        its = res[arm].pop("iters", ref_it)
        rel = (b - ref) / np.abs(ref)
        match = np.abs(rel) <= 1e-4
        res[arm]["matched"] = int(match.sum())
        res[arm]["lower"] = int((rel < -1e-4).sum())
        res[arm]["higher"] = int((rel > 1e-4).sum())
        res[arm]["iterations_on_matched"] = [int(its[match].sum()), int(ref_it[match].sum())]
        res[arm]["barrier_rel_diff_vs_geodesic_max"] = float(np.max(np.abs(rel)))
        res[arm]["barrier_meV_range"] = [float(b.min()), float(b.max())]
    for ch, o in zip(chs, orig):
        ch.chain0 = o
    return dict(chains=n, images=M_IMAGES, lattice=[L_SIDE, L_SIDE], tol=TOL, arms=res)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--train-n", type=int, default=320, help="training chains")
    ap.add_argument("--eval-n", type=int, default=48, help="held-out chains")
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default="", help="prefix of the parameter file (.npz) and record (.json) to write")
    ap.add_argument("--params", default="", help="evaluate these parameters instead of training")
    a = ap.parse_args(argv)
    torch.cuda.set_device(0)
    from . import build
    build.build()
    rec = {}
    if a.params:
        net = UN.UNet(L_SIDE, 64, W.load_params(a.params))
    else:
        t0 = time.perf_counter()
        chs = chains(SEEDS["train"], a.train_n)
        state, sec = converge(chs)
        data = samples(chs, state)
        rec["generate"] = dict(chains=a.train_n, samples=int(data["init"].shape[0]), gneb_seconds=sec,
                               wall_seconds=time.perf_counter() - t0)
        print("generated %d samples from %d chains (%.1f s of GNEB)" % (data["init"].shape[0], a.train_n, sec))
        for ch in chs:
            ch.ctx.close()
        net, hist = W.train(data, a.epochs, lr=a.lr)
        rec["train"] = dict(epochs=a.epochs, loss=hist)
        del data
        if a.out:
            W.save_params(a.out + ".npz", net.get_params())
    rec["evaluate"] = evaluate(net, a.eval_n)
    print(json.dumps(rec["evaluate"]))
    if a.out:
        with open(a.out + ".json", "w") as f:
            json.dump(rec, f, indent=1)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
