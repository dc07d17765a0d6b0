"""Batched GNEB workload: skyrmion-collapse paths of many chains of uneven
lattice sizes and image counts, stepped together through
sp_gneb_batch_step.

Per chain: relax a Neel skyrmion ansatz with the velocity projection
minimiser, accept it when its topological charge is -1 +- 0.1 and its energy
lies above the ferromagnet's (an isolated metastable skyrmion), otherwise
redraw the chain's parameters; the initial path is the great-circle
interpolation from the ferromagnet (image 0) to the skyrmion (last image).
Chains leave the batch once their maximum force drops below the tolerance.
All arithmetic runs in the library's kernels; this module only orchestrates.
"""
import time

import numpy as np
import torch

from . import binding as B
from . import inputs as I


class Chain:
    def __init__(self, draw, ctx, chain0, Q, dE, relax_iters):
        self.draw = draw
        self.ctx = ctx
        self.chain0 = chain0
        self.Q = Q
        self.dE = dE
        self.relax_iters = relax_iters
        self.M = chain0.shape[0]
        self.N = chain0.shape[1]


def relax(ctx, state, dt=0.1, tol=1e-6, max_iter=200000):
    n = ctx.spins(state)
    v = torch.zeros_like(n)
    it, mt = ctx.minimise(n, v, dt=dt, tol=tol, max_iter=max_iter, check_every=256)
    return n, it, mt


def prepare(n_chains=48, seed=4, precision="f32", relax_tol=1e-5, max_attempts=12, sizes=(64, 96, 128),
            images=(12, 40), log=None):
    chains = []
    for c in range(n_chains):
        for attempt in range(max_attempts):
            d = I.gneb_draw(seed, c, attempt, sizes, images)
            ctx = B.Context(d["geometry"], d["hamiltonian"], precision)
            r = I.site_positions(d["geometry"])
            centre = r.mean(axis=0)
            sk, it, mt = relax(ctx, I.neel_skyrmion(r, centre, d["radius"], I.SKYRMION_HELICITY), tol=relax_tol)
            fm = ctx.spins(I.ferromagnet(ctx.N))
            Q = ctx.topological_charge(sk).item()
            dE = (ctx.energy(sk)[0] - ctx.energy(fm)[0]).item()
            if abs(Q + 1) <= 0.1 and dE > 0 and mt < relax_tol:
                skn = sk.cpu().numpy()[:, :3].astype(np.float64)
                chain0 = I.slerp_chain(I.ferromagnet(ctx.N), skn, d["n_images"], r, centre)
                chains.append(Chain(d, ctx, chain0, Q, dE, it))
                break
            if log:
                log("chain %d attempt %d rejected: Q=%.3f dE=%.3f torque=%.2g" % (c, attempt, Q, dE, mt))
        else:
            raise RuntimeError("no metastable skyrmion for chain %d after %d draws" % (c, max_attempts))
    return chains


def run_batched(chains, dt=0.1, k_spring=1.0, tol=1e-5, chunk=200, max_iter=200000, persistent=False):
    """Step all chains together until each max force < tol (chains leave the
    batch as they converge).  persistent: each call's iterations run in one
    persistent cooperative launch instead of one launch per pass.  Returns
    per-chain results and the summed device time of the batched calls (CUDA
    events on the launching stream)."""
    for ch in chains:
        ch.ctx.set_option("gneb_persistent", int(bool(persistent)))
    active = list(range(len(chains)))
    state = {}
    for k in active:
        ch = chains[k]
        state[k] = dict(x=ch.ctx.spins(ch.chain0).reshape(-1, 4), v=None, iters=0, fmax=np.inf, E=None)
        state[k]["v"] = torch.zeros_like(state[k]["x"])
    gpu_ms = 0.0
    st = torch.cuda.current_stream()
    while active:
        offs, Ms, ctxs = [], [], []
        off = 0
        for k in active:
            offs.append(off)
            Ms.append(chains[k].M)
            ctxs.append(chains[k].ctx)
            off += chains[k].M * chains[k].N
        x = torch.cat([state[k]["x"] for k in active])
        v = torch.cat([state[k]["v"] for k in active])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        E, F = B.gneb_batch_step(ctxs, x, v, offs, Ms, n_iter=chunk, k_spring=k_spring, climbing=True, dt=dt)
        e1.record(st)
        torch.cuda.synchronize()
        gpu_ms += e0.elapsed_time(e1)
        Fh = F.cpu().numpy()
        Eh = E.cpu().numpy()
        e_off = 0
        still = []
        for j, k in enumerate(active):
            n = chains[k].M * chains[k].N
            state[k]["x"] = x[offs[j]:offs[j] + n].clone()
            state[k]["v"] = v[offs[j]:offs[j] + n].clone()
            state[k]["iters"] += chunk
            state[k]["fmax"] = float(Fh[j])
            state[k]["E"] = Eh[e_off:e_off + chains[k].M].copy()
            e_off += chains[k].M
            if Fh[j] >= tol and state[k]["iters"] < max_iter:
                still.append(k)
        active = still
    return state, gpu_ms / 1e3


def run_per_chain(chains, precision="f64", dt=0.1, k_spring=1.0, tol=1e-5, chunk=200, max_iter=200000):
    """The plain loop: one chain after the other, each in its own context of
    `precision`, through sp_gneb_step.  Returns per-chain results and summed
    device time."""
    out = {}
    gpu_ms = 0.0
    st = torch.cuda.current_stream()
    for k, ch in enumerate(chains):
        ctx = B.Context(ch.draw["geometry"], ch.draw["hamiltonian"], precision)
        x = ctx.spins(ch.chain0)
        v = torch.zeros_like(x)
        iters, fmax, E = 0, np.inf, None
        while fmax >= tol and iters < max_iter:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            Et, Ft = ctx.gneb_step(x, v, n_iter=chunk, k_spring=k_spring, climbing=True, dt=dt)
            e1.record(st)
            torch.cuda.synchronize()
            gpu_ms += e0.elapsed_time(e1)
            iters += chunk
            fmax = Ft.item()
            E = Et.cpu().numpy()
        out[k] = dict(iters=iters, fmax=fmax, E=E, x=x)
        ctx.close()
    return out, gpu_ms / 1e3
