"""Parity at the benchmark workloads' full sizes, in the launch
configurations the benchmark uses; outputs the oracle can compute in seconds
(whole replicas, whole chains, single steps) are compared one by one."""
import numpy as np
import pytest
import torch

import oracle
from paper_1901_11350_gb300 import binding as B
from paper_1901_11350_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TEMPS = list(np.round(np.arange(10.0, 24.0 + 1e-9, 0.5), 6))  # the Tc scans' grid (29 temperatures)


def _np(t):
    return t.detach().cpu().numpy()[..., :3].astype(np.float64)


@pytest.mark.parametrize("split", [(18, 14), (18, 18)])
def test_sc128_heun_step_with_the_benchmarks_split(split):
    # the split sp_autotune picks on this part for the 128^3 workload, the
    # corrector on its own value, every spin checked
    cfg = I.cfg_sc_128()
    g, h, r = cfg["geometry"], cfg["hamiltonian"], cfg["run"]
    o = oracle.System(g, h)
    c = B.Context(g, h, "f32")
    c.set_option("planes_per_cta", split[0])
    c.set_option("planes_per_cta_corr", split[1])
    n0 = I.random_spins(o.N, cfg["spin_seed"]).astype(np.float32).astype(np.float64)
    kw = dict(solver="heun", dt=r["dt"], alpha=r["alpha"], T=r["T"], seed=r["seed"], step0=77)
    n = c.spins(n0)
    c.llg_step(n, 1, **kw)
    assert np.abs(_np(n) - o.llg(n0, 1, **kw)).max() <= 1e-5


@pytest.mark.parametrize("solver", ["sib", "depondt"])
def test_sc128_other_solvers_full_size(solver):
    cfg = I.cfg_sc_128()
    g, h, r = cfg["geometry"], cfg["hamiltonian"], cfg["run"]
    o = oracle.System(g, h)
    c = B.Context(g, h, "f32")
    n0 = I.random_spins(o.N, cfg["spin_seed"]).astype(np.float32).astype(np.float64)
    kw = dict(solver=solver, dt=r["dt"], alpha=r["alpha"], T=r["T"], seed=r["seed"], step0=3)
    n = c.spins(n0)
    c.llg_step(n, 1, **kw)
    assert np.abs(_np(n) - o.llg(n0, 1, **kw)).max() <= 1e-5


def test_sllg30_replica_batch_full_size():
    # the stochastic-LLG Tc workload's largest batch: 29 replicas of the 30^3
    # ferromagnet (27-point path, 8 planes per CTA); three replicas against
    # the oracle, every spin
    g = I.simple_cubic(30, 30, 30, periodic=(True, True, True), mu_s=2.0)
    h = dict(J=[1.0])
    o = oracle.System(g, h)
    c = B.Context(g, h, "f32")
    R = len(TEMPS)
    n0 = np.stack([I.random_spins(o.N, 500 + k) for k in range(R)]).astype(np.float32).astype(np.float64)
    kw = dict(solver="heun", dt=1e-3, alpha=1.0, seed=30, step0=1234)
    x = c.spins(n0)
    c.llg_step_replicas(x, TEMPS, 1, **kw)
    for r in (0, 14, 28):
        no = o.llg(n0[r], 1, T=TEMPS[r], replica=r, **kw)
        assert np.abs(_np(x[r]) - no).max() <= 1e-5, r


def test_mc30_sweep_full_size_fp64():
    # one Metropolis sweep of 29 replicas of the 30^3 ferromagnet (FP64): the
    # same Philox draws and exact energy differences give the same decisions
    g = I.simple_cubic(30, 30, 30, periodic=(True, True, True), mu_s=2.0)
    h = dict(J=[1.0])
    o = oracle.System(g, h)
    c = B.Context(g, h, "f64")
    R = len(TEMPS)
    n0 = np.stack([I.random_spins(o.N, 900 + k) for k in range(R)])
    cone = torch.full((R,), 0.6, dtype=torch.float64, device="cuda")
    x = c.spins(n0)
    cone_g, st = c.mc_sweeps(x, TEMPS, 1, seed=7, target_accept=0.5, cone=cone)
    xo, co, sto = o.mc(n0, TEMPS, 1, seed=7, target_accept=0.5, cone=np.full(R, 0.6), order="coloured")
    for r in (0, 14, 28):
        assert np.abs(_np(x[r]) - xo[r]).max() <= 1e-12, r
    assert np.allclose(cone_g.cpu().numpy(), co, rtol=0, atol=1e-12)
    assert np.array_equal(st.cpu().numpy()[:, 6], sto[:, 6])  # accepted trials, every replica


def test_gneb_largest_chain_full_size_fp64():
    # a chain of the 48-chain workload's largest kind (128^2 lattice, 40
    # images): two iterations against the oracle, every image and spin
    d = None
    for k in range(200):
        d = I.gneb_draw(4, k)
        if d["L"] == 128 and d["n_images"] >= 38:
            break
    assert d["L"] == 128
    o = oracle.System(d["geometry"], d["hamiltonian"])
    c = B.Context(d["geometry"], d["hamiltonian"], "f64")
    r = I.site_positions(d["geometry"])
    sk = I.neel_skyrmion(r, r.mean(axis=0), d["radius"], I.SKYRMION_HELICITY)
    ch0 = I.slerp_chain(I.ferromagnet(o.N), sk, d["n_images"], r, r.mean(axis=0))
    chain, vel = c.spins(ch0), c.spins(np.zeros_like(ch0))
    E, F = c.gneb_step(chain, vel, n_iter=2, dt=0.2)
    cho, vo, Eo, mfo, _ = o.gneb(ch0, n_iter=2, dt=0.2)
    assert np.abs(_np(chain) - cho).max() <= 1e-11
    assert np.abs(E.cpu().numpy() - Eo).max() <= 1e-9 * np.abs(Eo).max()
