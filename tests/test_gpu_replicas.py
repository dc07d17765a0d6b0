"""Batches of replicas at different temperatures (sp_llg_step_replicas) and
the observable accumulator (sp_sample), against the oracle, against single
calls, and against the thermal equilibrium of independent moments."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1901_11350_gb300 import binding as B
from paper_1901_11350_gb300 import inputs as I

pytestmark = pytest.mark.gpu

_c2 = I.cfg_sc_128(4)
LATTICES = {
    # the 27-point path applies (Heun and Depondt)
    "sc_periodic": (dict(_c2["geometry"], n_cells=[13, 11, 9]), dict(_c2["hamiltonian"], B=[0.2, 0, 0.5])),
    # neighbour-table path only
    "hex_periodic": (I.hexagonal(12, 10, periodic=(True, True), mu_s=2.0),
                     dict(J=[1.0, 0.1], dmi_kind="interfacial", D=[0.3], K=[0.1], Khat=[[0, 0, 1]], B=[0, 0, 0.7])),
}
TEMPS = [0.0, 4.0, 25.0]


def _np(t):
    return t.detach().cpu().numpy()[..., :3].astype(np.float64)


def _start(N, R):
    return np.stack([I.random_spins(N, 40 + r) for r in range(R)])


def _path(c, path):
    # "cubic": a fixed split keeps batches of these small lattices on the
    # 27-point kernels (the balanced split would send them to the per-spin
    # kernels); "generic": the neighbour-table kernels
    if path == "cubic":
        c.set_option("planes_per_cta", 3)
    elif path == "generic":
        c.set_option("generic_stencil", 1)


@pytest.mark.parametrize("name", list(LATTICES))
@pytest.mark.parametrize("solver", ["depondt", "heun", "sib", "rk4"])
@pytest.mark.parametrize("path", ["default", "cubic", "generic"])
def test_replicas_match_oracle_fp64(name, solver, path):
    g, h = LATTICES[name]
    o = oracle.System(g, h)
    c = B.Context(g, h, "f64")
    _path(c, path)
    n0 = _start(c.N, len(TEMPS))
    kw = dict(solver=solver, dt=2e-3, alpha=0.2, seed=91, step0=5000000000)
    x = c.spins(n0)
    c.llg_step_replicas(x, TEMPS, 3, replica=7, **kw)
    for r, T in enumerate(TEMPS):
        no = o.llg(n0[r], 3, T=T, replica=7 + r, **kw)
        assert np.abs(_np(x[r]) - no).max() <= 1e-12, (r, T)


@pytest.mark.parametrize("name", list(LATTICES))
@pytest.mark.parametrize("solver", ["depondt", "heun", "sib"])
@pytest.mark.parametrize("path", ["cubic", "generic"])
def test_replicas_equal_single_calls_fp32(name, solver, path):
    # one launch per pass for all replicas gives each replica exactly what a
    # call on that replica alone gives (on the same kernel family)
    g, h = LATTICES[name]
    c = B.Context(g, h, "f32")
    c.set_option("small_path", 0)
    _path(c, path)
    n0 = _start(c.N, len(TEMPS))
    kw = dict(solver=solver, dt=1e-3, alpha=0.1, seed=5, step0=11)
    x = c.spins(n0)
    c.llg_step_replicas(x, TEMPS, 4, replica=3, **kw)
    for r, T in enumerate(TEMPS):
        y = c.spins(n0[r])
        c.llg_step(y, 4, T=T, replica=3 + r, **kw)
        assert torch.equal(x[r], y), (r, T)


def test_replica_batches_are_independent_of_their_neighbours():
    # a replica's trajectory does not depend on which other replicas share
    # the batch or where in it the replica sits (27-point path)
    g, h = LATTICES["sc_periodic"]
    c = B.Context(g, h, "f32")
    _path(c, "cubic")
    n0 = _start(c.N, 3)
    kw = dict(solver="heun", dt=1e-3, alpha=0.1, seed=8)
    x = c.spins(n0)
    c.llg_step_replicas(x, [3.0, 9.0, 1.0], 5, replica=0, **kw)
    y = c.spins(n0[1:])
    c.llg_step_replicas(y, [9.0, 1.0], 5, replica=1, **kw)
    assert torch.equal(x[1], y[0]) and torch.equal(x[2], y[1])


@pytest.mark.parametrize("path", ["cubic", "generic"])
@pytest.mark.parametrize("solver", ["heun", "rk4"])
def test_graph_replay_equals_step_by_step(path, solver):
    # 70 steps in one call (two replayed 32-step graphs and 6 single steps)
    # against 70 calls of one step each (no graph), then a second call that
    # reuses the cached graph from another first step
    g, h = LATTICES["sc_periodic"]
    c = B.Context(g, h, "f32")
    _path(c, path)
    n0 = _start(c.N, 3)
    kw = dict(solver=solver, dt=1e-3, alpha=0.1, seed=21)
    temps = [2.0, 8.0, 30.0]
    x = c.spins(n0)
    c.llg_step_replicas(x, temps, 70, step0=1000, replica=4, **kw)
    c.llg_step_replicas(x, temps, 40, step0=5000, replica=4, **kw)
    y = c.spins(n0)
    for s in range(70):
        c.llg_step_replicas(y, temps, 1, step0=1000 + s, replica=4, **kw)
    for s in range(40):
        c.llg_step_replicas(y, temps, 1, step0=5000 + s, replica=4, **kw)
    assert torch.equal(x, y)


def test_a_batch_of_one_runs_at_its_own_temperature():
    g, h = LATTICES["sc_periodic"]
    c = B.Context(g, h, "f32")
    n0 = _start(c.N, 1)
    kw = dict(solver="heun", dt=1e-3, alpha=0.1, seed=8)
    x = c.spins(n0)
    c.llg_step_replicas(x, [9.0], 5, replica=2, **kw)
    y = c.spins(n0[0])
    c.llg_step(y, 5, T=9.0, replica=2, **kw)
    assert torch.equal(x[0], y)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_sample_is_the_definition(prec):
    g, h = LATTICES["hex_periodic"]
    o = oracle.System(g, h)
    c = B.Context(g, h, prec)
    R = 3
    n0 = _start(c.N, R)
    if prec == "f32":
        n0 = n0.astype(np.float32).astype(np.float64)
    x = c.spins(n0)
    st = c.sample(x)
    st = c.sample(x, st)
    st = st.cpu().numpy()
    tol = 1e-12 if prec == "f64" else 1e-6
    for r in range(R):
        m = np.linalg.norm(n0[r].sum(axis=0)) / c.N
        E = o.energy(n0[r])[0]
        assert abs(st[r, 0] - 2 * m) <= tol * 2 * m
        assert abs(st[r, 1] - 2 * m * m) <= 2 * tol * m * m
        assert abs(st[r, 2] - 2 * m ** 4) <= 4 * tol * m ** 4
        assert abs(st[r, 3] - 2 * E) <= tol * 2 * abs(E)
        assert abs(st[r, 4] - 2 * E * E) <= 2 * tol * E * E
        assert st[r, 5] == 2 and st[r, 6] == 0 and st[r, 7] == 0


def test_independent_moments_reach_the_langevin_magnetisation():
    # 4096 uncoupled moments in B = 5 T along z at three temperatures: the
    # sampled magnetisation is <n_z> = coth x - 1/x, x = mu B / (k_B T)
    mu, Bz = 2.0, 5.0
    temps = [2.0, 6.0, 20.0]
    c = B.Context(I.square(64, 64, mu_s=mu), dict(B=[0, 0, Bz]), "f32")
    R = len(temps)
    x = c.spins(np.tile(I.ferromagnet(c.N)[None], (R, 1, 1)))
    kw = dict(solver="heun", dt=5e-3, alpha=0.5, seed=12)
    step = 0
    c.llg_step_replicas(x, temps, 4000, step0=step, **kw)
    step += 4000
    st = None
    for k in range(400):
        c.llg_step_replicas(x, temps, 50, step0=step, **kw)
        step += 50
        st = c.sample(x, st)
    st = st.cpu().numpy()
    for r, T in enumerate(temps):
        xx = mu * oracle.MU_B * Bz / (oracle.K_B * T)
        L = 1.0 / math.tanh(xx) - 1.0 / xx
        m = st[r, 0] / st[r, 5]
        assert abs(m - L) < 0.01, (T, m, L)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("R", [1, 29])
def test_sample_of_large_lattices_is_the_definition(prec, R):
    # 30^3 with bulk DMI: with 29 replicas each thread of the observables
    # kernel sums a strided share of several spins; with one replica the
    # blocks cover one spin per thread
    g = I.simple_cubic(30, 30, 30, periodic=(True, True, True), mu_s=2.0)
    h = dict(J=[1.0], dmi_kind="bulk", D=[0.2], K=[0.05], Khat=[[0, 0, 1]], B=[0, 0.1, 0.4])
    o = oracle.System(g, h)
    c = B.Context(g, h, prec)
    n0 = np.stack([I.random_spins(c.N, 600 + r) for r in range(R)])
    n0[:, :, 2] += 0.5  # a net magnetisation well above the sampling noise
    n0 /= np.linalg.norm(n0, axis=2, keepdims=True)
    if prec == "f32":
        n0 = n0.astype(np.float32).astype(np.float64)
    st = c.sample(c.spins(n0)).cpu().numpy()
    tol = 1e-12 if prec == "f64" else 1e-6
    for r in sorted({0, R // 2, R - 1}):
        m = np.linalg.norm(n0[r].sum(axis=0)) / c.N
        E = o.energy(n0[r])[0]
        assert abs(st[r, 0] - m) <= tol * m, r
        assert abs(st[r, 3] - E) <= tol * abs(E), r
        assert st[r, 5] == 1
