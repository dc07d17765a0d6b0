"""Edge cases of every GPU entry point: calls that do nothing, the smallest
chains and lattices, and states the dynamics must leave where they are."""
import numpy as np
import pytest
import torch

import oracle
from paper_1901_11350_gb300 import binding as B
from paper_1901_11350_gb300 import inputs as I

pytestmark = pytest.mark.gpu

HEX = (I.hexagonal(6, 6, periodic=(True, True), mu_s=2.0),
       dict(J=[1.0], dmi_kind="interfacial", D=[0.3], K=[0.1], Khat=[[0, 0, 1]], B=[0, 0, 1.0]))


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_zero_iteration_calls_change_nothing(prec):
    g, h = HEX
    c = B.Context(g, h, prec)
    n0 = c.spins(I.random_spins(c.N, 1))
    n = n0.clone()
    c.llg_step(n, 0, solver="heun", T=10.0)
    assert torch.equal(n, n0)
    v = c.spins(np.zeros((c.N, 3)))
    it, mt = c.minimise(n, v, max_iter=0)
    assert it == 0 and torch.equal(n, n0)
    rel = 1e-5 if prec == "f32" else 1e-10
    assert abs(mt - c.max_torque(n).item()) <= rel * mt
    x = torch.stack([n0.clone(), n0.clone()])
    cone, st = c.mc_sweeps(x, [5.0, 9.0], 0)
    assert torch.equal(x[0], n0) and torch.equal(x[1], n0) and float(st.abs().sum()) == 0.0
    chain = c.spins(I.slerp_chain(I.ferromagnet(c.N), I.random_spins(c.N, 2), 5))
    ch0 = chain.clone()
    vel = torch.zeros_like(chain)
    E, F = c.gneb_step(chain, vel, n_iter=0)
    assert torch.equal(chain, ch0)
    for k in range(5):  # per-image energies are the states' energies
        e = c.energy(chain[k].contiguous())[0].item()
        assert abs(E[k].item() - e) <= rel * abs(e)
    its, mts = B.minimise_batch([c], n0.clone(), torch.zeros_like(n0), [0], max_iter=0)
    assert its[0] == 0


def test_three_image_chain_matches_oracle():
    # the shortest chain: one movable image between the fixed endpoints
    g, h = HEX
    o = oracle.System(g, h)
    c = B.Context(g, h, "f64")
    r = I.site_positions(g)
    ch0 = I.slerp_chain(I.ferromagnet(c.N), I.neel_skyrmion(r, r.mean(axis=0), 2.5), 3, r, r.mean(axis=0))
    chain, vel = c.spins(ch0), c.spins(np.zeros_like(ch0))
    E, F = c.gneb_step(chain, vel, n_iter=10, dt=0.1)
    cho, vo, Eo, mfo, _ = o.gneb(ch0, n_iter=10, dt=0.1)
    assert np.abs(chain.cpu().numpy()[..., :3] - cho).max() <= 1e-11
    assert torch.equal(chain[0], c.spins(ch0[0])) and torch.equal(chain[2], c.spins(ch0[2]))


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_single_spin_everywhere(prec):
    # one spin in a field: LLG precesses and damps towards the field, the
    # minimiser aligns it, the Hessian is (mu B + 2K) on the tangent plane
    mu, Bz, K = 2.0, 1.0, 0.2
    c = B.Context(I.square(1, 1, mu_s=mu), dict(B=[0, 0, Bz], K=[K], Khat=[[0, 0, 1]]), prec)
    n = c.spins(np.array([[1.0, 0.0, 0.0]]))
    c.llg_step(n, 2000, solver="depondt", dt=1e-2, alpha=0.5)
    assert n[0, 2].item() > 0.99
    v = c.spins(np.zeros((1, 3)))
    it, mt = c.minimise(n, v, dt=0.1, tol=1e-5)
    assert mt < 1e-5 and n[0, 2].item() > 1 - 1e-6
    # at exactly +z the Hessian is a multiple of the identity on the tangent
    # plane: the Krylov space stops growing after one vector
    lam, mode = c.lowest_mode(c.spins(np.array([[0.0, 0.0, 1.0]])), krylov=8)
    exact = mu * oracle.MU_B * Bz + 2 * K
    assert abs(lam - exact) <= (1e-6 if prec == "f32" else 1e-13) * exact
    assert abs(mode[0, 2].item()) < 1e-6 and abs(torch.linalg.norm(mode[0, :3]).item() - 1) < 1e-6


@pytest.mark.parametrize("solver", ["depondt", "heun", "sib", "rk4"])
def test_stationary_ferromagnet_stays(solver):
    # the ferromagnet along the field has zero torque: deterministic LLG,
    # the minimiser and T = 0 Monte Carlo leave it exactly where it is
    g = I.simple_cubic(6, 6, 4)
    h = dict(J=[1.0, 0.1], K=[0.1], Khat=[[0, 0, 1]], B=[0, 0, 1.0])
    c = B.Context(g, h, "f64")
    n = c.spins(I.ferromagnet(c.N))
    c.llg_step(n, 50, solver=solver, dt=1e-3, alpha=0.3)
    assert torch.allclose(n[:, 2], torch.ones_like(n[:, 2]), rtol=0, atol=1e-14)
    assert c.max_torque(n).item() < 1e-12
    x = n[None].contiguous()
    c.mc_sweeps(x, [0.0], 20, seed=2, target_accept=0.0, cone=torch.full((1,), 0.3, dtype=torch.float64,
                                                                          device="cuda"))
    assert torch.equal(x[0], n)  # T = 0 never accepts a move that does not lower the energy


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_krylov_beyond_tangent_dimension(prec):
    # 6 spins span a 12-dimensional tangent space; asking for 64 Lanczos
    # vectors must still give the lowest eigenvalue of the dense Hessian
    g = I.square(3, 2, periodic=(False, False), mu_s=2.0)
    h = dict(J=[1.0], dmi_kind="interfacial", D=[0.4], K=[0.1], Khat=[[0, 0, 1]], B=[0.2, 0, 0.5])
    o = oracle.System(g, h)
    c = B.Context(g, h, prec)
    n0 = I.random_spins(c.N, 8)
    if prec == "f32":
        n0 = n0.astype(np.float32).astype(np.float64)  # both sides at the same state
    Hd, _ = o.hessian_dense(n0)
    w = np.linalg.eigvalsh(0.5 * (Hd + Hd.T))
    lam, mode = c.lowest_mode(c.spins(n0), krylov=64)
    scale = np.abs(w).max()
    assert abs(lam - w[0]) <= (1e-5 if prec == "f32" else 1e-12) * scale
    m = mode[:, :3].double().cpu().numpy()
    assert abs(np.linalg.norm(m) - 1) < 1e-5
    assert np.abs(np.sum(m * n0, axis=1)).max() < 1e-5  # tangent to every spin
