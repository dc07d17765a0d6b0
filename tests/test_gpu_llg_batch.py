"""Stochastic LLG of many systems of different lattices in one launch per
pass (sp_llg_step_batch; Eq. 3-4, Appendix B): each system must come out bit
for bit as sp_llg_step leaves it alone, on the neighbour-list kernels, at its
own temperature and thermal stream -- for the systems of one batch differing
in lattice, size, Hamiltonian and moment.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1901_11350_gb300 import binding as B
from paper_1901_11350_gb300 import build
from paper_1901_11350_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    B.lib()


def _systems():
    g1 = I.hexagonal(20, 16, periodic=(True, True), mu_s=2.0)
    h1 = dict(J=[1.0], dmi_kind="interfacial", D=[0.3], K=[0.1], Khat=[[0, 0, 1]], B=[0, 0, 1.0])
    g2 = I.simple_cubic(8, 8, 6, periodic=(True, True, False), mu_s=3.0)
    h2 = dict(J=[1.0, -0.2, 0.05], dmi_kind="bulk", D=[0.2], K=[0.05], Khat=[[0, 0, 1]])
    g3 = I.square(12, 9, mu_s=1.5)
    h3 = dict(J=[1.0], dmi_kind="interfacial", D=[0.3], K=[0.1], Khat=[[1, 0, 0]], B=[0.2, 0, 0.7])
    g4 = dict(bravais=[[1, 0, 0], [0.3, 1.1, 0], [0.1, 0.2, 0.9]], basis=[[0, 0, 0], [0.4, 0.3, 0.25]],
              n_cells=[5, 4, 3], periodic=[1, 0, 1], lattice_constant=1.7, mu_s=[2.0, 0.8])
    h4 = dict(J=[1.0, -0.3], dmi_kind="bulk", D=[0.2], K=[0.1, 0.3], Khat=[[0, 0, 1], [1, 1, 0]], B=[0.3, 0.1, -0.4])
    return [(g1, h1, 4.0), (g2, h2, 12.0), (g3, h3, 0.0), (g4, h4, 7.5)]


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("solver", ["heun", "depondt", "sib"])
def test_batch_of_lattices_matches_single_calls(prec, solver):
    sy = _systems()
    ctxs, singles, offs, off = [], [], [], 0
    kw = dict(solver=solver, dt=2e-3, alpha=0.2, seed=9, step0=31)
    for k, (g, h, T) in enumerate(sy):
        c = B.Context(g, h, prec)
        c.set_option("generic_stencil", 1)
        c.set_option("small_path", 0)
        n = c.spins(I.random_spins(c.N, 50 + k))
        c.llg_step(n, 7, T=T, replica=3 + k, **kw)
        ctxs.append(c)
        singles.append(n)
        offs.append(off)
        off += c.N + 5  # a gap between systems
    flat = torch.zeros((off, 4), dtype=ctxs[0].dtype, device="cuda")
    for c, o, k in zip(ctxs, offs, range(len(sy))):
        flat[o:o + c.N] = c.spins(I.random_spins(c.N, 50 + k))
    B.llg_step_batch(ctxs, flat, offs, [T for _, _, T in sy], n_steps=7, replica=3, **kw)
    for c, o, n in zip(ctxs, offs, singles):
        assert torch.equal(flat[o:o + c.N], n)
    # a longer run continues the step counter: graph replays of 32 steps and
    # 8 single steps, against the single calls' per-step launches
    kw2 = dict(kw, step0=kw["step0"] + 7)
    B.llg_step_batch(ctxs, flat, offs, [T for _, _, T in sy], n_steps=72, replica=3, **kw2)
    for k, (c, o, n) in enumerate(zip(ctxs, offs, singles)):
        c.llg_step(n, 72, T=sy[k][2], replica=3 + k, **kw2)
        assert torch.equal(flat[o:o + c.N], n)
    assert ctxs[0].sync_status()[0] == 0


def test_batch_matches_the_oracle_in_fp64():
    # the batch against the oracle directly (stochastic Heun, identical
    # Philox streams): every system of the batch to 1e-12
    sy = _systems()
    ctxs, offs, off, starts = [], [], 0, []
    for k, (g, h, T) in enumerate(sy):
        c = B.Context(g, h, "f64")
        ctxs.append(c)
        offs.append(off)
        starts.append(I.random_spins(c.N, 70 + k))
        off += c.N
    flat = torch.cat([c.spins(s) for c, s in zip(ctxs, starts)])
    kw = dict(solver="heun", dt=1e-3, alpha=0.1, seed=4, step0=0)
    B.llg_step_batch(ctxs, flat, offs, [T for _, _, T in sy], n_steps=5, replica=0, **kw)
    for k, ((g, h, T), c, o) in enumerate(zip(sy, ctxs, offs)):
        ref = oracle.System(g, h).llg(starts[k], 5, T=T, replica=k, **kw)
        got = flat[o:o + c.N].cpu().numpy()[:, :3]
        assert np.abs(got - ref).max() <= 1e-12


def test_batch_rejects_rk4_and_overlaps():
    sy = _systems()[:2]
    ctxs = [B.Context(g, h, "f32") for g, h, _ in sy]
    flat = torch.zeros((ctxs[0].N + ctxs[1].N, 4), device="cuda")
    with pytest.raises(B.SpinError) as e:
        B.llg_step_batch(ctxs, flat, [0, ctxs[0].N], [1.0, 1.0], solver="rk4")
    assert e.value.code == -4
    with pytest.raises(B.SpinError) as e:
        B.llg_step_batch(ctxs, flat, [0, 10], [1.0, 1.0])
    assert e.value.code == -1
