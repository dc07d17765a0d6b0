"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64 contexts must match the oracle to 1e-12 relative per evaluation and per
step; FP32 contexts to max |dn| <= 1e-5 per step from an identical input
state (and 1e-5 relative on fields).  Inputs come from the seeded generators
only.
"""
import math

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


def _cases():
    c1 = I.cfg_square_32()
    c2 = I.cfg_sc_128(4)
    return {
        "square32_open": (c1["geometry"], c1["hamiltonian"]),
        "sc_periodic_ragged": (dict(c2["geometry"], n_cells=[13, 11, 9]), dict(c2["hamiltonian"], B=[0.2, 0, 0.5])),
        "sc_periodic_n2": (dict(c2["geometry"], n_cells=[2, 3, 5]), c2["hamiltonian"]),
        "hex_periodic_2shells": (I.hexagonal(17, 15, periodic=(True, True), mu_s=2.0),
                                 dict(J=[1.0, 0.2], dmi_kind="interfacial", D=[0.3, 0.05], K=[0.1],
                                      Khat=[[0.3, 0, 1]], B=[0.1, -0.2, 1.5])),
        "two_basis_pairs": (dict(bravais=[[1, 0, 0], [0.3, 1.1, 0], [0.1, 0.2, 0.9]],
                                 basis=[[0, 0, 0], [0.4, 0.3, 0.25]], n_cells=[5, 4, 3], periodic=[1, 0, 1],
                                 lattice_constant=1.7, mu_s=[2.0, 0.8]),
                            dict(J=[1.0, -0.3], dmi_kind="bulk", D=[0.2], K=[0.1, 0.3],
                                 Khat=[[0, 0, 1], [1, 1, 0]], B=[0.3, 0.1, -0.4],
                                 pairs=[(0, 1, (1, 1, 0), 0.4, (0.1, -0.2, 0.3))])),
        "hex_dipole_open": (I.hexagonal(23, 19, mu_s=3.0),
                            dict(J=[1.0], dmi_kind="interfacial", D=[0.3], K=[0.2], Khat=[[0, 0, 1]],
                                 B=[0, 0, 0.3], dipole="fft")),
        "single_spin": (I.square(1, 1, mu_s=2.0), dict(B=[0, 0, 1.0], K=[0.3], Khat=[[1, 0, 0]])),
    }


CASES = _cases()


def _oracle(g, h):
    return oracle.System(g, h)


def _np(t):
    return t.detach().cpu().numpy()[..., :3].astype(np.float64)


@pytest.mark.parametrize("name", list(CASES))
def test_field_and_energy_fp64(name):
    g, h = CASES[name]
    o = _oracle(g, h)
    c = B.Context(g, h, "f64")
    n0 = I.random_spins(o.N, 3)
    n = c.spins(n0)
    Bg = _np(c.effective_field(n))
    Bo = o.field(n0)
    scale = np.abs(Bo).max() + 1e-300
    assert np.abs(Bg - Bo).max() <= 1e-12 * scale
    assert np.abs(_np(c.gradient(n)) + Bo).max() <= 1e-12 * scale
    e = c.energy(n).cpu().numpy()
    eo = o.energy(n0)
    assert np.abs(e - eo).max() <= 1e-12 * (np.abs(eo).max() + 1)
    t = c.max_torque(n).item()
    to = np.linalg.norm(np.cross(n0, Bo), axis=1).max()
    assert abs(t - to) <= 1e-12 * (to + 1)


@pytest.mark.parametrize("name", list(CASES))
def test_field_fp32(name):
    g, h = CASES[name]
    o = _oracle(g, h)
    c = B.Context(g, h, "f32")
    n0 = I.random_spins(o.N, 4)
    n0 = n0.astype(np.float32).astype(np.float64)
    Bg = _np(c.effective_field(c.spins(n0)))
    Bo = o.field(n0)
    assert np.abs(Bg - Bo).max() <= 1e-5 * np.abs(Bo).max()


CUBIC = ["square32_open", "sc_periodic_ragged", "sc_periodic_n2", "single_spin"]


def _ctx(g, h, prec, path):
    # "default": the library's choice (the single-CTA path for these small
    # lattices); "generic": one launch per pass with the neighbour-table
    # stencil; "cubic": the 27-point plane-streaming path
    c = B.Context(g, h, prec)
    if path == "generic":
        c.set_option("generic_stencil", 1)
        c.set_option("small_path", 0)
    elif path == "cubic":
        c.set_option("small_path", 0)
    return c


def test_cubic_path_detection():
    for name, (g, h) in CASES.items():
        c = B.Context(g, h, "f32")
        assert c.get_option("has_cubic_path") == (1 if name in CUBIC else 0), name


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("solver", ["depondt", "heun", "sib", "rk4"])
@pytest.mark.parametrize("T", [0.0, 10.0])
@pytest.mark.parametrize("path", ["default", "generic", "cubic"])
def test_llg_step_fp64(name, solver, T, path):
    if path == "cubic" and name not in CUBIC:
        pytest.skip("no 27-point path for this lattice")
    g, h = CASES[name]
    o = _oracle(g, h)
    c = _ctx(g, h, "f64", path)
    n0 = I.random_spins(o.N, 5)
    kw = dict(solver=solver, dt=2e-3, alpha=0.2, T=T, seed=77, step0=123456789012, replica=3)
    n = c.spins(n0)
    c.llg_step(n, 3, **kw)
    no = o.llg(n0, 3, **kw)
    assert np.abs(_np(n) - no).max() <= 1e-12


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("solver", ["depondt", "heun", "sib", "rk4"])
@pytest.mark.parametrize("path", ["default", "generic", "cubic"])
def test_llg_step_fp32_per_step(name, solver, path):
    if path == "generic" and name not in CUBIC:
        pytest.skip("generic is the default path here")
    if path == "cubic" and name not in CUBIC:
        pytest.skip("no 27-point path for this lattice")
    g, h = CASES[name]
    o = _oracle(g, h)
    c = _ctx(g, h, "f32", path)
    n0 = I.random_spins(o.N, 6).astype(np.float32).astype(np.float64)
    kw = dict(solver=solver, dt=1e-3, alpha=0.1, T=10.0, seed=1, step0=40)
    n = c.spins(n0)
    c.llg_step(n, 1, **kw)
    no = o.llg(n0, 1, **kw)
    assert np.abs(_np(n) - no).max() <= 1e-5
    assert np.abs(np.linalg.norm(_np(n), axis=1) - 1).max() <= 1e-6


def test_square32_depondt_1000_steps_fp64():
    # the 32x32 square workload: 1000 damped Depondt steps, spins and energy
    cfg = I.cfg_square_32()
    g, h, r = cfg["geometry"], cfg["hamiltonian"], cfg["run"]
    o = _oracle(g, h)
    c = B.Context(g, h, "f64")
    n0 = I.random_spins(o.N, cfg["spin_seed"])
    n = c.spins(n0)
    c.llg_step(n, r["n_steps"], solver=r["solver"], dt=r["dt"], alpha=r["alpha"])
    no = o.llg(n0, r["n_steps"], solver=r["solver"], dt=r["dt"], alpha=r["alpha"])
    assert np.abs(_np(n) - no).max() <= 1e-11
    eo = o.energy(no)[0]
    assert abs(c.energy(n)[0].item() - eo) <= 1e-12 * abs(eo)


def test_stochastic_heun_100_steps_fp64():
    cfg = I.cfg_sc_128(12)
    g, h, r = cfg["geometry"], cfg["hamiltonian"], cfg["run"]
    o = _oracle(g, h)
    c = B.Context(g, h, "f64")
    n0 = I.random_spins(o.N, cfg["spin_seed"])
    kw = dict(solver="heun", dt=r["dt"], alpha=r["alpha"], T=r["T"], seed=r["seed"])
    n = c.spins(n0)
    c.llg_step(n, 100, **kw)
    no = o.llg(n0, 100, **kw)
    assert np.abs(_np(n) - no).max() <= 1e-11


@pytest.mark.parametrize("zc,zcc", [(1, 0), (2, 1), (5, 3), (7, 0), (40, 2), (1000, 11)])
def test_cubic_plane_chunking_is_exact(zc, zcc):
    # the result may not depend on how (tile, plane) units are split between
    # CTAs, including runs that cross from one column tile to the next, nor
    # on the corrector taking a split of its own (zcc > 0)
    cfg = I.cfg_sc_128(4)
    g = dict(cfg["geometry"], n_cells=[37, 19, 23])
    c = B.Context(g, cfg["hamiltonian"], "f32")
    n0 = I.random_spins(c.N, 2)
    kw = dict(solver="heun", dt=1e-3, alpha=0.1, T=10.0, seed=3)
    a = c.spins(n0)
    c.llg_step(a, 3, **kw)
    c.set_option("planes_per_cta", zc)
    c.set_option("planes_per_cta_corr", zcc)
    assert c.get_option("planes_per_cta_corr") == (zcc or zc)
    b = c.spins(n0)
    c.llg_step(b, 3, **kw)
    assert torch.equal(a, b)


def test_autotune_keeps_spins_and_picks_a_valid_chunking():
    cfg = I.cfg_sc_128(4)
    g = dict(cfg["geometry"], n_cells=[40, 24, 30])
    c = B.Context(g, cfg["hamiltonian"], "f32")
    n = c.spins(I.random_spins(c.N, 3))
    before = n.clone()
    zc = c.autotune(n)
    assert torch.equal(n, before)
    assert zc >= 1 and c.get_option("planes_per_cta") == zc


def test_llg_resume_is_bit_exact_on_gpu():
    cfg = I.cfg_sc_128(8)
    c = B.Context(cfg["geometry"], cfg["hamiltonian"], "f32")
    n0 = I.random_spins(c.N, 1)
    kw = dict(solver="heun", dt=1e-3, alpha=0.1, T=10.0, seed=1)
    a = c.spins(n0)
    c.llg_step(a, 10, **kw)
    b = c.spins(n0)
    c.llg_step(b, 4, **kw)
    c.llg_step(b, 6, step0=4, **kw)
    assert torch.equal(a, b)


def test_dipole_fp32_against_direct_sum():
    g = I.hexagonal(37, 29, mu_s=3.0)
    h = dict(dipole="fft")
    o = _oracle(g, dict(dipole="direct"))
    n0 = I.random_spins(o.N, 9)
    Bo = o.dipole_field(n0, "direct")
    c = B.Context(g, h, "f32")
    Bg = _np(c.effective_field(c.spins(n0)))
    assert np.abs(Bg - Bo).max() <= 1e-5 * np.abs(Bo).max()
    c64 = B.Context(g, h, "f64")
    Bg64 = _np(c64.effective_field(c64.spins(n0)))
    assert np.abs(Bg64 - Bo).max() <= 1e-12 * np.abs(Bo).max()


def test_dipole_warp_fft_path_ragged_sizes():
    # 300 x 283 cells pad to 1024 x 1024: the FP32 warp-FFT path, with rows
    # not a multiple of its 4-row blocks; against the FP64 direct sum at
    # sampled sites and against the radix-2 kernels on every site
    g = I.hexagonal(300, 283, mu_s=3.0)
    h = dict(J=[1.0], dipole="fft")
    n0 = I.random_spins(300 * 283, 13)
    c = B.Context(g, h, "f32")
    Bf = _np(c.effective_field(c.spins(n0)))
    c.set_option("generic_fft", 1)
    Bg = _np(c.effective_field(c.spins(n0)))
    assert np.abs(Bf - Bg).max() <= 2e-6 * np.abs(Bg).max()
    o = _oracle(g, dict(J=[1.0], dipole="direct"))
    idx = np.random.default_rng(1).choice(o.N, 300, replace=False)
    idx = np.concatenate([idx, [0, 299, 300 * 282, o.N - 1]])
    ref = o.field(n0, dipole="none")[idx] + o.dipole_field_direct_at(n0, idx)
    assert np.abs(Bf[idx] - ref).max() <= 1e-5 * np.abs(ref).max()


def test_vp_minimiser_parity_fp64():
    c1 = I.cfg_square_32()
    g = dict(c1["geometry"], n_cells=[12, 10, 1], periodic=[1, 0, 0])
    h = c1["hamiltonian"]
    o = _oracle(g, h)
    c = B.Context(g, h, "f64")
    n0 = I.random_spins(o.N, 12)
    n, v = c.spins(n0), c.spins(np.zeros_like(n0))
    it, mt = c.minimise(n, v, dt=0.1, tol=0.0, max_iter=60, check_every=16)
    no, vo, ito, mto = o.minimise(n0, dt=0.1, tol=0.0, max_iter=60)
    assert it == ito == 60
    assert np.abs(_np(n) - no).max() <= 1e-10
    assert np.abs(_np(v) - vo).max() <= 1e-10
    assert abs(mt - mto) <= 1e-10 * mto
    # converge to a tolerance: same iteration count and final energy
    n, v = c.spins(n0), c.spins(np.zeros_like(n0))
    it, mt = c.minimise(n, v, dt=0.1, tol=1e-8, max_iter=20000, check_every=50)
    no, vo, ito, mto = o.minimise(n0, dt=0.1, tol=1e-8, max_iter=20000)
    # the iteration at which max torque first drops below tol depends on
    # rounding once the run is near it; the converged energy does not
    assert mt < 1e-8 and abs(it - ito) <= 10
    eo = o.energy(no)[0]
    assert abs(c.energy(n)[0].item() - eo) <= 1e-10 * abs(eo)


def test_gneb_parity_fp64():
    g = I.hexagonal(9, 8, periodic=(True, True), mu_s=2.0)
    h = dict(J=[1.0], dmi_kind="interfacial", D=[0.35], K=[0.08], Khat=[[0, 0, 1]], B=[0, 0, 1.2])
    o = _oracle(g, h)
    c = B.Context(g, h, "f64")
    r = I.site_positions(g)
    a = I.ferromagnet(o.N)
    b = I.neel_skyrmion(r, r.mean(axis=0), 3.5)
    chain0 = I.slerp_chain(a, b, 7, r, r.mean(axis=0))
    chain, vel = c.spins(chain0), c.spins(np.zeros_like(chain0))
    E, F = c.gneb_step(chain, vel, n_iter=25, k_spring=1.0, climbing=True, dt=0.1)
    ch_o, v_o, E_o, mf_o, it_o = o.gneb(chain0, n_iter=25, k_spring=1.0, climbing=True, dt=0.1)
    assert np.abs(_np(chain) - ch_o).max() <= 1e-10
    assert np.abs(_np(vel) - v_o).max() <= 1e-10
    assert np.abs(E.cpu().numpy() - E_o).max() <= 1e-10 * np.abs(E_o).max()
    assert abs(F.item() - mf_o) <= 1e-10 * mf_o
    # splitting the iterations over two calls gives the same chain
    chain2, vel2 = c.spins(chain0), c.spins(np.zeros_like(chain0))
    c.gneb_step(chain2, vel2, n_iter=10, dt=0.1)
    c.gneb_step(chain2, vel2, n_iter=15, dt=0.1)
    assert torch.equal(chain, chain2)


def test_gneb_stoner_wohlfarth_barrier_fp64():
    mu, K, Bz = 2.0, 1.0, 3.0
    g = I.square(1, 1, mu_s=mu)
    c = B.Context(g, dict(B=[0, 0, Bz], K=[K], Khat=[[0, 0, 1]]), "f64")
    chain0 = I.slerp_chain(np.array([[0, 0, -1.0]]), np.array([[0, 0, 1.0]]), 9)
    chain, vel = c.spins(chain0), c.spins(np.zeros_like(chain0))
    for _ in range(20):
        E, F = c.gneb_step(chain, vel, n_iter=50, dt=0.5)
        if F.item() < 1e-12:
            break
    hh = mu * oracle.MU_B * Bz / (2 * K)
    E = E.cpu().numpy()
    assert abs(E.max() - E[0] - K * (1 - hh) ** 2) < 1e-12


@pytest.mark.parametrize("zc,rows", [(None, 1), (3, 1), (128, 1), (None, 2), (7, 2)])
def test_sc128_heun_step_fp32_full_size(zc, rows):
    # the 128^3 stochastic Heun workload at full size, in the launch
    # configuration the benchmark uses (and two other plane chunkings),
    # every spin checked
    cfg = I.cfg_sc_128()
    g, h, r = cfg["geometry"], cfg["hamiltonian"], cfg["run"]
    o = _oracle(g, h)
    c = B.Context(g, h, "f32")
    assert c.get_option("has_cubic_path") == 1
    c.set_option("cubic_rows", rows)
    if zc is not None:
        c.set_option("planes_per_cta", zc)
    n0 = I.random_spins(o.N, cfg["spin_seed"]).astype(np.float32).astype(np.float64)
    kw = dict(solver="heun", dt=r["dt"], alpha=r["alpha"], T=r["T"], seed=r["seed"], step0=5000)
    n = c.spins(n0)
    c.llg_step(n, 1, **kw)
    no = o.llg(n0, 1, **kw)
    assert np.abs(_np(n) - no).max() <= 1e-5


def test_hex512_dipole_fp32_on_crop():
    # the 512x512 dipolar monolayer: FP32 FFT field against the FP64 direct
    # sum over all 262144 spins, at the sites of a 64x64 crop
    cfg = I.cfg_hex_dipole()
    g, h = cfg["geometry"], cfg["hamiltonian"]
    o = _oracle(g, dict(h, dipole="direct"))
    n0 = I.random_spins(o.N, cfg["spin_seed"])
    c = B.Context(g, dict(h), "f32")
    Bg = _np(c.effective_field(c.spins(n0)))
    Bl = o.field(n0, dipole="none")
    idx = np.array([(224 + y) * 512 + 224 + x for y in range(64) for x in range(64)])
    Bd = o.dipole_field_direct_at(n0, idx)
    ref = Bl[idx] + Bd
    assert np.abs(Bg[idx] - ref).max() <= 1e-5 * np.abs(ref).max()
    assert np.abs((Bg[idx] - Bl[idx]) - Bd).max() <= 1e-4 * np.abs(Bd).max()


def _batch_chains():
    out = []
    g = I.hexagonal(9, 8, periodic=(True, True), mu_s=2.0)
    h = dict(J=[1.0], dmi_kind="interfacial", D=[0.35], K=[0.08], Khat=[[0, 0, 1]], B=[0, 0, 1.2])
    r = I.site_positions(g)
    out.append((g, h, I.slerp_chain(I.ferromagnet(72), I.neel_skyrmion(r, r.mean(0), 3.5), 7, r, r.mean(0))))
    g = I.square(6, 5, periodic=(True, False), mu_s=1.5)
    h = dict(J=[1.0, 0.1], dmi_kind="interfacial", D=[0.2], K=[0.2], Khat=[[0, 0, 1]], B=[0, 0, 0.5])
    out.append((g, h, I.slerp_chain(I.random_spins(30, 1), I.random_spins(30, 2), 5)))
    g = I.simple_cubic(4, 4, 3, periodic=(True, True, False))
    h = dict(J=[1.0, -0.2], dmi_kind="bulk", D=[0.2], K=[0.05], Khat=[[0, 0, 1]], B=[0, 0, 0.3])
    out.append((g, h, I.slerp_chain(I.ferromagnet(48), I.ferromagnet(48, (0, 0.2, -1)), 4)))
    return out


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_gneb_batch_matches_single_chains(prec):
    chains = _batch_chains()
    ctxs, single, offs, Ms = [], [], [], []
    off = 0
    for g, h, ch0 in chains:
        c = B.Context(g, h, prec)
        ch, v = c.spins(ch0), c.spins(np.zeros_like(ch0))
        E, F = c.gneb_step(ch, v, n_iter=25, k_spring=0.7, climbing=True, dt=0.1)
        single.append((ch, v, E, F))
        ctxs.append(c)
        offs.append(off)
        Ms.append(ch0.shape[0])
        off += ch0.shape[0] * ch0.shape[1]
    flat = torch.cat([c.spins(ch0).reshape(-1, 4) for c, (_, _, ch0) in zip(ctxs, chains)])
    vel = torch.zeros_like(flat)
    E, F = B.gneb_batch_step(ctxs, flat, vel, offs, Ms, n_iter=25, k_spring=0.7, climbing=True, dt=0.1)
    e0 = 0
    for k, (ch, v, Es, Fs) in enumerate(single):
        n = ch.numel() // 4
        assert torch.equal(flat[offs[k]:offs[k] + n], ch.reshape(-1, 4))
        assert torch.equal(vel[offs[k]:offs[k] + n], v.reshape(-1, 4))
        assert torch.equal(E[e0:e0 + Ms[k]], Es)
        assert F[k].item() == Fs.item()
        e0 += Ms[k]
    if prec == "f64":
        for k, (g, h, ch0) in enumerate(chains):
            ch_o, v_o, E_o, mf_o, _ = _oracle(g, h).gneb(ch0, n_iter=25, k_spring=0.7, climbing=True, dt=0.1)
            assert np.abs(_np(single[k][0]) - ch_o).max() <= 1e-10


@pytest.mark.parametrize("periodic", [True, False])
def test_topological_charge_matches_oracle(periodic):
    L = 24
    g = I.hexagonal(L, L, periodic=(periodic, periodic))
    r = I.site_positions(g)
    n0 = I.perturbed(I.neel_skyrmion(r, r.mean(axis=0), 6.0), 0.05, 4)
    qo = _oracle(g, dict()).topological_charge(n0)
    for prec, tol in (("f64", 1e-12), ("f32", 1e-5)):
        c = B.Context(g, dict(J=[1.0]), prec)
        q = c.topological_charge(c.spins(n0)).item()
        assert abs(q - qo) <= tol
    if periodic:
        assert abs(qo + 1) < 1e-9


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_minimise_batch_matches_single_systems(prec):
    # systems of different sizes and Hamiltonians relaxed together must each
    # follow the single-system iteration exactly
    systems = [
        (I.hexagonal(12, 9, periodic=(True, True)), dict(J=[1.0], dmi_kind="interfacial", D=[0.3], K=[0.1],
                                                         Khat=[[0, 0, 1]], B=[0, 0, 1.0])),
        (I.square(7, 5, periodic=(True, False)), dict(J=[1.0, 0.2], dmi_kind="interfacial", D=[0.2], B=[0, 0, 2.0])),
        (I.simple_cubic(4, 3, 3), dict(J=[1.0], K=[0.3], Khat=[[1, 0, 0]], B=[0.1, 0, 0.5])),
    ]
    ctxs, single, offs = [], [], []
    off = 0
    for k, (g, h) in enumerate(systems):
        c = B.Context(g, h, prec)
        n0 = I.random_spins(c.N, 40 + k)
        n, v = c.spins(n0), c.spins(np.zeros_like(n0))
        it, mt = c.minimise(n, v, dt=0.1, tol=1e-7, max_iter=3000, check_every=50)
        ctxs.append(c)
        single.append((n0, n, v, it, mt))
        offs.append(off)
        off += c.N
    flat = torch.cat([c.spins(s[0]) for c, s in zip(ctxs, single)])
    vel = torch.zeros_like(flat)
    its, mts = B.minimise_batch(ctxs, flat, vel, offs, dt=0.1, tol=1e-7, max_iter=3000, check_every=50)
    for k, (n0, n, v, it, mt) in enumerate(single):
        N = ctxs[k].N
        assert its[k] == it and mts[k] == mt
        assert torch.equal(flat[offs[k]:offs[k] + N], n)
        assert torch.equal(vel[offs[k]:offs[k] + N], v)


def _skyrmion_chain_case(M=9):
    g = I.hexagonal(9, 8, periodic=(True, True), mu_s=2.0)
    h = dict(J=[1.0], dmi_kind="interfacial", D=[0.35], K=[0.08], Khat=[[0, 0, 1]], B=[0, 0, 1.2])
    r = I.site_positions(g)
    a = I.ferromagnet(I.n_spins(g))
    b = I.neel_skyrmion(r, r.mean(axis=0), 3.5)
    return g, h, I.slerp_chain(a, b, M, r, r.mean(axis=0))


@pytest.mark.parametrize("w", [0.0, 0.5])
def test_gneb_image_kinds_and_energy_weight_fp64(w):
    # explicit climbing and falling images and energy-weighted springs follow
    # the oracle iteration for iteration.  The velocity projection amplifies
    # rounding: a 1e-15 change of the start grows to ~1e-11 in 30 iterations
    # (measured on the oracle), so the chains are compared after 12.
    g, h, chain0 = _skyrmion_chain_case(9)
    o = _oracle(g, h)
    c = B.Context(g, h, "f64")
    kinds = ["normal", "normal", "falling", "normal", "climbing", "normal", "normal", "climbing", "normal"]
    chain, vel = c.spins(chain0), c.spins(np.zeros_like(chain0))
    E, F = c.gneb_step(chain, vel, n_iter=12, k_spring=1.0, dt=0.1, image_types=kinds, energy_weight=w)
    ch_o, v_o, E_o, mf_o, _ = o.gneb(chain0, n_iter=12, k_spring=1.0, dt=0.1, image_types=kinds, energy_weight=w)
    assert np.abs(_np(chain) - ch_o).max() <= 1e-11
    assert np.abs(_np(vel) - v_o).max() <= 1e-11
    assert np.abs(E.cpu().numpy() - E_o).max() <= 1e-12 * np.abs(E_o).max()
    assert abs(F.item() - mf_o) <= 1e-10 * mf_o


@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("f32", 1e-4)])
def test_gneb_path_analysis_matches_oracle(prec, tol):
    g, h, chain0 = _skyrmion_chain_case(7)
    o = _oracle(g, h)
    c = B.Context(g, h, prec)
    chain = c.spins(chain0)
    P = c.gneb_path(chain, n_interp=6, charge=True)
    Po = o.gneb_path(chain0, n_interp=6, charge=True)
    scale = np.abs(Po["E"]).max()
    assert np.abs(P["E"] - Po["E"]).max() <= tol * scale
    assert np.abs(P["r"] - Po["r"]).max() <= tol * Po["r"][-1]
    assert np.abs(P["slope"] - Po["slope"]).max() <= tol * max(1.0, np.abs(Po["slope"]).max()) * 10
    assert np.abs(P["E_interp"] - Po["E_interp"]).max() <= tol * scale * 10
    assert np.abs(P["Q"] - Po["Q"]).max() <= 10 * tol
    assert abs(Po["Q"][0]) < 1e-9 and abs(Po["Q"][-1] + 1) < 1e-6


def test_gneb_batch_with_image_kinds_matches_single_chains():
    g, h, chain0 = _skyrmion_chain_case(7)
    kinds = ["normal", "falling", "normal", "climbing", "normal", "normal", "normal"]
    ctxs = [B.Context(g, h, "f64"), B.Context(g, h, "f64")]
    single = []
    for c in ctxs:
        ch, v = c.spins(chain0), c.spins(np.zeros_like(chain0))
        c.gneb_step(ch, v, n_iter=20, dt=0.1, image_types=kinds, energy_weight=0.3)
        single.append(ch)
    N = ctxs[0].N
    flat = torch.cat([ctxs[0].spins(chain0).reshape(-1, 4)] * 2)
    vel = torch.zeros_like(flat)
    B.gneb_batch_step(ctxs, flat, vel, [0, 7 * N], [7, 7], n_iter=20, dt=0.1, image_types=kinds * 2,
                      energy_weight=0.3)
    for k in range(2):
        assert torch.equal(flat[k * 7 * N:(k + 1) * 7 * N].reshape(7, N, 4), single[k].reshape(7, N, 4))


MC_CASES = [
    ("sc4", I.simple_cubic(4, 4, 4), dict(J=[1.0, -0.2], dmi_kind="bulk", D=[0.2], K=[0.1], Khat=[[0, 0, 1]],
                                         B=[0, 0.3, 0.8]), 8),
    ("hex9", I.hexagonal(9, 9, periodic=(True, True), mu_s=2.0),
     dict(J=[1.0], dmi_kind="interfacial", D=[0.3], K=[0.05], Khat=[[0, 0, 1]], B=[0, 0, 1.0]), 9),
    ("hex6open", I.hexagonal(6, 5, periodic=(True, False), mu_s=3.0), dict(J=[1.0], B=[0.2, 0, 0.5]), 4),
    # nearest-neighbour bonds only: (c0 + c1 + c2) mod 2
    ("sc6nn", I.simple_cubic(6, 4, 4), dict(J=[1.0], dmi_kind="bulk", D=[0.25], K=[0.1], Khat=[[0, 0, 1]],
                                           B=[0, 0.3, 0.8]), 2),
    ("sq6x5open", I.square(6, 5, periodic=(True, False), mu_s=2.0), dict(J=[1.0], B=[0, 0, 0.4]), 2),
    # odd periodic extents: (c0 + c1 + c2) mod 3 (the product colouring has 27)
    ("sc9x3x3nn", I.simple_cubic(9, 3, 3), dict(J=[1.0], K=[0.1], Khat=[[0, 0, 1]], B=[0.2, 0, 0.5]), 3),
    # mod 5: no product colouring exists
    ("sc5nn", I.simple_cubic(5, 5, 5), dict(J=[1.0], dmi_kind="bulk", D=[0.2], B=[0, 0, 0.3]), 5),
]


@pytest.mark.parametrize("resident", [1, 0], ids=["resident", "per_colour"])
@pytest.mark.parametrize("name,g,h,ncol", MC_CASES, ids=[c[0] for c in MC_CASES])
def test_mc_sweeps_fp64_match_oracle(name, g, h, ncol, resident):
    o = _oracle(g, h)
    c = B.Context(g, h, "f64")
    c.set_option("mc_resident", resident)
    assert c.mc_colours() == ncol == o.mc_colours()
    R = 3
    T = [2.0, 8.0, 30.0]
    x0 = np.stack([I.random_spins(c.N, 70 + r) for r in range(R)])
    x = torch.stack([c.spins(x0[r]) for r in range(R)])
    # thermalisation with the adaptive cone, then sampling with the cone fixed
    cone, stats = c.mc_sweeps(x, T, 20, seed=9, target_accept=0.4, sample=False)
    cone, stats = c.mc_sweeps(x, T, 20, seed=9, sweep0=20, target_accept=0.0, sample=True, cone=cone, stats=stats)
    xo, co, so = o.mc(x0, T, 20, seed=9, target_accept=0.4, sample=False, order="coloured")
    xo, co, so = o.mc(xo, T, 20, seed=9, sweep0=20, target_accept=0.0, sample=True, cone=co, stats=so,
                      order="coloured")
    assert np.abs(_np(x) - xo).max() <= 1e-11
    assert np.abs(cone.cpu().numpy() - co).max() <= 1e-12
    st = stats.cpu().numpy()
    assert np.array_equal(st[:, 5:], so[:, 5:])          # sample, accepted and trial counts
    assert np.allclose(st[:, :5], so[:, :5], rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("resident", [1, 0], ids=["resident", "per_colour"])
def test_mc_graph_replay_and_resume_are_bit_exact(resident):
    # 40 sweeps in one call (one resident launch, or graph replay) equal 40
    # single-sweep calls
    g, h = MC_CASES[0][1], MC_CASES[0][2]
    c = B.Context(g, h, "f64")
    c.set_option("mc_resident", resident)
    x0 = c.spins(I.random_spins(c.N, 5))[None].repeat(2, 1, 1).contiguous()
    x1 = x0.clone()
    ca, sa = c.mc_sweeps(x0, [4.0, 9.0], 40, seed=3, target_accept=0.5)
    cb, sb = None, None
    for k in range(40):
        cb, sb = c.mc_sweeps(x1, [4.0, 9.0], 1, seed=3, sweep0=k, target_accept=0.5, cone=cb, stats=sb)
    assert torch.equal(x0, x1) and torch.equal(ca, cb) and torch.equal(sa, sb)


@pytest.mark.parametrize("dims,prec", [((10, 10, 10), "f32"), ((10, 10, 10), "f64"), ((12, 12, 12), "f32"),
                                       ((16, 16, 8), "f32"), ((9, 9, 9), "f32")])
def test_mc_resident_equals_per_colour_launches(dims, prec):
    # 29 replicas as in the Tc workload (10^3 is its smallest lattice; 16 x
    # 16 x 8 the largest the resident kernel takes; 9^3 has three colours):
    # one resident CTA per replica gives the spins, cones and counts of the
    # per-colour launches; the observable sums differ only in summation order
    g = I.simple_cubic(*dims, periodic=(True, True, True), mu_s=2.0)
    h = dict(J=[1.0])
    temps = list(np.round(np.arange(10.0, 24.0 + 1e-9, 0.5), 6))
    R = len(temps)
    x0 = np.stack([I.random_spins(int(np.prod(dims)), 300 + r) for r in range(R)])
    out = []
    for resident in (1, 0):
        c = B.Context(g, h, prec)
        c.set_option("mc_resident", resident)
        x = torch.stack([c.spins(x0[r]) for r in range(R)])
        cone, st = c.mc_sweeps(x, temps, 37, seed=4, target_accept=0.5, sample=True)
        cone, st = c.mc_sweeps(x, temps, 21, seed=4, sweep0=37, target_accept=0.0, cone=cone, stats=st)
        out.append((x, cone, st))
    (xa, ca, sa), (xb, cb, sb) = out
    assert torch.equal(xa, xb) and torch.equal(ca, cb)
    assert torch.equal(sa[:, 5:], sb[:, 5:])
    assert torch.allclose(sa[:, :5], sb[:, :5], rtol=1e-12, atol=0)


def test_mc_fp32_samples_the_same_distribution():
    # FP32 decisions differ from FP64 ones near the acceptance threshold, so
    # the FP32 chain is compared through its mean energy and magnetisation
    g = I.simple_cubic(8, 8, 8)
    h = dict(J=[1.0], B=[0, 0, 0.2])
    res = {}
    for prec in ("f64", "f32"):
        c = B.Context(g, h, prec)
        R = 16
        x = c.spins(I.ferromagnet(c.N))[None].repeat(R, 1, 1).contiguous()
        cone, st = c.mc_sweeps(x, [12.0] * R, 300, seed=1, target_accept=0.5, sample=False)
        cone, st = c.mc_sweeps(x, [12.0] * R, 1500, seed=1, sweep0=300, target_accept=0.0, cone=cone)
        st = st.cpu().numpy()
        res[prec] = (st[:, 3] / st[:, 5], st[:, 0] / st[:, 5])
    for k in range(2):
        a, b = res["f64"][k], res["f32"][k]
        err = np.sqrt(a.var() / len(a) + b.var() / len(b))
        assert abs(a.mean() - b.mean()) < 5 * err + 1e-12, (k, a.mean(), b.mean(), err)


HESS_CASE = (I.hexagonal(3, 3, periodic=(True, True), mu_s=2.0),
             dict(J=[1.0], dmi_kind="interfacial", D=[0.4], K=[0.3], Khat=[[0.2, 0.3, 0.93]], B=[0.1, -0.4, 1.3]))


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_hessian_apply_matches_oracle(prec, tol):
    g, h = HESS_CASE
    o = _oracle(g, h)
    c = B.Context(g, h, prec)
    n0 = I.random_spins(c.N, 17)
    v0 = np.random.default_rng(2).standard_normal((c.N, 3))
    out = c.hessian_apply(c.spins(n0), c.spins(v0))
    ref = o.hessian_apply(n0, v0)
    assert np.abs(_np(out) - ref).max() <= tol * np.abs(ref).max()


def test_lowest_mode_matches_dense_eigendecomposition():
    g, h = HESS_CASE
    o = _oracle(g, h)
    c = B.Context(g, h, "f64")
    n0 = I.random_spins(c.N, 17)
    lam, mode = c.lowest_mode(c.spins(n0), krylov=2 * c.N)
    lam_o, mode_o = o.lowest_mode(n0)
    assert abs(lam - lam_o) <= 1e-10 * max(1.0, abs(lam_o))
    assert abs(abs(np.sum(_np(mode) * mode_o)) - 1.0) < 1e-9


def test_lowest_mode_of_a_large_ferromagnet_is_the_magnon_gap():
    # 32 x 32 hexagonal ferromagnet along z, B and K along z, no DMI: the
    # lowest eigenvalue is the q = 0 magnon, mu B + 2K
    mu, Bz, K = 2.0, 0.8, 0.1
    g = I.hexagonal(32, 32, periodic=(True, True), mu_s=mu)
    c = B.Context(g, dict(J=[1.0], K=[K], Khat=[[0, 0, 1]], B=[0, 0, Bz]), "f64")
    lam, _ = c.lowest_mode(c.spins(I.perturbed(I.ferromagnet(c.N), 0.0, 0)), krylov=120)
    assert abs(lam - (mu * oracle.MU_B * Bz + 2 * K)) < 1e-8


@pytest.mark.parametrize("case", ["single", "hex3"])
def test_mmf_matches_oracle(case):
    if case == "single":
        g, h = I.square(1, 1, mu_s=2.0), dict(B=[0, 0, 2.0], K=[0.3], Khat=[[1, 0, 0]])
        n0 = np.array([[0.82, 0.33, 0.47]])
        it = 60
    else:
        g, h = HESS_CASE
        n0 = I.perturbed(I.ferromagnet(9), 0.3, 4)
        it = 15
    n0 = n0 / np.linalg.norm(n0, axis=1, keepdims=True)
    o = _oracle(g, h)
    c = B.Context(g, h, "f64")
    x, v, mode = c.spins(n0), c.spins(np.zeros_like(n0)), c.spins(np.zeros_like(n0))
    mf, lam = c.mmf(x, v, mode, it, dt=0.1, krylov=2 * c.N)
    xo, vo, Fo, lam_o = o.mmf(n0, it, dt=0.1)
    assert np.abs(_np(x) - xo).max() <= 1e-9
    assert abs(lam - lam_o) <= 1e-9 * max(1.0, abs(lam_o))
    assert abs(mf - np.linalg.norm(Fo, axis=1).max()) <= 1e-9 * max(1.0, mf)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("solver", ["depondt", "heun", "sib"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_small_lattice_path_equals_the_multi_launch_path(name, solver, prec):
    # the single-CTA kernel runs the grid kernels' per-spin code from shared
    # memory: the same bits after many steps, with and without the noise
    g, h = CASES[name]
    if h.get("dipole", "none") != "none":
        pytest.skip("the dipole term is not on the single-CTA path")
    for T in (0.0, 10.0):
        a, b = _ctx(g, h, prec, "default"), _ctx(g, h, prec, "generic")
        n0 = I.random_spins(a.N, 21)
        kw = dict(solver=solver, dt=2e-3, alpha=0.2, T=T, seed=5, step0=77, replica=1)
        x, y = a.spins(n0), b.spins(n0)
        a.llg_step(x, 40, **kw)
        b.llg_step(y, 40, **kw)
        assert torch.equal(x, y), (name, solver, prec, T)


@pytest.mark.parametrize("dims", [(13, 11, 9), (32, 16, 5), (40, 37, 6), (8, 8, 8)])
@pytest.mark.parametrize("solver", ["heun", "depondt", "sib", "rk4"])
def test_cubic_two_columns_per_thread_is_bit_identical(dims, solver):
    # the 27-point kernels with two columns per thread (32 x 16 tiles) run the
    # same per-spin arithmetic as with one (32 x 8): the same bits, on
    # ragged tiles and with several work splits
    c2 = I.cfg_sc_128(4)
    g, h = dict(c2["geometry"], n_cells=list(dims)), dict(c2["hamiltonian"], B=[0.2, 0, 0.5])
    n0 = I.random_spins(int(np.prod(dims)), 31)
    kw = dict(solver=solver, dt=2e-3, alpha=0.2, T=8.0, seed=3, step0=11)
    ref = None
    for rows, per in ((1, 0), (2, 0), (2, 1), (2, 3)):
        c = _ctx(g, h, "f32", "cubic")
        c.set_option("cubic_lean", 0)  # the general passes at both heights
        c.set_option("cubic_rows", rows)
        if per:
            c.set_option("planes_per_cta", per)
        assert c.get_option("cubic_rows") == rows
        n = c.spins(n0)
        c.llg_step(n, 5, **kw)
        if ref is None:
            ref = n
        else:
            assert torch.equal(n, ref), (rows, per)


def test_autotune_chooses_a_tile_height_and_split():
    cfg = I.cfg_sc_128(64)
    c = B.Context(cfg["geometry"], cfg["hamiltonian"], "f32")
    c.set_option("cubic_lean", 0)  # the general passes, whose heights give the same bits
    n = c.spins(I.random_spins(c.N, 1))
    n0 = n.clone()
    c.autotune(n)
    assert torch.equal(n, n0)
    assert c.get_option("cubic_rows") in (1, 2) and c.get_option("cubic_rows_corr") in (1, 2)
    assert c.get_option("planes_per_cta") >= 1 and c.get_option("planes_per_cta_corr") >= 1
    # whatever was chosen, the step gives the one-column result bit for bit
    ref = B.Context(cfg["geometry"], cfg["hamiltonian"], "f32")
    ref.set_option("small_path", 0)
    ref.set_option("cubic_lean", 0)
    m = ref.spins(I.random_spins(c.N, 1))
    kw = dict(solver="heun", dt=1e-3, alpha=0.1, T=10.0, seed=1)
    c.llg_step(n, 3, **kw)
    ref.llg_step(m, 3, **kw)
    assert torch.equal(n, m)
    # with the lean passes allowed (this lattice fits them) the autotuned step
    # stays within FP32 rounding of the general passes
    d = B.Context(cfg["geometry"], cfg["hamiltonian"], "f32")
    x = d.spins(I.random_spins(c.N, 1))
    d.autotune(x)
    d.llg_step(x, 3, **kw)
    assert (x - m).abs().max().item() <= 2e-6
