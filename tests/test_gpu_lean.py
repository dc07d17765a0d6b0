"""The lean FP32 stochastic Heun passes of the 27-point path (cubic_lean.cu).

They are taken for FP32 Heun calls on one lattice without the dipole term
whose xy plane is cut into whole 32 x 8 column tiles; the 128^3 benchmark
lattice is one.  They compute the same method as the general 27-point
passes with a smaller instruction budget per spin, so the checks are:

  * one step from an identical FP32 state against the FP64 oracle, every
    spin, to the FP32 bound of 1e-5 (periodic, open and mixed boundaries;
    no, bulk and interfacial DMI; with and without the thermal field);
  * five steps against the general passes of the same context type, to a
    bound of FP32 rounding differences (2e-6);
  * bit-identical results under every split of the (tile, plane) units
    between CTAs, and with one or two columns per thread (32 x 8 or 32 x 16
    tiles): the per-spin arithmetic depends on neither.
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


def _np(t):
    return t.double().cpu().numpy()[:, :3]


SC = I.cfg_sc_128(4)["hamiltonian"]
CASES = {
    # the benchmark's Hamiltonian (three shells, bulk DMI) on whole tiles
    "sc_32x16x6_periodic": (I.simple_cubic(32, 16, 6), SC),
    # two tiles across x, open along z (zero planes beyond the ends)
    "sc_64x8x5_open_z": (I.simple_cubic(64, 8, 5, periodic=(True, True, False)), dict(SC, B=[0.2, 0, 0.5])),
    # open everywhere: halo records outside the lattice are zero
    "sc_32x24x4_open": (I.simple_cubic(32, 24, 4, periodic=(False, False, False)),
                        dict(J=[1.0, -0.2], dmi_kind="bulk", D=[0.3], K=[0.1], Khat=[[0.3, 0.1, 1.0]],
                             B=[0.1, -0.2, 1.0])),
    # interfacial DMI (face vectors zhat x ohat) and a tilted axis
    "sc_32x8x7_interfacial": (I.simple_cubic(32, 8, 7, periodic=(True, False, True)),
                              dict(J=[1.0], dmi_kind="interfacial", D=[0.25], K=[0.05], Khat=[[0, 0, 1]])),
    # exchange only (no DMI term)
    "sc_32x8x3_no_dmi": (I.simple_cubic(32, 8, 3), dict(J=[1.0, 0.1, -0.05], K=[0.05], Khat=[[0, 0, 1]])),
    # the 2D square workload's lattice (one plane, open)
    "square_32x32_open": (I.cfg_square_32()["geometry"], I.cfg_square_32()["hamiltonian"]),
}


def _ctx(g, h, lean):
    c = B.Context(g, h, "f32")
    c.set_option("small_path", 0)
    c.set_option("cubic_lean", lean)
    return c


def test_lean_option_reports_when_the_passes_are_taken():
    for g, h in CASES.values():
        assert _ctx(g, h, 1).get_option("cubic_lean") == 1
        assert _ctx(g, h, 0).get_option("cubic_lean") == 0
    # ragged tiles, FP64, two columns per thread: the general passes
    c = _ctx(I.simple_cubic(33, 16, 4), SC, 1)
    assert c.get_option("cubic_lean") == 0
    assert B.Context(I.simple_cubic(32, 16, 4), SC, "f64").get_option("cubic_lean") == 0
    c = _ctx(I.simple_cubic(32, 8, 4), SC, 1)  # 8 rows: no whole 32 x 16 tiles
    c.set_option("cubic_rows", 2)
    assert c.get_option("cubic_lean") == 0
    c = _ctx(I.simple_cubic(32, 16, 4), SC, 1)
    c.set_option("cubic_rows", 2)
    assert c.get_option("cubic_lean") == 1


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("T", [0.0, 10.0])
def test_lean_step_matches_oracle(name, T):
    g, h = CASES[name]
    o = oracle.System(g, h)
    c = _ctx(g, h, 1)
    n0 = I.random_spins(o.N, 6).astype(np.float32).astype(np.float64)
    kw = dict(solver="heun", dt=1e-3, alpha=0.1, T=T, seed=1, step0=40)
    n = c.spins(n0)
    c.llg_step(n, 1, **kw)
    no = o.llg(n0, 1, **kw)
    assert np.abs(_np(n) - no).max() <= 1e-5
    assert np.abs(np.linalg.norm(_np(n), axis=1) - 1).max() <= 1e-6
    assert c.sync_status()[0] == 0


@pytest.mark.parametrize("name", list(CASES))
def test_lean_steps_match_the_general_passes(name):
    g, h = CASES[name]
    n0 = I.random_spins(int(np.prod(g["n_cells"])), 9)
    kw = dict(solver="heun", dt=2e-3, alpha=0.2, T=8.0, seed=3, step0=11, replica=2)
    out = []
    for lean in (1, 0):
        c = _ctx(g, h, lean)
        n = c.spins(n0)
        c.llg_step(n, 5, **kw)
        out.append(n)
    assert (out[0] - out[1]).abs().max().item() <= 2e-6


@pytest.mark.parametrize("name", [k for k, (g, h) in CASES.items() if g["n_cells"][1] % 16 == 0])
@pytest.mark.parametrize("T", [0.0, 10.0])
def test_lean_two_columns_per_thread_give_the_same_bits(name, T):
    # two adjacent columns per thread (32 x 16 tiles) share the rows they
    # read; the per-spin arithmetic is that of one column per thread
    g, h = CASES[name]
    n0 = I.random_spins(int(np.prod(g["n_cells"])), 12)
    kw = dict(solver="heun", dt=2e-3, alpha=0.2, T=T, seed=4, step0=7)
    out = []
    for rows in ((1, 1), (2, 2), (2, 1), (1, 2)):
        c = _ctx(g, h, 1)
        c.set_option("cubic_rows", rows[0])
        c.set_option("cubic_rows_corr", rows[1])
        assert c.get_option("cubic_lean") == 1
        n = c.spins(n0)
        c.llg_step(n, 4, **kw)
        out.append(n)
    for n in out[1:]:
        assert torch.equal(n, out[0])


@pytest.mark.parametrize("zc,zcc", [(1, 0), (2, 1), (5, 3), (7, 0), (40, 2), (1000, 11)])
@pytest.mark.parametrize("rows", [1, 2])
def test_lean_plane_chunking_is_exact(zc, zcc, rows):
    g, h = I.simple_cubic(64, 16, 23), dict(SC, B=[0.2, 0, 0.5])
    n0 = I.random_spins(int(np.prod(g["n_cells"])), 2)
    kw = dict(solver="heun", dt=1e-3, alpha=0.1, T=10.0, seed=3)
    c = _ctx(g, h, 1)
    c.set_option("cubic_rows", rows)
    a = c.spins(n0)
    c.llg_step(a, 3, **kw)
    c.set_option("planes_per_cta", zc)
    c.set_option("planes_per_cta_corr", zcc)
    assert c.get_option("cubic_lean") == 1
    b = c.spins(n0)
    c.llg_step(b, 3, **kw)
    assert torch.equal(a, b)
