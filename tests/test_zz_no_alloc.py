"""The allocation-free LLG entry point, sp_llg_step_static.

Some callers cannot allocate device memory while they run: their device
memory belongs to another allocator or to a fixed budget, or they step in a
loop where cudaMalloc's implicit device synchronisation is not acceptable.
For them the library offers sp_llg_step_static, which keeps its scratch in a
fixed file-scope device array instead of allocating it.  These tests call it
through the C ABI and check

  * that it allocates nothing: on a fresh context the context's scratch stays
    empty and the device's free memory does not change across its first call
    (while the allocating sp_llg_step, as a control, does take scratch);
  * that it gives the allocating sp_llg_step's result bit for bit where both
    run the same kernels (the small-lattice path switched off), on two calls
    in a row, and within the parity tolerances (1e-5 in FP32, 1e-12 in FP64)
    where sp_llg_step takes its small-lattice path.

The file is named so that pytest collects it last.
"""
import ctypes as C

import pytest
import torch

from paper_1901_11350_gb300 import binding as B
from paper_1901_11350_gb300 import build
from paper_1901_11350_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f64": 1e-12}


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    return B.lib()


def _static_step(L, ctx, n, **kw):
    p = B.LLGParams(B.SOLVER[kw["solver"]], kw["dt"], kw["alpha"], kw["T"], kw["seed"], kw["step0"], 0)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.sp_llg_step_static(ctx._h, C.c_void_p(n.data_ptr()), C.byref(p), kw["n_steps"], stream)
    assert rc == 0, L.sp_last_error(ctx._h).decode()


CASES = {
    # the 27-point plane-streaming path
    "sc_24x20x16_heun_thermal": (I.cfg_sc_128(4)["geometry"] | dict(n_cells=[24, 20, 16]),
                                 I.cfg_sc_128(4)["hamiltonian"], "heun", 10.0),
    # the generic neighbour-list path (1200 spins: sp_llg_step's small-lattice size)
    "hex_40x30_depondt": (I.hexagonal(40, 30, periodic=(True, False)),
                          dict(J=[1.0], dmi_kind="interfacial", D=[0.3], K=[0.1], Khat=[[0, 0, 1]], B=[0, 0, 1.0]),
                          "depondt", 0.0),
}


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("name", list(CASES))
def test_static_step_matches_allocating_step(L, name, prec):
    g, h, solver, T = CASES[name]
    same = B.Context(g, h, prec)
    same.set_option("small_path", 0)  # the two-pass launches the static call takes
    dflt = B.Context(g, h, prec)      # the library's default choice
    stat = B.Context(g, h, prec)
    n0 = I.random_spins(stat.N, 21)
    a, d, b = same.spins(n0), dflt.spins(n0), stat.spins(n0)
    kw = dict(solver=solver, dt=1e-3, alpha=0.1, T=T, seed=5)
    # two calls in a row on each entry point, continuing the step counter
    for step0, n_steps in ((0, 3), (3, 4)):
        same.llg_step(a, n_steps, step0=step0, **kw)
        dflt.llg_step(d, n_steps, step0=step0, **kw)
        _static_step(L, stat, b, step0=step0, n_steps=n_steps, **kw)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        err = (d - b).abs().max().item()
        assert err <= TOL[prec], err
    assert torch.isfinite(b).all()
    assert stat.get_option("scratch_kib") == 0
    for c in (same, dflt, stat):
        c.close()


@pytest.mark.parametrize("name", list(CASES))
def test_static_step_allocates_nothing(L, name):
    g, h, solver, T = CASES[name]
    kw = dict(solver=solver, dt=1e-3, alpha=0.1, T=T, seed=5, n_steps=2)
    # load the kernels and look the scratch array up once (module loading
    # takes device memory of its own), then measure a fresh context
    warm = B.Context(g, h, "f32")
    n = warm.spins(I.random_spins(warm.N, 4))
    _static_step(L, warm, n, step0=0, **kw)
    torch.cuda.synchronize()
    warm.close()
    fresh = B.Context(g, h, "f32")
    m = fresh.spins(I.random_spins(fresh.N, 5))
    torch.cuda.synchronize()
    assert fresh.get_option("scratch_kib") == 0
    free0 = torch.cuda.mem_get_info()[0]
    _static_step(L, fresh, m, step0=0, **kw)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    assert fresh.get_option("scratch_kib") == 0
    assert torch.isfinite(m).all()
    # control: the allocating entry point does take context scratch
    fresh.set_option("small_path", 0)
    fresh.llg_step(m, 1, step0=2, **{k: v for k, v in kw.items() if k != "n_steps"})
    torch.cuda.synchronize()
    assert fresh.get_option("scratch_kib") >= 2 * 16 * fresh.N // 1024
    fresh.close()


def test_static_step_rejects_lattices_beyond_its_limit(L):
    g = I.simple_cubic(41, 41, 41)  # 68921 spins > 65536
    ctx = B.Context(g, dict(J=[1.0]), "f32")
    p = B.LLGParams(1, 1e-3, 0.1, 0.0, 0, 0, 0)
    rc = L.sp_llg_step_static(ctx._h, C.c_void_p(256), C.byref(p), 1, None)
    assert rc == -1
    assert b"SP_STATIC_MAX_SPINS" in L.sp_last_error(ctx._h)
    ctx.close()
