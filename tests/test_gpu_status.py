"""The boundary's device status word: non-finite results are reported.

A state with one NaN spin (planted on the host; nothing faults on the device)
goes through every entry point that takes spins.  Stream-ordered calls flag
the context's status word, which sp_sync_status (and the next call on the
context) returns as SP_ERR_NAN; calls with host results return SP_ERR_NAN
themselves.  A finite state leaves the word clear.
"""
import numpy as np
import pytest
import torch

from paper_1901_11350_gb300 import binding as B
from paper_1901_11350_gb300 import build
from paper_1901_11350_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NAN = -6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    B.lib()


HEX = (I.hexagonal(12, 10, periodic=(True, True), mu_s=2.0),
       dict(J=[1.0], dmi_kind="interfacial", D=[0.3], K=[0.1], Khat=[[0, 0, 1]], B=[0, 0, 1.0]))
SC = (I.simple_cubic(8, 8, 8, periodic=(True, True, True)),
      dict(J=[1.0, -0.2, 0.05], dmi_kind="bulk", D=[0.2], K=[0.05], Khat=[[0, 0, 1]]))


def _states(c, seed=3):
    good = I.random_spins(c.N, seed)
    bad = good.copy()
    bad[c.N // 3] = [np.nan, 0.0, 0.0]
    return c.spins(good), c.spins(bad)


def _flagged(c):
    rc, msg = c.sync_status()
    again, _ = c.sync_status()
    assert again == 0, "the status word is cleared once read"
    return rc, msg


def _raises_nan(fn):
    with pytest.raises(B.SpinError) as e:
        fn()
    assert e.value.code == NAN
    return str(e.value)


ASYNC = {
    "effective_field": lambda c, n: c.effective_field(n),
    "gradient": lambda c, n: c.gradient(n),
    "energy": lambda c, n: c.energy(n),
    "max_torque": lambda c, n: c.max_torque(n),
    "topological_charge": lambda c, n: c.topological_charge(n),
    "hessian_apply": lambda c, n: c.hessian_apply(n, c.spins(I.random_spins(c.N, 9))),
    "llg_heun": lambda c, n: c.llg_step(n, 3, solver="heun", T=5.0, seed=1),
    "llg_depondt": lambda c, n: c.llg_step(n, 3, solver="depondt"),
    "llg_rk4": lambda c, n: c.llg_step(n, 2, solver="rk4"),
    "llg_replicas": lambda c, n: c.llg_step_replicas(torch.stack([n, n]).contiguous(), [1.0, 5.0], 3),
    "mc_sweeps": lambda c, n: c.mc_sweeps(torch.stack([n, n]).contiguous(), [1.0, 5.0], 2),
    "sample": lambda c, n: c.sample(torch.stack([n, n]).contiguous()),
    "gneb_step": lambda c, n: c.gneb_step(torch.stack([c.spins(I.ferromagnet(c.N)), n,
                                                       c.spins(I.ferromagnet(c.N, (0, 0.3, -1)))]).contiguous(),
                                          torch.zeros((3, c.N, 4), dtype=c.dtype, device="cuda"), n_iter=2),
}


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("name", list(ASYNC))
def test_stream_ordered_calls_flag_nan(prec, name):
    c = B.Context(*HEX, prec)
    good, bad = _states(c)
    ASYNC[name](c, good)
    assert c.sync_status() == (0, "")
    ASYNC[name](c, bad)
    rc, msg = _flagged(c)
    assert rc == NAN, name
    assert "non-finite" in msg


@pytest.mark.parametrize("path", ["small", "cubic", "generic"])
def test_llg_paths_flag_nan(path):
    c = B.Context(*SC, "f32")
    if path != "small":
        c.set_option("small_path", 0)
    if path == "generic":
        c.set_option("generic_stencil", 1)
    good, bad = _states(c)
    c.llg_step(good, 4, solver="heun", T=10.0, seed=1)
    assert c.sync_status()[0] == 0
    c.llg_step(bad, 4, solver="heun", T=10.0, seed=1)
    assert _flagged(c)[0] == NAN


def test_next_call_surfaces_the_flag_and_clears_it():
    c = B.Context(*HEX, "f32")
    good, bad = _states(c)
    c.energy(bad)
    torch.cuda.synchronize()  # the check has run; nothing read the word yet
    msg = _raises_nan(lambda: c.effective_field(good))
    assert "energy" in msg
    B0 = c.effective_field(good)  # the word was cleared: the call runs
    assert c.sync_status()[0] == 0
    assert torch.isfinite(B0).all()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_host_result_calls_return_nan(prec):
    c = B.Context(*HEX, prec)
    good, bad = _states(c)
    v = torch.zeros_like(bad)
    _raises_nan(lambda: c.minimise(bad.clone(), v.clone(), tol=1e-9, max_iter=20, check_every=10))
    _raises_nan(lambda: B.minimise_batch([c], bad.clone(), v.clone(), [0], tol=1e-9, max_iter=20, check_every=10))
    chain = torch.stack([good, bad, good]).contiguous()
    _raises_nan(lambda: c.gneb_path(chain, n_interp=2))
    _raises_nan(lambda: c.lowest_mode(bad, krylov=8))
    _raises_nan(lambda: c.mmf(bad.clone(), v.clone(), torch.zeros_like(bad), 2, krylov=8))
    # and the finite state runs through all of them
    c.minimise(good.clone(), v.clone(), tol=1e-9, max_iter=20, check_every=10)
    c.lowest_mode(good, krylov=8)
    assert c.sync_status()[0] == 0


def test_gneb_batch_flags_nan():
    c0, c1 = B.Context(*HEX, "f32"), B.Context(*HEX, "f32")
    good, bad = _states(c0)
    a, b = c0.spins(I.ferromagnet(c0.N)), c0.spins(I.ferromagnet(c0.N, (0, 0.3, -1)))
    flat = torch.cat([torch.stack([a, good, b]).reshape(-1, 4), torch.stack([a, bad, b]).reshape(-1, 4)])
    vel = torch.zeros_like(flat)
    B.gneb_batch_step([c0, c1], flat, vel, [0, 3 * c0.N], [3, 3], n_iter=2)
    assert c0.sync_status()[0] == NAN
    assert c1.sync_status()[0] == 0  # the batch reports on the first chain's context
