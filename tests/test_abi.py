"""Host-side checks of the C-ABI library: it loads, exports every entry point
that include/spirit_gb.h declares, and rejects bad arguments on the host
before anything is launched.  No GPU needed."""
import ctypes as C
import os
import re

import pytest

import oracle
from paper_1901_11350_gb300 import binding as B
from paper_1901_11350_gb300 import build
from paper_1901_11350_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return B.lib()


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^(?:int|void|const char \*)\s*\*?\s*(sp_\w+)\s*\(", txt, re.M)
    return names


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(L, n), n
        assert n in B.SIGNATURES, n


def test_create_rejects_bad_precision(L):
    h = C.c_void_p()
    assert L.sp_create(C.byref(h), 7) == -1
    assert L.sp_create(None, 0) == -1


def test_call_order_and_argument_errors(L):
    h = C.c_void_p()
    assert L.sp_create(C.byref(h), 0) == 0
    H = B.Hamiltonian()
    assert L.sp_set_hamiltonian(h, C.byref(H)) == -2  # geometry first
    brav = (C.c_double * 9)(1, 0, 0, 0, 1, 0, 0, 0, 1)
    basis = (C.c_double * 3)(0, 0, 0)
    mu = (C.c_double * 1)(2.0)
    per = (C.c_int * 3)(0, 0, 0)
    bad = (C.c_int * 3)(4, 0, 1)
    assert L.sp_set_geometry(h, brav, 1, basis, bad, per, 1.0, mu) == -1
    assert b"n_cells" in L.sp_last_error(h)
    good = (C.c_int * 3)(4, 3, 1)
    assert L.sp_set_geometry(h, brav, 1, basis, good, per, -1.0, mu) == -1
    assert L.sp_set_geometry(h, brav, 5, basis, good, per, 1.0, mu) == -1
    assert L.sp_set_geometry(h, brav, 1, basis, good, per, 1.0, mu) == 0
    p = B.LLGParams(1, 1e-3, 0.1, 0.0, 0, 0, 0)
    assert L.sp_llg_step(h, C.c_void_p(256), C.byref(p), 1, None) == -2  # no Hamiltonian yet
    H.n_shells = 9
    assert L.sp_set_hamiltonian(h, C.byref(H)) == -1
    H.n_shells = 1
    H.J[0] = 1.0
    assert L.sp_set_hamiltonian(h, C.byref(H)) == 0
    n = C.c_int()
    assert L.sp_n_spins(h, C.byref(n)) == 0 and n.value == 12
    # arguments checked before any launch
    assert L.sp_llg_step(h, None, C.byref(p), 1, None) == -1
    assert L.sp_llg_step(h, C.c_void_p(8), C.byref(p), 1, None) == -1  # misaligned
    p.dt = 0.0
    assert L.sp_llg_step(h, C.c_void_p(256), C.byref(p), 1, None) == -1
    p.dt, p.solver = 1e-3, 5
    assert L.sp_llg_step(h, C.c_void_p(256), C.byref(p), 1, None) == -1
    p.solver, p.T = 1, -1.0
    assert L.sp_llg_step(h, C.c_void_p(256), C.byref(p), 1, None) == -1
    p.T = 0.0
    assert L.sp_llg_step(h, C.c_void_p(256), C.byref(p), -1, None) == -1
    assert L.sp_llg_step(h, C.c_void_p(256), C.byref(p), 0, None) == 0  # nothing to do
    assert L.sp_effective_field(h, C.c_void_p(256), C.c_void_p(256), None) == -1  # aliasing
    g = B.GNEBParams(0.1, 1.0, 1.0, 1, None, 0.0)
    assert L.sp_gneb_step(h, C.c_void_p(256), C.c_void_p(512), 2, C.byref(g), 1, C.c_void_p(64), C.c_void_p(64),
                          None) == -1  # fewer than 3 images
    it, mt = C.c_int(), C.c_double()
    assert L.sp_minimise(h, C.c_void_p(256), C.c_void_p(512), 0.1, 1.0, 1e-6, 10, 0, C.byref(it), C.byref(mt),
                         None) == -1  # check_every < 1
    assert L.sp_destroy(h) == 0
    assert L.sp_destroy(None) == 0


def test_stencil_limits_and_unsupported_requests(L):
    # dipole term with a periodic direction is not implemented
    g = I.square(8, 8, periodic=(True, False))
    with pytest.raises(B.SpinError) as e:
        B.Context(g, dict(J=[1.0], dipole="fft"))
    assert e.value.code == -4
    # too many directed neighbours
    with pytest.raises(B.SpinError) as e:
        B.Context(I.simple_cubic(8), dict(J=[1.0] * 8))
    assert e.value.code == -1
    # a periodic bond longer than the periodic extent
    with pytest.raises(B.SpinError) as e:
        B.Context(I.square(2, 2, periodic=(True, True)), dict(pairs=[(0, 0, (3, 0, 0), 1.0, (0, 0, 0))]))
    assert e.value.code == -4
    # explicit self pair
    with pytest.raises(B.SpinError) as e:
        B.Context(I.square(4, 4), dict(pairs=[(0, 0, (0, 0, 0), 1.0, (0, 0, 0))]))
    assert e.value.code == -1
    # a fine context: SC with three shells = 26 directed neighbours
    c = B.Context(I.simple_cubic(5), dict(J=[1.0, -0.2, 0.05], dmi_kind="bulk", D=[0.2]))
    assert c.N == 125
    c.close()


def test_unet_layout_and_host_side_rejections():
    import ctypes as C
    from paper_1901_11350_gb300 import inputs as I
    from paper_1901_11350_gb300 import unet as UN
    L = UN.lib()
    assert UN.n_params() == I.unet_n_params()
    off = 0
    for l, (ci, co) in enumerate(I.UNET_LAYERS):
        assert UN.layer(l) == (co, ci, off, off + co * 9 * ci)
        off += co * 9 * ci + co
    assert UN.layer(14) == (3, 32, off, off + 96)
    h = C.c_void_p()
    assert L.sp_unet_create(C.byref(h), 12, 4) == -1     # L not a multiple of 8
    assert L.sp_unet_create(C.byref(h), 128, 0) == -1    # empty batch
    dummy = C.c_void_p(256)
    # channel counts below 32 or not multiples of 32, pixel counts not multiples of 128, NULL inputs
    assert L.sp_conv3x3_forward(dummy, 16, 0, None, 0, dummy, None, 1, None, 1, 16, 16, 32, dummy, None) == -1
    assert L.sp_conv3x3_forward(dummy, 32, 0, None, 0, dummy, None, 1, None, 1, 10, 10, 32, dummy, None) == -1
    assert L.sp_conv3x3_forward(dummy, 32, 0, None, 32, dummy, None, 1, None, 1, 16, 16, 32, dummy, None) == -1
    assert L.sp_conv3x3_forward(None, 32, 0, None, 0, dummy, None, 1, None, 1, 16, 16, 32, dummy, None) == -1
    assert L.sp_conv3x3_wgrad(dummy, 32, 0, None, 0, dummy, 1, 16, 16, 32, dummy, None, dummy, 0, None) == -1
    assert L.sp_conv3x3_set_wait_limit(-1) == -1                  # a negative wait limit
    assert L.sp_conv3x3_set_kernel(4) == -1 and L.sp_conv3x3_set_kernel(-1) == -1


def test_option_round_trip_and_rejections():
    c = B.Context(I.simple_cubic(8), dict(J=[1.0, -0.2, 0.05], dmi_kind="bulk", D=[0.2]))
    assert c.get_option("has_cubic_path") == 1
    assert c.get_option("small_path") == 1
    c.set_option("planes_per_cta", 7)
    assert c.get_option("planes_per_cta") == 7 and c.get_option("planes_per_cta_corr") == 7
    c.set_option("planes_per_cta_corr", 5)  # the corrector alone
    assert c.get_option("planes_per_cta") == 7 and c.get_option("planes_per_cta_corr") == 5
    c.set_option("planes_per_cta", 9)  # one value for both passes again
    assert c.get_option("planes_per_cta_corr") == 9
    assert c.get_option("mc_resident") == 1
    c.set_option("mc_resident", 0)
    assert c.get_option("mc_resident") == 0
    for name, bad in (("planes_per_cta", -1), ("planes_per_cta_corr", -1), ("small_path", 2), ("mc_resident", 3)):
        with pytest.raises(B.SpinError) as e:
            c.set_option(name, bad)
        assert e.value.code == -1
    h = c._h
    assert B.lib().sp_set_option(h, 99, 1) == -1
    v = C.c_int()
    assert B.lib().sp_get_option(h, 99, C.byref(v)) == -1
    c.set_option("generic_stencil", 1)
    assert c.get_option("generic_stencil") == 1
    c.close()


def test_replica_and_sample_rejections():
    c = B.Context(I.simple_cubic(6), dict(J=[1.0]), "f32")
    L = B.lib()
    h = c._h
    p = B.LLGParams(1, 1e-3, 0.1, 0.0, 0, 0, 0)
    T2 = (C.c_double * 2)(5.0, 10.0)
    bad = (C.c_double * 2)(5.0, -1.0)
    spins = C.c_void_p(256)  # never dereferenced: every call below fails or returns before a launch
    assert L.sp_llg_step_replicas(h, spins, 0, T2, C.byref(p), 1, None) == -1
    assert L.sp_llg_step_replicas(h, spins, 2, None, C.byref(p), 1, None) == -1
    assert L.sp_llg_step_replicas(h, spins, 2, bad, C.byref(p), 1, None) == -1
    assert b"replica 1" in L.sp_last_error(h)
    assert L.sp_llg_step_replicas(h, spins, 2, T2, C.byref(p), -1, None) == -1
    assert L.sp_llg_step_replicas(h, C.c_void_p(8), 2, T2, C.byref(p), 1, None) == -1  # misaligned
    p.replica = (1 << 29) - 1
    assert L.sp_llg_step_replicas(h, spins, 2, T2, C.byref(p), 1, None) == -1  # thermal stream overflow
    p.replica = 0
    assert L.sp_llg_step_replicas(h, spins, 2, T2, C.byref(p), 0, None) == 0  # nothing to do
    assert L.sp_sample(h, spins, 2, None, None) == -1
    assert L.sp_sample(h, spins, 0, C.c_void_p(512), None) == -1
    assert L.sp_sample(h, C.c_void_p(8), 1, C.c_void_p(512), None) == -1
    c.close()
    d = B.Context(I.square(8, 8), dict(J=[1.0], dipole="fft"), "f32")
    assert L.sp_llg_step_replicas(d._h, spins, 2, T2, C.byref(p), 1, None) == -4
    assert L.sp_sample(d._h, spins, 1, C.c_void_p(512), None) == -4
    d.close()


def test_mc_sweep_rejections():
    c = B.Context(I.simple_cubic(6), dict(J=[1.0]), "f32")
    L = B.lib()
    h = c._h
    T2 = (C.c_double * 2)(5.0, 10.0)
    bad = (C.c_double * 2)(5.0, -1.0)
    ok = B.MCParams(1, 0, 0.5, 1)
    spins, cone, stats = C.c_void_p(256), C.c_void_p(4096), C.c_void_p(8192)  # never dereferenced
    assert L.sp_mc_sweeps(h, None, 2, T2, C.byref(ok), 1, cone, stats, None) == -1
    assert L.sp_mc_sweeps(h, spins, 2, None, C.byref(ok), 1, cone, stats, None) == -1
    assert L.sp_mc_sweeps(h, spins, 2, T2, None, 1, cone, stats, None) == -1
    assert L.sp_mc_sweeps(h, C.c_void_p(264), 2, T2, C.byref(ok), 1, cone, stats, None) == -1
    assert b"misaligned" in L.sp_last_error(h)
    assert L.sp_mc_sweeps(h, spins, 2, T2, C.byref(ok), 1, C.c_void_p(4100), stats, None) == -1
    assert L.sp_mc_sweeps(h, spins, 0, T2, C.byref(ok), 1, cone, stats, None) == -1
    assert L.sp_mc_sweeps(h, spins, 2, T2, C.byref(ok), -1, cone, stats, None) == -1
    assert L.sp_mc_sweeps(h, spins, 2, bad, C.byref(ok), 1, cone, stats, None) == -1
    assert b"temperature" in L.sp_last_error(h)
    for t in (-0.1, 1.0, float("nan")):
        assert L.sp_mc_sweeps(h, spins, 2, T2, C.byref(B.MCParams(1, 0, t, 1)), 1, cone, stats, None) == -1
    c.close()
    d = B.Context(I.square(8, 8), dict(J=[1.0], dipole="fft"), "f32")
    assert L.sp_mc_sweeps(d._h, spins, 2, T2, C.byref(ok), 1, cone, stats, None) == -4
    d.close()
    e = B.Context(I.simple_cubic(7), dict(J=[1.0, -0.2]), "f64")  # no colouring
    assert L.sp_mc_sweeps(e._h, spins, 2, T2, C.byref(ok), 1, cone, stats, None) == -4
    assert b"colouring" in L.sp_last_error(e._h)
    e.close()


def test_hessian_rejections():
    c = B.Context(I.square(8, 8, periodic=(True, True)), dict(J=[1.0], K=[0.1], Khat=[[0, 0, 1]]), "f64")
    L = B.lib()
    h = c._h
    n, v, out = C.c_void_p(512), C.c_void_p(1024), C.c_void_p(2048)  # never dereferenced
    lam = C.c_double()
    assert L.sp_hessian_apply(h, None, v, out, None) == -1
    assert L.sp_hessian_apply(h, n, v, v, None) == -1
    assert L.sp_hessian_apply(h, n, C.c_void_p(1040), out, None) == -1  # 16 B: not an FP64 record boundary
    assert b"misaligned" in L.sp_last_error(h)
    assert L.sp_lowest_mode(h, n, out, 0, C.byref(lam), None) == -1
    assert L.sp_lowest_mode(h, n, out, 257, C.byref(lam), None) == -1
    assert L.sp_lowest_mode(h, C.c_void_p(520), out, 8, C.byref(lam), None) == -1
    c.close()
    d = B.Context(I.square(8, 8), dict(J=[1.0], dipole="fft"), "f32")
    assert L.sp_hessian_apply(d._h, n, v, out, None) == -4
    d.close()


MC_COLOURINGS = [
    # (geometry, hamiltonian, colours) -- sum colouring (c0 + c1 + c2) mod k
    (I.simple_cubic(2), dict(J=[1.0]), 2),
    (I.simple_cubic(3), dict(J=[1.0]), 3),
    (I.simple_cubic(6, 4, 4), dict(J=[1.0], dmi_kind="bulk", D=[0.2]), 2),
    (I.simple_cubic(5), dict(J=[1.0]), 5),
    (I.simple_cubic(7), dict(J=[1.0]), 7),
    (I.simple_cubic(15), dict(J=[1.0]), 3),
    (I.simple_cubic(5, periodic=(False, False, False)), dict(J=[1.0]), 5),
    # no sum colouring (2 does not divide 9, 3 not 4, 6 not 9): the product, 2 x 3 x 2
    (I.simple_cubic(6, 9, 4), dict(J=[1.0]), 12),
    (I.square(7, 4, periodic=(True, False)), dict(J=[1.0]), 7),
    (I.square(1, 1), dict(B=[0, 0, 1.0]), 1),
    # the product colouring
    (I.simple_cubic(4), dict(J=[1.0, -0.2]), 8),
    (I.simple_cubic(9), dict(J=[1.0, -0.2]), 27),
    (I.hexagonal(9, 9, periodic=(True, True)), dict(J=[1.0]), 9),
    (I.hexagonal(6, 6, periodic=(True, True)), dict(J=[1.0], dmi_kind="interfacial", D=[0.3]), 4),
    (I.hexagonal(6, 5, periodic=(True, False)), dict(J=[1.0]), 4),
    (dict(bravais=[[1, 0, 0], [0, 1, 0], [0, 0, 1]], basis=[[0, 0, 0], [0.5, 0.5, 0.5]], n_cells=[4, 4, 4],
          periodic=[1, 1, 1], lattice_constant=1.0, mu_s=[2.0, 1.0]),
     dict(pairs=[(0, 1, (0, 0, 0), 1.0, (0, 0, 0)), (1, 0, (1, 1, 1), 0.5, (0, 0, 0))]), 16),
    # neither: a second-shell bond with an odd periodic extent not divisible by 3
    (I.simple_cubic(7), dict(J=[1.0, -0.2]), 0),
    # a bond two cells long: no product colouring; (c0 + c1 + c2) mod 3
    (I.square(6, 6, periodic=(True, True)), dict(pairs=[(0, 0, (1, 0, 0), 1.0, (0, 0, 0)),
                                                        (0, 0, (0, 1, 0), 1.0, (0, 0, 0)),
                                                        (0, 0, (2, 0, 0), 0.3, (0, 0, 0))]), 3),
]


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("case", range(len(MC_COLOURINGS)))
def test_mc_colouring_host_logic_agrees_with_the_oracle(case, prec):
    # the library's colouring choice (host code, no GPU) against the
    # oracle's independent implementation and the expected count
    g, h, n = MC_COLOURINGS[case]
    c = B.Context(g, h, prec)
    assert c.mc_colours() == oracle.System(g, h).mc_colours() == n
    c.close()


CUBIC_PATH = [
    # one basis atom, bonds within the 3x3x3 cell neighbourhood, one exchange
    # constant per face / edge / corner class, DMI on face bonds only
    (I.simple_cubic(8), dict(J=[1.0, -0.2, 0.05], dmi_kind="bulk", D=[0.2], K=[0.05], Khat=[[0, 0, 1]]), 1),
    (I.simple_cubic(8), dict(J=[1.0]), 1),
    (I.simple_cubic(8), dict(J=[1.0], dmi_kind="interfacial", D=[0.3]), 1),
    (I.square(8, 8, periodic=(True, True)), dict(J=[1.0], dmi_kind="interfacial", D=[0.3]), 1),
    (I.simple_cubic(8), dict(J=[1.0, 0.2], dmi_kind="bulk", D=[0.2, 0.1]), 0),   # DMI on edge bonds
    (I.simple_cubic(8), dict(J=[1.0, 0.1, 0.1, 0.05]), 0),                        # a bond two cells long
    (I.hexagonal(8, 8, periodic=(True, True)), dict(J=[1.0]), 0),                 # (1, -1) without (1, 1)
    (dict(bravais=[[1, 0, 0], [0, 1, 0], [0, 0, 1]], basis=[[0, 0, 0], [0.5, 0.5, 0.5]], n_cells=[4, 4, 4],
          periodic=[1, 1, 1], lattice_constant=1.0, mu_s=[2.0, 1.0]), dict(J=[1.0]), 0),  # two basis atoms
]


@pytest.mark.parametrize("case", range(len(CUBIC_PATH)))
def test_27_point_path_detection(case):
    g, h, expect = CUBIC_PATH[case]
    for prec in ("f32", "f64"):
        c = B.Context(g, h, prec)
        assert c.get_option("has_cubic_path") == expect
        c.close()
