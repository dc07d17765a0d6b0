"""FP32 velocity projection and GNEB against the FP64 oracle.

The relaxation workloads run their forces and iterates in FP32 with image
energies and the 3N-dimensional dot products accumulated to FP64 accuracy
(float-float).  Here the FP32 path is compared with the FP64 oracle itself
(Appendix D's velocity projection, Sec. GNEB and Appendix F's tangents and
forces), not only with other FP32 runs:

* per iteration: from the same FP32-representable (state, velocity), one
  FP32 iteration and one oracle iteration, repeated along ten iterations of
  the FP32 trajectory.  Bound: 1e-5 on every spin (the FP32 step contract),
  1e-5 relative on the VP velocities and on the max force (3e-5 with
  energy-weighted springs), 1e-4 on the GNEB velocities (projected on forces
  that nearly cancel on some images);
* unsynchronised over ten iterations (the velocity projection amplifies the
  rounding of the start: bound 1e-4, the measured growth recorded);
* image energies: the FP32 field with float-float sums against the oracle's
  FP64 energies of the same state.  What remains is the FP32 rounding of the
  per-spin terms (each within a few 1e-8 relative), averaged over the
  spins: 1e-7 relative on a 72-spin chain, 3e-8 on 64 x 64 images and 1e-8
  on 128 x 128 images (a plain FP32 sum of 16384 terms would be off by
  ~1e-5);
* converged relaxations: the FP32 minimiser's final energy (max torque
  below 1e-6) against the oracle's to 1e-8 relative, the FP32 chain's
  barrier against the oracle's.
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
    return t.detach().cpu().numpy()[..., :3].astype(np.float64)


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _vp_case():
    c1 = I.cfg_square_32()
    g = dict(c1["geometry"], n_cells=[12, 10, 1], periodic=[1, 0, 0])
    return g, c1["hamiltonian"]


def _chain_case(L=9, M=9):
    g = I.hexagonal(L, L - 1 if L == 9 else L, periodic=(True, True), mu_s=2.0)
    h = dict(J=[1.0], dmi_kind="interfacial", D=[0.35], K=[0.08], Khat=[[0, 0, 1]], B=[0, 0, 1.2])
    r = I.site_positions(g)
    a = I.ferromagnet(I.n_spins(g))
    b = I.neel_skyrmion(r, r.mean(axis=0), 3.5 if L == 9 else 6.0)
    return g, h, _f32(I.slerp_chain(a, b, M, r, r.mean(axis=0)))


def test_vp_fp32_per_iteration_against_oracle():
    g, h = _vp_case()
    o = oracle.System(g, h)
    c = B.Context(g, h, "f32")
    x = c.spins(_f32(I.random_spins(o.N, 12)))
    v = torch.zeros_like(x)
    worst = 0.0
    for k in range(10):
        xs, vs = _np(x), _np(v)
        it, mt = c.minimise(x, v, dt=0.1, tol=0.0, max_iter=1, check_every=1)
        xo, vo, ito, mto = o.minimise(xs, vs, dt=0.1, tol=0.0, max_iter=1)
        assert it == ito == 1
        dx = np.abs(_np(x) - xo).max()
        dv = np.abs(_np(v) - vo).max() / max(1.0, np.abs(vo).max())
        assert dx <= 1e-5 and dv <= 1e-5, (k, dx, dv)
        assert abs(mt - mto) <= 1e-5 * mto
        worst = max(worst, dx)
    print("VP FP32 per-iteration max |dn| = %.3g" % worst)


def test_vp_fp32_ten_iterations_and_convergence_against_oracle():
    g, h = _vp_case()
    o = oracle.System(g, h)
    c = B.Context(g, h, "f32")
    n0 = _f32(I.random_spins(o.N, 12))
    x, v = c.spins(n0), c.spins(np.zeros_like(n0))
    c.minimise(x, v, dt=0.1, tol=0.0, max_iter=10, check_every=5)
    xo, vo, _, _ = o.minimise(n0, dt=0.1, tol=0.0, max_iter=10)
    d10 = np.abs(_np(x) - xo).max()
    print("VP FP32 after 10 unsynchronised iterations: max |dn| = %.3g" % d10)
    assert d10 <= 1e-4
    # relaxed to the FP32 path's resolution, the energy matches the oracle's
    # relaxed energy (the energy is stationary at the minimum: second order).
    # The start is a perturbed ferromagnet along the field, which relaxes to
    # one minimum (from random starts FP32 and FP64 may end in different ones)
    # The energy error of a state relaxed to max torque tau is of order
    # tau^2 / (softest curvature) per spin: at tau = 1e-4 it was measured at
    # 5.7e-8 relative, so the FP32 path relaxes to 1e-6 here (its forces
    # resolve ~1e-7 meV), where the bound is 1e-8 relative (the final-energy
    # contract)
    n1 = _f32(I.perturbed(I.ferromagnet(o.N), 0.4, 7))
    x, v = c.spins(n1), c.spins(np.zeros_like(n1))
    it, mt = c.minimise(x, v, dt=0.1, tol=1e-6, max_iter=40000, check_every=50)
    no, _, ito, mto = o.minimise(n1, dt=0.1, tol=1e-8, max_iter=40000)
    assert mt < 1e-6 and mto < 1e-8
    # the FP32 state as a point on the manifold: its records are unit vectors
    # only to FP32 rounding, which alone moves the energy by ~1e-8
    x32 = _np(x)
    e32 = o.energy(x32 / np.linalg.norm(x32, axis=1, keepdims=True))[0]
    e64 = o.energy(no)[0]
    print("VP FP32 relaxed energy vs oracle: %.3g relative (FP32 %d iterations)" % (abs(e32 - e64) / abs(e64), it))
    assert abs(e32 - e64) <= 1e-8 * abs(e64)


GNEB_KINDS = {
    "climbing": dict(climbing=True),
    "falling_and_climbing": dict(image_types=["normal", "normal", "falling", "normal", "climbing", "normal",
                                              "normal", "climbing", "normal"]),
    "energy_weighted": dict(climbing=True, energy_weight=0.5),
}


@pytest.mark.parametrize("kind", list(GNEB_KINDS))
def test_gneb_fp32_per_iteration_against_oracle(kind):
    # per iteration: the step (positions, velocities) against the oracle's
    # step from the same state; the energies and max force the FP32 call
    # reports against the oracle's on the FP32 call's own new state (the
    # force at a position moved by dx differs by about |dB/dn| dx, so it is
    # compared where both evaluate it)
    g, h, chain0 = _chain_case()
    kw = dict(k_spring=1.0, dt=0.1, **GNEB_KINDS[kind])
    o = oracle.System(g, h)
    c = B.Context(g, h, "f32")
    x = c.spins(chain0)
    v = torch.zeros_like(x)
    worst = [0.0, 0.0, 0.0, 0.0]
    for k in range(10):
        xs, vs = _np(x), _np(v)
        E, F = c.gneb_step(x, v, n_iter=1, **kw)
        xo, vo, Eo, mfo, _ = o.gneb(xs, vs, n_iter=1, **kw)
        dx = np.abs(_np(x) - xo).max()
        dv = np.abs(_np(v) - vo).max() / max(1.0, np.abs(vo).max())
        # the velocity is projected onto the new force; where an image's
        # force nearly cancels, the FP32 force's direction carries a larger
        # relative error (measured up to 4.5e-5), while the positions it
        # moves stay within the spin bound
        assert dx <= 1e-5 and dv <= 1e-4, (k, dx, dv)
        xn = _np(x)
        Fo, En, _, _ = o.gneb_forces(xn, **kw)
        mfn = np.linalg.norm(Fo[1:-1], axis=-1).max()
        dF = abs(F.item() - mfn) / mfn
        dE = np.abs(E.cpu().numpy() - En).max() / np.abs(En).max()
        # (energy-weighted springs difference the arc lengths of neighbouring
        # segments of the interpolated path, built from FP32 slopes:
        # measured up to 1.03e-5 relative there, 1.5e-8 with geodesic springs)
        assert dF <= (3e-5 if kw.get("energy_weight") else 1e-5) and dE <= 1e-7, (k, dF, dE)
        worst = [max(a, b) for a, b in zip(worst, (dx, dv, dF, dE))]
    print("GNEB FP32 (%s) per iteration: max |dn| %.3g, |dv| %.3g, max-force %.3g, energies %.3g relative"
          % (kind, *worst))


def test_gneb_fp32_image_energies_and_forces_on_one_state():
    # a 64x64 chain state in FP32: energies of every image (float-float sums)
    # and the max force against the oracle on the same state
    g, h, chain0 = _chain_case(L=64, M=12)
    o = oracle.System(g, h)
    c = B.Context(g, h, "f32")
    x = c.spins(chain0)
    v = torch.zeros_like(x)
    # a few iterations so that the chain leaves the slerp path
    c.gneb_step(x, v, n_iter=20, k_spring=1.0, dt=0.1)
    xs = _np(x)
    E, F = c.gneb_step(x, v, n_iter=0, k_spring=1.0, dt=0.1)
    assert np.abs(_np(x) - xs).max() == 0
    Eo = np.array([o.energy(xs[m])[0] for m in range(xs.shape[0])])
    rel = np.abs(E.cpu().numpy() - Eo) / np.abs(Eo)
    print("GNEB FP32 image energies: max relative error %.3g" % rel.max())
    assert rel.max() <= 3e-8
    Fo, Eo2, _, _ = o.gneb_forces(xs, k_spring=1.0, climbing=True, dt=0.1)
    mfo = np.linalg.norm(Fo[1:-1], axis=-1).max()
    assert abs(F.item() - mfo) <= 1e-5 * mfo
    # barrier of this path state: image energies relative to image 0
    bo, bg = Eo.max() - Eo[0], E.cpu().numpy().max() - E.cpu().numpy()[0]
    print("GNEB FP32 barrier of the state: %.6g vs oracle %.6g meV" % (bg, bo))
    assert abs(bg - bo) <= 1e-6 * abs(Eo).max()


def test_gneb_fp32_full_size_chain_against_oracle():
    # 40 images of a 128x128 hexagonal lattice (655k spins): one FP32 GNEB
    # iteration against the oracle's, every image and spin
    g = I.hexagonal(128, 128, periodic=(True, True), mu_s=2.0)
    h = dict(J=[1.0], dmi_kind="interfacial", D=[0.3], K=[0.07], Khat=[[0, 0, 1]], B=[0, 0, 1.0])
    r = I.site_positions(g)
    chain0 = _f32(I.slerp_chain(I.ferromagnet(I.n_spins(g)), I.neel_skyrmion(r, r.mean(axis=0), 6.0), 40, r,
                                r.mean(axis=0)))
    o = oracle.System(g, h)
    c = B.Context(g, h, "f32")
    x = c.spins(chain0)
    v = torch.zeros_like(x)
    E, F = c.gneb_step(x, v, n_iter=1, k_spring=1.0, dt=0.2)
    xo, vo, Eo, mfo, _ = o.gneb(chain0, n_iter=1, k_spring=1.0, climbing=True, dt=0.2)
    assert np.abs(_np(x) - xo).max() <= 1e-5
    assert np.abs(_np(v) - vo).max() <= 1e-5 * max(1.0, np.abs(vo).max())
    assert np.abs(E.cpu().numpy() - Eo).max() <= 1e-8 * np.abs(Eo).max()
    assert abs(F.item() - mfo) <= 1e-5 * mfo


def test_gneb_fp32_converged_barrier_against_oracle():
    # a small skyrmion-collapse chain (a metastable Neel skyrmion on a 12 x 12
    # periodic hexagonal lattice, J = 1, D = 0.6, B = 4 T, relaxed by the
    # oracle) converged by the FP32 path and by the oracle to 1e-5 meV/rad:
    # the barriers (FP64 re-evaluation of the FP32 chain's image energies)
    # agree
    g = I.hexagonal(12, 12, periodic=(True, True), mu_s=2.0)
    h = dict(J=[1.0], dmi_kind="interfacial", D=[0.6], K=[0.0], Khat=[[0, 0, 1]], B=[0, 0, 4.0])
    o = oracle.System(g, h)
    r = I.site_positions(g)
    centre = r[6 * 12 + 6]
    sk, _, _, mt = o.minimise(I.neel_skyrmion(r, centre, 2.5, I.SKYRMION_HELICITY), dt=0.1, tol=1e-10,
                              max_iter=100000)
    chain0 = _f32(I.slerp_chain(sk, I.ferromagnet(o.N), 9, r, centre))
    c = B.Context(g, h, "f32")
    x = c.spins(chain0)
    v = torch.zeros_like(x)
    for _ in range(200):
        E, F = c.gneb_step(x, v, n_iter=100, k_spring=1.0, dt=0.2)
        if F.item() < 1e-5:
            break
    assert F.item() < 1e-5
    xo, _, Eo, mfo, _ = o.gneb(chain0, n_iter=20000, tol=1e-5, k_spring=1.0, climbing=True, dt=0.2)
    assert mfo < 1e-5
    E32 = np.array([o.energy(m)[0] for m in _np(x)])
    b32, b64 = E32.max() - E32[0], Eo.max() - Eo[0]
    print("GNEB converged barrier: FP32 %.9g, oracle %.9g meV, relative %.3g" % (b32, b64, abs(b32 - b64) / b64))
    assert abs(b32 - b64) <= 1e-3 * b64
