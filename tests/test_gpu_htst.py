"""Hessian spectrum and HTST rate prefactor on the GPU (Sec. HTST, appendix
on the curved manifold) against the oracle's dense eigen-decomposition and
against closed forms.

Bounds: eigenvalues 1e-10 of the spectral radius (FP64 Lanczos over the
whole tangent space with full reorthogonalisation); log-determinants, Omega_0
and v 1e-8 relative (small eigenvalues enter through their logarithm).
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


def _np(t):
    return t.detach().cpu().numpy()[..., :3].astype(np.float64)


@pytest.mark.parametrize("L", [6, 32])
def test_spectrum_matches_dense_oracle(L):
    g = I.hexagonal(L, L - 1, periodic=(True, True), mu_s=2.0)
    h = dict(J=[1.0, 0.2], dmi_kind="interfacial", D=[0.35, 0.05], K=[0.1], Khat=[[0.2, 0, 1]], B=[0.1, 0, 1.1])
    o = oracle.System(g, h)
    c = B.Context(g, h, "f64")
    n0 = I.random_spins(o.N, 8)
    ev = c.hessian_spectrum(c.spins(n0))
    eo = o.hessian_eigen(n0)[0]
    scale = np.abs(eo).max()
    assert np.abs(ev - eo).max() <= 1e-10 * scale


def test_spectrum_of_the_ferromagnet_keeps_every_degenerate_eigenvalue():
    # 16 x 16 periodic square ferromagnet: 512 eigenvalues, most of them
    # four- or eight-fold degenerate -- the restarts at closed Krylov spaces
    # must find every copy
    L, mu_s, Bz, K, J = 16, 2.0, 0.7, 0.2, 1.0
    g = I.square(L, L, periodic=(True, True), mu_s=mu_s)
    c = B.Context(g, dict(J=[J], K=[K], Khat=[[0, 0, 1]], B=[0, 0, Bz]), "f64")
    ev = c.hessian_spectrum(c.spins(I.ferromagnet(c.N)))
    q = 2 * math.pi * np.arange(L) / L
    w = mu_s * oracle.MU_B * Bz + 2 * K + J * (4 - 2 * np.cos(q)[:, None] - 2 * np.cos(q)[None, :])
    ref = np.sort(np.concatenate([w.ravel(), w.ravel()]))
    assert np.abs(ev - ref).max() <= 1e-10 * ref.max()


def _single_spin(mu_s, K, Bx, Bz):
    from scipy.optimize import brentq
    mu = mu_s * oracle.MU_B
    dE = lambda p: 2 * K * math.cos(p) * math.sin(p) - mu * (Bx * math.cos(p) - Bz * math.sin(p))  # noqa: E731
    d2E = lambda p: 2 * K * math.cos(2 * p) + mu * (Bx * math.sin(p) + Bz * math.cos(p))  # noqa: E731
    E = lambda p: -K * math.cos(p) ** 2 - mu * (Bx * math.sin(p) + Bz * math.cos(p))  # noqa: E731
    grid = np.linspace(-math.pi, math.pi, 4001)
    roots = [brentq(dE, a, b, xtol=1e-15) for a, b in zip(grid[:-1], grid[1:]) if dE(a) * dE(b) < 0]
    lam = lambda p: (d2E(p), 2 * K * math.cos(p) ** 2 + mu * (Bx * math.sin(p) + Bz * math.cos(p)))  # noqa: E731
    pm = max([p for p in roots if min(lam(p)) > 0], key=E)
    ps = [p for p in roots if lam(p)[0] < 0 < lam(p)[1]][0]
    return pm, ps, lam(pm), mu


def test_htst_single_spin_closed_form():
    mu_s, K, Bx, Bz = 2.0, 1.0, 1.5, 3.0
    pm, ps, lm, mu = _single_spin(mu_s, K, Bx, Bz)
    c = B.Context(I.square(1, 1, mu_s=mu_s), dict(B=[Bx, 0, Bz], K=[K], Khat=[[0, 0, 1]]), "f64")
    nm = c.spins(np.array([[math.sin(pm), 0.0, math.cos(pm)]]))
    ns = c.spins(np.array([[math.sin(ps), 0.0, math.cos(ps)]]))
    r = c.htst(nm, ns, zero_tol=1e-9)
    freq = oracle.GAMMA / (2 * math.pi * mu) * math.sqrt(lm[0] * lm[1])
    assert r["n_neg_min"] == 0 and r["n_neg_sad"] == 1
    assert abs(r["prefactor"] - freq) <= 1e-10 * freq


def _converged_collapse_path():
    # the paper's HTST example in small: an isolated Neel skyrmion with J = 1,
    # D = 0.6 J (interfacial), B = 4 T, on a 12 x 12 periodic hexagonal
    # lattice, centred on a site and relaxed (metastable, 4.8 meV above the
    # ferromagnet); its collapse path by climbing-image GNEB in FP64.  The
    # minimum has two translational (near-)zero modes, the saddle one
    # negative mode and no zero mode.
    g = I.hexagonal(12, 12, periodic=(True, True), mu_s=2.0)
    h = dict(J=[1.0], dmi_kind="interfacial", D=[0.6], K=[0.0], Khat=[[0, 0, 1]], B=[0, 0, 4.0])
    c = B.Context(g, h, "f64")
    r = I.site_positions(g)
    centre = r[6 * 12 + 6]
    sk = c.spins(I.neel_skyrmion(r, centre, 2.5, I.SKYRMION_HELICITY))
    it, mt = c.minimise(sk, torch.zeros_like(sk), dt=0.1, tol=1e-11, max_iter=100000, check_every=500)
    assert mt < 1e-11
    assert abs(c.topological_charge(sk).item() + 1) < 1e-6
    chain0 = I.slerp_chain(_np(sk), I.ferromagnet(c.N), 9, r, centre)
    x = c.spins(chain0)
    v = torch.zeros_like(x)
    for _ in range(400):
        E, F = c.gneb_step(x, v, n_iter=250, k_spring=1.0, climbing=True, dt=0.2)
        if F.item() < 1e-9:
            break
    assert F.item() < 1e-9
    E = E.cpu().numpy()
    return g, h, c, x[0].contiguous(), x[int(np.argmax(E))].contiguous()


def test_htst_skyrmion_collapse_matches_oracle():
    g, h, c, nm, ns = _converged_collapse_path()
    o = oracle.System(g, h)
    zt = 1e-5
    r = c.htst(nm, ns, zero_tol=zt)
    ro = o.htst(_np(nm), _np(ns), zero_tol=zt)
    print("HTST 12x12 skyrmion collapse: dE %.6g meV, Omega0 %.6g, v %.6g, prefactor %.6g, lowest eigenvalues "
          "min %s sad %s" % (r["dE"], r["omega0"], r["v"], r["prefactor"], ro["eig_min"][:3], ro["eig_sad"][:3]))
    assert r["n_neg_sad"] == ro["n_neg_sad"] == 1
    assert r["n_neg_min"] == ro["n_neg_min"] == 0
    assert r["n_zero_min"] == 2 and r["n_zero_sad"] == 0
    assert (r["n_zero_min"], r["n_zero_sad"]) == (ro["n_zero_min"], ro["n_zero_sad"])
    for k in ("log_det_min", "log_det_sad"):
        assert abs(r[k] - ro[k]) <= 1e-9 * abs(ro[k]) + 1e-9
    for k in ("omega0", "v", "prefactor"):
        assert abs(r[k] - ro[k]) <= 1e-8 * abs(ro[k])
    assert abs(r["dE"] - ro["dE"]) <= 1e-10 * abs(ro["E_min"])
    assert abs(r["lambda_unstable"] - ro["lambda_unstable"]) <= 1e-10 * np.abs(ro["eig_sad"]).max()
