"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints, closed forms, exact identities of a quadratic Hamiltonian,
brute force on tiny inputs, or published known-answer vectors.  Runs on the
CPU (no GPU marker).
"""
import math
import os

import numpy as np
import pytest
from scipy.special import zeta

import oracle
from paper_1901_11350_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ----------------------------------------------------------------------------
# Philox4x32-10 thermal-noise source (Eq. 4 and the text after it)
# ----------------------------------------------------------------------------
def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    return rows


def test_philox_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for r in rows:
        assert oracle.philox4x32_10(r[0:4], r[4:6]) == r[6:10]


def test_thermal_normals_statistics():
    # Eq. 4 text: three independent standard normals per spin and step.
    z = np.array([oracle.thermal_normals(123, step, 0, i) for step in range(40) for i in range(2500)])
    n = z.shape[0]
    assert abs(z.mean()) < 5 / math.sqrt(3 * n)
    assert np.allclose(z.mean(axis=0), 0, atol=5 / math.sqrt(n))
    assert np.allclose(z.var(axis=0), 1, atol=0.02)
    assert np.allclose(((z - z.mean(0)) ** 4).mean(0) / z.var(0) ** 2, 3.0, atol=0.1)
    c = np.corrcoef(z.T)
    assert np.abs(c - np.eye(3)).max() < 0.02
    # different replicas and seeds give different streams
    a = oracle.thermal_normals(1, 5, 0, 7)
    assert not np.allclose(a, oracle.thermal_normals(1, 5, 1, 7))
    assert not np.allclose(a, oracle.thermal_normals(2, 5, 0, 7))
    assert np.array_equal(a, oracle.thermal_normals(1, 5, 0, 7))


# ----------------------------------------------------------------------------
# Single-spin damped Larmor precession (closed form of Sec. LLG, Fig. 5)
# ----------------------------------------------------------------------------
def _larmor_error(solver, dt, t_end=100.0, alpha=0.1, B=1.0, mu=2.0):
    s = oracle.System(I.square(1, 1, mu_s=mu), dict(B=[0, 0, B]))
    n = np.array([[1.0, 0.0, 0.0]])
    err = 0.0
    g = oracle.GAMMA
    steps = int(round(t_end / dt))
    chunk = 100
    for k0 in range(0, steps, chunk):
        for k in range(k0 + 1, min(steps, k0 + chunk) + 1):
            n = s.llg(n, 1, solver=solver, dt=dt, alpha=alpha)
            t = k * dt
            nz = math.tanh(alpha * g * B * t / (1 + alpha ** 2))
            ph = g * B * t / (1 + alpha ** 2)
            r = math.sqrt(1 - nz * nz)
            exact = np.array([math.cos(ph) * r, math.sin(ph) * r, nz])
            err = max(err, float(np.abs(n[0] - exact).max()))
    return err, n


def test_larmor_depondt_matches_paper_error():
    # Fig. 5: B = 1 T, alpha = 0.1, dt = 10 fs; Depondt error around 3e-7.
    e1, n = _larmor_error("depondt", 0.01)
    assert 1e-7 < e1 < 5e-7
    assert abs(np.linalg.norm(n) - 1) < 1e-14
    e2, _ = _larmor_error("depondt", 0.005)
    assert 3.5 < e1 / e2 < 4.5  # second order


def test_larmor_heun_matches_paper_error():
    # Fig. 5 caption: Heun error within 1e-6.
    e1, _ = _larmor_error("heun", 0.01)
    assert 3e-7 < e1 < 1e-6
    e2, _ = _larmor_error("heun", 0.005)
    assert 3.5 < e1 / e2 < 4.5


# ----------------------------------------------------------------------------
# Geometry: neighbour shells against a brute-force O(N^2) distance scan
# ----------------------------------------------------------------------------
def _bond_counts(geometry, radii):
    r = I.site_positions(geometry)
    n0, n1, n2 = geometry["n_cells"]
    per = geometry["periodic"]
    A = np.asarray(geometry["bravais"], dtype=float) * geometry.get("lattice_constant", 1.0)
    counts = [0] * len(radii)
    shifts = [np.zeros(3)]
    if any(per):
        # all images within one period in each periodic direction
        rng = [range(-1, 2) if (per[k] and geometry["n_cells"][k] > 1) else range(0, 1) for k in range(3)]
        shifts = [a * A[0] * n0 + b * A[1] * n1 + c * A[2] * n2 for a in rng[0] for b in rng[1] for c in rng[2]]
    for i in range(len(r)):
        for sh in shifts:
            d = np.linalg.norm(r[i + 1:] + sh - r[i], axis=1) if not any(per) else \
                np.linalg.norm(r + sh - r[i], axis=1)
            for q, R in enumerate(radii):
                counts[q] += int(np.sum(np.abs(d - R) < 1e-9))
    if any(per):
        counts = [c // 2 for c in counts]
    return counts


@pytest.mark.parametrize("case", ["square_open", "hex_open", "sc_periodic"])
def test_ferromagnet_energy_closed_form(case):
    if case == "square_open":
        cfg = I.cfg_square_32()
        g, h, radii = cfg["geometry"], cfg["hamiltonian"], [1.0]
    elif case == "hex_open":
        g = I.hexagonal(13, 9, mu_s=3.0)
        h = dict(B=[0, 0, 0.7], K=[0.2], Khat=[[0, 0, 1]], J=[1.0, 0.3], dmi_kind="interfacial", D=[0.3])
        radii = [1.0, math.sqrt(3.0)]
    else:
        cfg = I.cfg_sc_128(6)
        g, h, radii = cfg["geometry"], cfg["hamiltonian"], [1.0, math.sqrt(2.0), math.sqrt(3.0)]
        h = dict(h, B=[0, 0, 0.4])
    s = oracle.System(g, h)
    for q, R in enumerate(radii):
        assert abs(s.shell_radius(q) - R) < 1e-12
    bonds = _bond_counts(g, radii)
    N = s.N
    mu = g["mu_s"][0]
    E = -sum(J * nb for J, nb in zip(h["J"], bonds)) - N * h["K"][0] - N * mu * oracle.MU_B * h["B"][2]
    e = s.energy(I.ferromagnet(N))
    assert abs(e[0] - E) < 1e-9 * abs(E)
    assert e[4] == 0.0  # DMI vanishes for a collinear state
    if case == "square_open":
        assert bonds == [1984]
        assert abs(E - (-1984 - 102.4 - 1024 * 2 * oracle.MU_B)) < 1e-9


def test_sc_shell_neighbour_counts():
    s = oracle.System(I.cfg_sc_128(5)["geometry"], I.cfg_sc_128(5)["hamiltonian"])
    assert s.n_neighbours(0) == 6 + 12 + 8
    s = oracle.System(I.hexagonal(8, 8, periodic=(True, True)), dict(J=[1.0, 0.5, 0.1]))
    assert s.n_neighbours(0) == 6 + 6 + 6
    assert abs(s.shell_radius(2) - 2.0) < 1e-12


# ----------------------------------------------------------------------------
# Flat spin spirals E(q) (closed forms for J shells + DMI)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("m", [1, 2, 3, 5])
def test_spiral_energy_sc_bulk_helix(m):
    L = 16
    cfg = I.cfg_sc_128(L)
    g, h = cfg["geometry"], cfg["hamiltonian"]
    s = oracle.System(g, h)
    q = 2 * math.pi * m / L
    n = I.flat_spiral(I.site_positions(g), [q, 0, 0], [0, 1, 0], [0, 0, 1])
    J1, J2, J3 = h["J"]
    D, K = h["D"][0], h["K"][0]
    Ec = -J1 * (math.cos(q) + 2) - J2 * (4 * math.cos(q) + 2) - 4 * J3 * math.cos(q) - D * math.sin(q) - K / 2
    assert abs(s.energy(n)[0] / s.N - Ec) < 1e-11


@pytest.mark.parametrize("m", [1, 2, 3])
def test_spiral_energy_hex_interfacial_cycloid(m):
    L = 24
    g = I.hexagonal(L, L, periodic=(True, True))
    J, D, K = 1.0, 0.3, 0.2
    s = oracle.System(g, dict(J=[J], dmi_kind="interfacial", D=[D], K=[K], Khat=[[0, 0, 1]]))
    q = 4 * math.pi * m / L
    n = I.flat_spiral(I.site_positions(g), [q, 0, 0], [0, 0, 1], [1, 0, 0])
    half_shell = [(1.0, 0.0), (0.5, math.sqrt(3) / 2), (-0.5, math.sqrt(3) / 2)]
    Ec = -sum(J * math.cos(q * dx) for dx, _ in half_shell) - D * sum(math.sin(q * dx) * dx for dx, _ in half_shell) - K / 2
    assert abs(s.energy(n)[0] / s.N - Ec) < 1e-11


def test_spiral_square_lattice_minimum():
    # NN square lattice cycloid: E(q)/N = -J(cos q + 1) - D sin q, minimum at tan q = D/J
    L = 40
    g = I.square(L, L, periodic=(True, True))
    J, D = 1.0, 0.3
    s = oracle.System(g, dict(J=[J], dmi_kind="interfacial", D=[D]))
    r = I.site_positions(g)
    E = []
    for m in range(0, 8):
        q = 2 * math.pi * m / L
        E.append(s.energy(I.flat_spiral(r, [q, 0, 0], [0, 0, 1], [1, 0, 0]))[0] / s.N)
        assert abs(E[-1] - (-J * (math.cos(q) + 1) - D * math.sin(q))) < 1e-12
    q_star = math.atan(D / J)
    assert abs(2 * math.pi * int(np.argmin(E)) / L - q_star) < 2 * math.pi / L


# ----------------------------------------------------------------------------
# Exact identities of a Hamiltonian quadratic in n (Eq. 1 without quadruplets)
# ----------------------------------------------------------------------------
def _systems():
    out = []
    c = I.cfg_square_32()
    out.append(("square", dict(c["geometry"], n_cells=[7, 6, 1]), c["hamiltonian"]))
    c = I.cfg_sc_128(4)
    out.append(("sc", c["geometry"], dict(c["hamiltonian"], B=[0.3, -0.2, 0.5])))
    out.append(("hex_dipole", I.hexagonal(6, 5, mu_s=3.0),
                dict(J=[1.0], dmi_kind="interfacial", D=[0.3], K=[0.2], Khat=[[0, 0, 1]], dipole="direct",
                     B=[0.1, 0, 0.2])))
    out.append(("two_basis", dict(bravais=[[1, 0, 0], [0.3, 1.1, 0], [0.1, 0.2, 0.9]],
                                  basis=[[0, 0, 0], [0.4, 0.3, 0.25]], n_cells=[3, 4, 2],
                                  periodic=[0, 0, 0], lattice_constant=1.7, mu_s=[2.0, 0.8]),
                dict(J=[1.0, -0.3], dmi_kind="bulk", D=[0.2, 0.05], K=[0.1, 0.3], Khat=[[0, 0, 1], [1, 1, 0]],
                     dipole="direct", B=[0.3, 0.1, -0.4],
                     pairs=[(0, 1, (1, 1, 0), 0.4, (0.1, -0.2, 0.3))])))
    return out


@pytest.mark.parametrize("name,g,h", _systems(), ids=[x[0] for x in _systems()])
def test_gradient_is_exact_finite_difference(name, g, h):
    s = oracle.System(g, h)
    n = I.random_spins(s.N, 17)
    B = s.field(n)
    rng = np.random.default_rng(5)
    hstep = 1e-3
    E0 = abs(s.energy(n)[0]) + 1
    for _ in range(12):
        i, k = int(rng.integers(s.N)), int(rng.integers(3))
        p, m = n.copy(), n.copy()
        p[i, k] += hstep
        m[i, k] -= hstep
        fd = (s.energy(p)[0] - s.energy(m)[0]) / (2 * hstep)
        # H is a polynomial of degree 2 in R^3N: central differences are exact
        assert abs(fd + B[i, k]) < 1e-12 * E0 / hstep


@pytest.mark.parametrize("name,g,h", _systems(), ids=[x[0] for x in _systems()])
def test_energy_equals_quadratic_form(name, g, h):
    s = oracle.System(g, h)
    n = I.random_spins(s.N, 21)
    B = s.field(n)
    mu = np.asarray(g["mu_s"], dtype=float)[np.arange(s.N) % s.n_basis]
    Bz = mu[:, None] * oracle.MU_B * np.asarray(h.get("B", [0, 0, 0]), dtype=float)[None, :]
    quad = B - Bz
    E_quad = -np.sum(n * (Bz + 0.5 * quad))
    e = s.energy(n)
    assert abs(e[0] - E_quad) < 1e-12 * (abs(e[0]) + 1)
    assert abs(e[0] - e[1:].sum()) < 1e-12 * (abs(e[0]) + 1)


def test_pair_swap_symmetry():
    # relabelling i <-> j of an explicit pair (d -> -d, D -> -D) leaves E unchanged
    g = dict(bravais=[[1, 0, 0], [0, 1, 0], [0, 0, 1]], basis=[[0, 0, 0], [0.5, 0.5, 0]],
             n_cells=[4, 3, 1], periodic=[1, 0, 0], lattice_constant=1.0, mu_s=[1.0, 2.0])
    p1 = dict(pairs=[(0, 1, (1, 0, 0), 0.7, (0.1, 0.2, -0.3))])
    p2 = dict(pairs=[(1, 0, (-1, 0, 0), 0.7, (-0.1, -0.2, 0.3))])
    n = I.random_spins(24, 3)
    a = oracle.System(g, p1).energy(n)
    b = oracle.System(g, p2).energy(n)
    assert np.allclose(a, b, rtol=0, atol=1e-13)


# ----------------------------------------------------------------------------
# Dipole-dipole term (Sec. "Dipolar interactions")
# ----------------------------------------------------------------------------
def test_dipole_two_spins_by_hand():
    # head-to-tail along the bond: E = -2 C mu^2 / r^3; side by side: +C mu^2 / r^3
    r, mu = 2.5, 1.7
    g = dict(bravais=[[r, 0, 0], [0, 1, 0], [0, 0, 1]], basis=[[0, 0, 0]], n_cells=[2, 1, 1],
             periodic=[0, 0, 0], lattice_constant=1.0, mu_s=[mu])
    s = oracle.System(g, dict(dipole="direct"))
    C = oracle.C_DIP
    assert abs(s.energy(np.array([[1.0, 0, 0], [1.0, 0, 0]]))[5] - (-2 * C * mu * mu / r ** 3)) < 1e-15
    assert abs(s.energy(np.array([[0, 0, 1.0], [0, 0, 1.0]]))[5] - (C * mu * mu / r ** 3)) < 1e-15
    # the head-to-tail pair is the lower-energy arrangement
    sf = oracle.System(g, dict(dipole="fft"))
    assert abs(sf.energy(np.array([[1.0, 0, 0], [1.0, 0, 0]]))[5] - (-2 * C * mu * mu / r ** 3)) < 1e-15


@pytest.mark.parametrize("case", ["hex_2d", "two_basis_3d", "square_ragged"])
def test_dipole_fft_equals_direct_sum(case):
    # the paper's own check: FFT convolution vs direct summation for random
    # states with spatially non-symmetric basis cells
    if case == "hex_2d":
        g = I.hexagonal(12, 10, mu_s=3.0)
    elif case == "two_basis_3d":
        g = dict(bravais=[[1, 0, 0], [0.5, math.sqrt(3) / 2, 0], [0, 0, 1]], basis=[[0, 0, 0], [0.3, 0.1, 0.2]],
                 n_cells=[6, 5, 3], periodic=[0, 0, 0], lattice_constant=1.3, mu_s=[2.0, 0.7])
    else:
        g = I.square(9, 7, mu_s=2.0)
    s = oracle.System(g, dict(dipole="direct"))
    n = I.random_spins(s.N, 3)
    Bd = s.dipole_field(n, "direct")
    Bf = s.dipole_field(n, "fft")
    assert np.abs(Bd - Bf).max() < 1e-12 * np.abs(Bd).max()
    sf = oracle.System(g, dict(dipole="fft"))
    assert abs(s.energy(n)[5] - sf.energy(n)[5]) < 1e-12 * abs(s.energy(n)[5])


def test_dipole_monolayer_converges_to_lattice_sum():
    # Homogeneously magnetised square monolayer: at the centre of an open
    # (2R+1)^2 lattice B_z = -C mu^2 S_R with S_R -> S = sum' 1/|r|^3 =
    # 4 zeta(3/2) beta(3/2) and S - S_R = 4 sqrt(2) / (R + 1/2) + O(R^-3).
    beta = 4 ** -1.5 * (zeta(1.5, 0.25) - zeta(1.5, 0.75))
    S = 4 * zeta(1.5) * beta
    assert abs(S - 9.0336216831) < 1e-9
    prev = None
    for R in (8, 16, 32):
        L = 2 * R + 1
        s = oracle.System(I.square(L, L, mu_s=1.0), dict(dipole="fft"))
        B = s.dipole_field(I.ferromagnet(s.N), "fft")
        c = R + L * R
        val = -B[c, 2] / oracle.C_DIP
        assert abs(B[c, 0]) < 1e-12 and abs(B[c, 1]) < 1e-12
        assert abs(val + 4 * math.sqrt(2) / (R + 0.5) - S) < 0.2 / R ** 2
        if prev is not None:
            assert abs(S - val) < 0.55 * abs(S - prev)  # error ~ 1/R
        prev = val


# ----------------------------------------------------------------------------
# LLG invariants
# ----------------------------------------------------------------------------
def test_llg_unit_length_and_damped_energy_decrease():
    c = I.cfg_square_32()
    g = dict(c["geometry"], n_cells=[10, 9, 1])
    s = oracle.System(g, c["hamiltonian"])
    n = I.random_spins(s.N, 0)
    E = [s.energy(n)[0]]
    for _ in range(20):
        n = s.llg(n, 10, solver="depondt", dt=2e-3, alpha=0.3)
        E.append(s.energy(n)[0])
        assert np.abs(np.linalg.norm(n, axis=1) - 1).max() < 1e-14
    assert all(b < a for a, b in zip(E, E[1:]))
    n2 = I.random_spins(s.N, 0)
    for _ in range(20):
        n2 = s.llg(n2, 10, solver="heun", dt=2e-3, alpha=0.3)
        assert np.abs(np.linalg.norm(n2, axis=1) - 1).max() < 1e-14


@pytest.mark.parametrize("solver", ["depondt", "heun"])
def test_llg_energy_drift_second_order_at_zero_damping(solver):
    c = I.cfg_square_32()
    g = dict(c["geometry"], n_cells=[8, 8, 1])
    s = oracle.System(g, c["hamiltonian"])
    n0 = I.random_spins(s.N, 4)
    E0 = s.energy(n0)[0]
    # at alpha = 0 the energy is conserved by the flow; the integrators'
    # drift (max over the run) must fall at least like dt^2 (Depondt's is
    # observed to fall like dt^3)
    drift = []
    for dt in (0.005, 0.0025):
        n, mx = n0.copy(), 0.0
        for _ in range(int(round(0.5 / dt / 10))):
            n = s.llg(n, 10, solver=solver, dt=dt, alpha=0.0)
            mx = max(mx, abs(s.energy(n)[0] - E0))
        drift.append(mx)
    assert drift[0] / drift[1] > 3.5
    assert drift[0] < 1e-3


@pytest.mark.parametrize("solver", ["heun", "depondt"])
def test_langevin_macrospin_equilibrium(solver):
    # independent spins in a field: <n_z> = coth(x) - 1/x, x = mu B / (kB T)
    mu, B, x = 1.0, 1.0, 1.0
    T = mu * oracle.MU_B * B / (oracle.K_B * x)
    s = oracle.System(I.square(40, 25, mu_s=mu), dict(B=[0, 0, B]))
    n = I.random_spins(s.N, 11)
    dt, alpha = 0.05, 0.5
    n = s.llg(n, 400, solver=solver, dt=dt, alpha=alpha, T=T, seed=7)
    acc = []
    for k in range(60):
        n = s.llg(n, 50, solver=solver, dt=dt, alpha=alpha, T=T, seed=7, step0=400 + 50 * k)
        acc.append(n[:, 2].mean())
    L = 1 / math.tanh(x) - 1 / x
    assert abs(np.mean(acc) - L) < 0.012


def test_thermal_run_is_reproducible_and_seeded():
    s = oracle.System(I.square(5, 4, mu_s=2.0), dict(J=[1.0], B=[0, 0, 1.0]))
    n0 = I.random_spins(s.N, 1)
    a = s.llg(n0, 20, solver="heun", dt=1e-3, alpha=0.1, T=10.0, seed=9)
    b = s.llg(s.llg(n0, 7, solver="heun", dt=1e-3, alpha=0.1, T=10.0, seed=9), 13, solver="heun", dt=1e-3,
              alpha=0.1, T=10.0, seed=9, step0=7)
    assert np.array_equal(a, b)  # counter-based: resuming at step0 is bit-exact
    c = s.llg(n0, 20, solver="heun", dt=1e-3, alpha=0.1, T=10.0, seed=10)
    assert np.abs(a - c).max() > 1e-4


# ----------------------------------------------------------------------------
# Velocity projection minimiser (Appendix D)
# ----------------------------------------------------------------------------
def test_vp_relaxes_to_ferromagnet_closed_form():
    c = I.cfg_square_32()
    g = dict(c["geometry"], n_cells=[16, 16, 1], periodic=[1, 1, 0])
    s = oracle.System(g, c["hamiltonian"])
    N = s.N
    E_fm = -2 * N * 1.0 - N * 0.1 - N * 2.0 * oracle.MU_B * 1.0
    n, v, it, mt = s.minimise(I.perturbed(I.ferromagnet(N), 0.1, 3), dt=0.1, tol=1e-10, max_iter=20000)
    assert mt < 1e-10 and it < 20000
    assert abs(s.energy(n)[0] - E_fm) < 1e-10 * abs(E_fm)


def test_vp_relaxes_perturbed_spiral_back_to_its_energy():
    # J + DMI, no anisotropy or field: every commensurate flat spiral is stationary
    L = 40
    g = dict(I.square(L, 4, periodic=(True, True)))
    J, D = 1.0, 0.3
    s = oracle.System(g, dict(J=[J], dmi_kind="interfacial", D=[D]))
    m = 2  # q = 2 pi m / L closest to atan(D/J)
    q = 2 * math.pi * m / L
    n0 = I.flat_spiral(I.site_positions(g), [q, 0, 0], [0, 0, 1], [1, 0, 0])
    n, v, it, mt = s.minimise(I.perturbed(n0, 0.02, 8), dt=0.1, tol=1e-9, max_iter=50000)
    assert mt < 1e-9
    E_exp = s.N * (-J * (math.cos(q) + 1) - D * math.sin(q))
    assert abs(s.energy(n)[0] - E_exp) < 1e-9 * abs(E_exp)


# ----------------------------------------------------------------------------
# GNEB (Sec. GNEB, Appendix F)
# ----------------------------------------------------------------------------
def test_gneb_climbing_image_hits_stoner_wohlfarth_barrier():
    # single uniaxial spin in a field along the axis: E = -K cos^2 - mu B cos,
    # saddle at cos = -h, barrier from the metastable state K (1 - h)^2
    mu, K, B = 2.0, 1.0, 3.0
    s = oracle.System(I.square(1, 1, mu_s=mu), dict(B=[0, 0, B], K=[K], Khat=[[0, 0, 1]]))
    h = mu * oracle.MU_B * B / (2 * K)
    chain = I.slerp_chain(np.array([[0, 0, -1.0]]), np.array([[0, 0, 1.0]]), 9)
    ch, v, E, mf, it = s.gneb(chain, n_iter=20000, tol=1e-12, dt=0.5, climbing=True)
    assert mf < 1e-12
    assert abs(E.max() - E[0] - K * (1 - h) ** 2) < 1e-12
    ci = int(np.argmax(E))
    assert abs(ch[ci, 0, 2] + h) < 1e-10  # at the saddle cos(theta) = -h
    # without climbing the highest image only brackets the barrier
    ch2, _, E2, mf2, _ = s.gneb(chain, n_iter=20000, tol=1e-12, dt=0.5, climbing=False)
    assert E2.max() - E2[0] <= K * (1 - h) ** 2 + 1e-12


def test_gneb_images_equidistant_without_climbing():
    mu, K, B = 2.0, 1.0, 3.0
    s = oracle.System(I.square(1, 1, mu_s=mu), dict(B=[0, 0, B], K=[K], Khat=[[0, 0, 1]]))
    chain = I.slerp_chain(np.array([[0.3, 0, -1.0]]) / np.linalg.norm([0.3, 0, -1]), np.array([[0, 0, 1.0]]), 7)
    ch, v, E, mf, it = s.gneb(chain, n_iter=40000, tol=1e-11, dt=0.3, climbing=False, k_spring=2.0)
    _, _, l, _ = s.gneb_forces(ch, climbing=False, k_spring=2.0)
    assert np.abs(l - l.mean()).max() < 1e-9


def _tangent_hessian(s, n, h=1e-5):
    # 2x2 Hessian of E on the sphere at n by finite differences of the
    # projected gradient along an orthonormal tangent basis
    n = n / np.linalg.norm(n)
    t1 = np.cross(n, [0.3, 0.7, 0.1])
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(n, t1)
    Hm = np.zeros((2, 2))
    for a, ta in enumerate((t1, t2)):
        gp = -s.field(((n + h * ta) / np.linalg.norm(n + h * ta))[None])[0]
        gm = -s.field(((n - h * ta) / np.linalg.norm(n - h * ta))[None])[0]
        for b, tb in enumerate((t1, t2)):
            Hm[a, b] = (np.dot(gp, tb) - np.dot(gm, tb)) / (2 * h)
    # Riemannian correction -(n.grad) I for the embedded sphere
    g0 = -s.field(n[None])[0]
    return 0.5 * (Hm + Hm.T) - np.dot(n, g0) * np.eye(2)


def test_gneb_gaussian_landscape_saddle():
    # Appendix G landscape (Fig. 7): the climbing image converges onto a
    # first-order saddle point found independently by Newton iteration.
    G = np.loadtxt(os.path.join(GOLDEN, "gaussian_landscape.txt"))
    assert G.shape == (7, 5)
    s = oracle.System(I.square(1, 1, mu_s=1.0), dict(gauss=G.tolist()))
    a = np.array([[-0.1906, -0.0058, -0.9816]])
    b = np.array([[0.9859, -0.1633, -0.0367]])
    a, _, _, ta = s.minimise(a / np.linalg.norm(a), dt=0.05, tol=1e-13, max_iter=100000)
    b, _, _, tb = s.minimise(b / np.linalg.norm(b), dt=0.05, tol=1e-13, max_iter=100000)
    assert ta < 1e-13 and tb < 1e-13
    for m in (a, b):
        assert np.all(np.linalg.eigvalsh(_tangent_hessian(s, m[0])) > 0)  # minima
    chain = I.slerp_chain(a, b, 15)
    ch, v, E, mf, it = s.gneb(chain, n_iter=200000, tol=1e-11, dt=0.02, climbing=True, k_spring=0.5)
    assert mf < 1e-11
    ci = int(np.argmax(E))
    x = ch[ci, 0]
    ev = np.linalg.eigvalsh(_tangent_hessian(s, x))
    assert ev[0] < 0 < ev[1]  # first-order saddle
    # Newton on the projected gradient from a perturbed start lands on the same point
    y = x + np.array([2e-3, -1e-3, 1.5e-3])
    y /= np.linalg.norm(y)
    for _ in range(30):
        t1 = np.cross(y, [0.3, 0.7, 0.1]); t1 /= np.linalg.norm(t1)
        t2 = np.cross(y, t1)
        g = -s.field(y[None])[0]
        gt = np.array([np.dot(g, t1), np.dot(g, t2)])
        step = np.linalg.solve(_tangent_hessian(s, y, 1e-6), -gt)
        y = y + step[0] * t1 + step[1] * t2
        y /= np.linalg.norm(y)
    assert np.linalg.norm(y - x) < 1e-8
    assert abs(s.energy(y[None])[0] - E[ci]) < 1e-10


# ----------------------------------------------------------------------------
# Topological charge (Appendix A)
# ----------------------------------------------------------------------------
def test_topological_charge_octant_triangle():
    # one spherical triangle spanned by x, y, z is an octant: A = 4 pi / 8
    s = oracle.System(I.hexagonal(2, 2), dict())
    n = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0], [0, 1.0, 0]])
    assert abs(s.topological_charge(n) - 1 / 8) < 1e-15


def test_topological_charge_of_skyrmion_and_ferromagnet():
    L = 32
    g = I.hexagonal(L, L, periodic=(True, True))
    s = oracle.System(g, dict())
    r = I.site_positions(g)
    centre = r.mean(axis=0)
    q = s.topological_charge(I.neel_skyrmion(r, centre, 8.0))
    assert abs(q + 1) < 1e-9
    assert abs(s.topological_charge(I.ferromagnet(s.N))) < 1e-12


# ----------------------------------------------------------------------------
# SIB (Appendix C) and RK4
# ----------------------------------------------------------------------------
def test_sib_is_second_order_and_norm_preserving():
    e = [_larmor_error("sib", dt, t_end=40.0)[0] for dt in (0.02, 0.01)]
    assert 3.8 < e[0] / e[1] < 4.2
    # the implicit midpoint step is a Cayley rotation: |n| = 1 without renormalisation
    c = I.cfg_square_32()
    s = oracle.System(dict(c["geometry"], n_cells=[9, 7, 1]), c["hamiltonian"])
    n = s.llg(I.random_spins(s.N, 2), 500, solver="sib", dt=2e-3, alpha=0.2, T=20.0, seed=3)
    assert np.abs(np.linalg.norm(n, axis=1) - 1).max() < 1e-13


def test_sib_step_solves_the_two_implicit_midpoint_equations():
    # Appendix C for one spin in a constant field, solved here with a library
    # linear solver instead of Cramer's rule:
    #   predictor  x_p = n + dt (n + x_p)/2 x A(n)
    #   corrector  x   = n + dt (n + x)/2 x A((n + x_p)/2)
    # i.e. (I + dt/2 [A]x) y = n + dt/2 n x A with [A]x y = A x y.
    mu, alpha, dt = 1.5, 0.2, 0.05
    s = oracle.System(I.square(1, 1, mu_s=mu), dict(B=[0.3, -0.4, 1.1]))
    n0 = np.array([0.6, 0.0, 0.8])
    B = s.field(n0[None])[0]  # Zeeman only: the same for any spin direction
    gp = -oracle.GAMMA / ((1 + alpha ** 2) * mu * oracle.MU_B)

    def A(m):
        return gp * (B + alpha * np.cross(m, B))

    def midpoint_solve(n, a):
        K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
        return np.linalg.solve(np.eye(3) + 0.5 * dt * K, n + 0.5 * dt * np.cross(n, a))

    xp = midpoint_solve(n0, A(n0))
    x = midpoint_solve(n0, A(0.5 * (n0 + xp)))
    n1 = s.llg(n0[None], 1, solver="sib", dt=dt, alpha=alpha)[0]
    assert np.abs(n1 - x).max() < 1e-15


def test_rk4_is_fourth_order():
    e = [_larmor_error("rk4", dt, t_end=40.0)[0] for dt in (0.04, 0.02)]
    assert 14.0 < e[0] / e[1] < 18.0
    assert e[1] < 1e-10


# ---------------------------------------------------------------- warm-start network
from oracle import unet as U  # noqa: E402


def _brute_conv(x, W, b):
    B, H, Wd, Ci = x.shape
    Co = W.shape[0]
    out = np.zeros((B, H, Wd, Co))
    for bb in range(B):
        for y in range(H):
            for xx in range(Wd):
                for o in range(Co):
                    s = b[o]
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            t = 3 * (dy + 1) + (dx + 1)
                            for i in range(Ci):
                                s += W[o, t, i] * x[bb, (y + dy) % H, (xx + dx) % Wd, i]
                    out[bb, y, xx, o] = s
    return out


def test_unet_conv_matches_brute_force():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 4, 2))
    W = rng.standard_normal((3, 9, 2))
    b = rng.standard_normal(3)
    assert np.allclose(U.conv3x3(x, W, b), _brute_conv(x, W, b), rtol=0, atol=1e-12)


def _fd_grad(f, arr, idx, h=1e-6):
    old = arr[idx]
    arr[idx] = old + h
    fp = f()
    arr[idx] = old - h
    fm = f()
    arr[idx] = old
    return (fp - fm) / (2 * h)


def test_unet_conv_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 4, 4, 3))
    W = rng.standard_normal((2, 9, 3))
    b = rng.standard_normal(2)
    R = rng.standard_normal((2, 4, 4, 2))
    f = lambda: float(np.sum(R * U.conv3x3(x, W, b)))  # noqa: E731
    dx, dW, db = U.conv3x3_backward(x, W, R)
    for arr, g in ((x, dx), (W, dW), (b, db)):
        for idx in np.ndindex(arr.shape):
            assert abs(_fd_grad(f, arr, idx) - g[idx]) < 1e-7


def test_unet_pool_upsample_backward_match_finite_differences():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((1, 4, 6, 2))
    for fwd, bwd in ((U.pool, U.pool_backward), (U.upsample, U.upsample_backward)):
        R = rng.standard_normal(fwd(x).shape)
        f = lambda: float(np.sum(R * fwd(x)))  # noqa: E731
        g = bwd(R)
        for idx in np.ndindex(x.shape):
            assert abs(_fd_grad(f, x, idx) - g[idx]) < 1e-8
    # mean pooling of a constant is that constant; upsampling then pooling is the identity
    assert np.allclose(U.pool(np.full((1, 4, 4, 1), 2.5)), 2.5)
    assert np.allclose(U.pool(U.upsample(x)), x)


def _small_net(seed, widths=(4, 4, 6, 8), in_ch=8, L=8, B=2):
    rng = np.random.default_rng(seed)
    arch = U.architecture(widths, in_ch)
    flat = []
    for _, ci, co, _ in arch:
        flat += [rng.standard_normal(co * 9 * ci) * np.sqrt(2.0 / (9 * ci)), rng.standard_normal(co) * 0.1]
    flat += [rng.standard_normal(3 * widths[0]), rng.standard_normal(3) * 0.1]
    params = U.unpack(np.concatenate(flat), widths, in_ch)
    spins = rng.standard_normal((B, L * L, 3))
    spins /= np.linalg.norm(spins, axis=-1, keepdims=True)
    feats = rng.uniform(0, 1, (B, 4))
    x = U.network_input(spins, feats, L, in_ch)
    t = rng.standard_normal((B, L, L, 3))
    t /= np.linalg.norm(t, axis=-1, keepdims=True)
    return params, x, t


def test_unet_network_gradient_matches_finite_differences():
    params, x, t = _small_net(4)
    loss, grads = U.loss_and_gradient(params, x, t)
    _, _, y = U.forward(params, x)
    assert abs(loss - U.loss_of(y, t)) < 1e-14
    rng = np.random.default_rng(5)
    f = lambda: U.loss_of(U.forward(params, x)[2], t)  # noqa: E731
    for name in list(params):
        for k in (0, 1):
            arr, g = params[name][k], grads[name][k]
            for _ in range(3):
                idx = tuple(int(rng.integers(0, s)) for s in arr.shape)
                fd = _fd_grad(f, arr, idx, h=1e-5)
                assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(g[idx])) + 1e-9, (name, k, idx, fd, g[idx])


def test_unet_loss_special_cases():
    params, x, t = _small_net(6)
    _, _, y = U.forward(params, x)
    m = y / np.linalg.norm(y, axis=-1, keepdims=True)
    assert abs(U.loss_of(y, m)) < 1e-14          # prediction equal to the target
    assert abs(U.loss_of(y, -m) - 2.0) < 1e-14   # opposite target
    assert abs(U.loss_of(3.7 * y, t) - U.loss_of(y, t)) < 1e-14  # only the direction counts


def test_unet_adam_first_step_closed_form():
    # from zero moments the bias-corrected first step is lr * g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    p = np.array([1.0, 1.0, 1.0, 1.0])
    p1, m1, v1 = U.adam_step(p, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    assert np.allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def test_unet_layout_matches_the_input_recipe():
    from paper_1901_11350_gb300 import inputs as I
    arch = U.architecture()
    assert [(ci, co) for _, ci, co, _ in arch] == I.UNET_LAYERS
    flat = I.unet_init(7)
    assert flat.size == I.unet_n_params()
    params = U.unpack(flat)
    assert np.array_equal(U.pack(params), flat.astype(np.float64))
    assert np.all(params["e1a"][0][:, :, I.UNET_REAL_INPUTS:] == 0)


# ----------------------------------------------------------------------------
# GNEB refinements (Sec. GNEB): falling image, energy-weighted springs,
# path interpolation
# ----------------------------------------------------------------------------
WELL_SIGMA = 0.15
THREE_WELLS = [[-1.0, WELL_SIGMA, 1.0, 0.0, 0.0], [-1.0, WELL_SIGMA, 0.0, 1.0, 0.0],
               [-1.0, WELL_SIGMA, -1.0, 0.0, 0.0]]


def _equator_chain(M, phi0=0.0, phi1=np.pi):
    phi = np.linspace(phi0, phi1, M)
    return np.stack([np.cos(phi), np.sin(phi), np.zeros(M)], axis=1)[:, None, :], phi


def _three_well_system():
    return oracle.System(I.square(1, 1, mu_s=1.0), dict(gauss=THREE_WELLS))


def test_gneb_falling_image_reaches_the_minimum_fixed_by_symmetry():
    # wells at x, y and -x: on the path x -> y -> -x the mirror symmetry
    # x -> -x fixes the intermediate minimum at y exactly; the climbing
    # images converge onto two first-order saddles that are mirror images.
    s = _three_well_system()
    # an asymmetric start: image 4 at 73 degrees, so every image has to move
    phi = np.pi * (np.arange(9) / 8.0) ** 1.3
    ch0 = np.stack([np.cos(phi), np.sin(phi), np.zeros(9)], axis=1)[:, None, :]
    assert abs(phi[4] - np.pi / 2) > 0.25
    a, _, _, ta = s.minimise(ch0[0], dt=0.05, tol=1e-13, max_iter=100000)
    b, _, _, tb = s.minimise(ch0[-1], dt=0.05, tol=1e-13, max_iter=100000)
    assert ta < 1e-13 and tb < 1e-13
    ch0[0], ch0[-1] = a, b
    types = ["normal", "normal", "climbing", "normal", "falling", "normal", "climbing", "normal", "normal"]
    ch, v, E, mf, it = s.gneb(ch0, n_iter=300000, tol=1e-11, dt=0.02, k_spring=0.5, image_types=types)
    assert mf < 1e-11
    # the well is quartic at its centre (force ~ offset^3), so the position is
    # fixed to about the cube root of the force tolerance and the energy to
    # its fourth power
    assert np.linalg.norm(ch[4, 0] - np.array([0.0, 1.0, 0.0])) < 1e-3
    e_y = -1.0 - 2.0 * np.exp(-1.0 / (2 * WELL_SIGMA ** 2))
    assert abs(E[4] - e_y) < 1e-12
    # a minimum: the energy rises for every small tilt (the well is quartic at
    # its centre, so its Hessian vanishes there)
    for ang in np.linspace(0, 2 * np.pi, 12, endpoint=False):
        d = np.array([np.cos(ang), 0.0, np.sin(ang)]) * 0.05
        y = (ch[4, 0] + d) / np.linalg.norm(ch[4, 0] + d)
        assert s.energy(y[None])[0] > E[4]
    for k in (2, 6):
        ev = np.linalg.eigvalsh(_tangent_hessian(s, ch[k, 0]))
        assert ev[0] < 0 < ev[1]
    mirror = ch[2, 0] * np.array([-1.0, 1.0, 1.0])
    assert np.linalg.norm(mirror - ch[6, 0]) < 1e-8
    assert abs(E[2] - E[6]) < 1e-12
    assert E[2] > E[4] and E[6] > E[4]


def test_gneb_path_slopes_and_coordinates_in_closed_form():
    # a chain on the equator of the three-well landscape: the reaction
    # coordinate is the azimuth, and dE/dr is the derivative of
    # E(phi) = sum_k a exp(-(1 - cos(phi - phi_k))^2 / (2 s^2)).
    s = _three_well_system()
    ch, phi = _equator_chain(13, 0.1, 2.9)
    P = s.gneb_path(ch, n_interp=8)
    assert np.allclose(P["r"], phi - phi[0], rtol=0, atol=1e-13)
    centres = [0.0, np.pi / 2, np.pi]
    s2 = WELL_SIGMA ** 2
    E = lambda p: sum(-np.exp(-(1 - np.cos(p - c)) ** 2 / (2 * s2)) for c in centres)  # noqa: E731
    dE = lambda p: sum(-np.exp(-(1 - np.cos(p - c)) ** 2 / (2 * s2)) * (-(1 - np.cos(p - c)) * np.sin(p - c) / s2)
                       for c in centres)  # noqa: E731
    assert np.allclose(P["E"], E(phi), rtol=0, atol=1e-14)
    assert np.allclose(P["slope"], dE(phi), rtol=0, atol=1e-12)


def test_gneb_path_interpolation_is_the_cubic_hermite_spline():
    from scipy.interpolate import CubicHermiteSpline
    s = _three_well_system()
    ch, _ = _equator_chain(7, 0.2, 2.6)
    ch = ch + 0.05 * np.random.default_rng(2).standard_normal(ch.shape)  # off the great circle
    ch /= np.linalg.norm(ch, axis=-1, keepdims=True)
    P = s.gneb_path(ch, n_interp=5)
    spl = CubicHermiteSpline(P["r"], P["E"], P["slope"])
    assert np.allclose(P["E_interp"], spl(P["r_interp"]), rtol=0, atol=1e-13)
    # the reaction coordinate is the running sum of geodesic angles
    ang = [np.arctan2(np.linalg.norm(np.cross(ch[k, 0], ch[k + 1, 0])), np.dot(ch[k, 0], ch[k + 1, 0]))
           for k in range(len(ch) - 1)]
    assert np.allclose(P["r"][1:], np.cumsum(ang), rtol=0, atol=1e-14)


def test_energy_weighted_segment_length_against_quadrature():
    from scipy.integrate import quad
    from scipy.interpolate import CubicHermiteSpline
    rng = np.random.default_rng(3)
    for _ in range(50):
        h = rng.uniform(0.05, 2.0)
        Ea, Eb = rng.uniform(-5, 5, 2)
        da, db = rng.uniform(-30, 30, 2)
        w = rng.uniform(0, 0.95)
        d = CubicHermiteSpline([0, h], [Ea, Eb], [da, db]).derivative()
        ref, _ = quad(lambda x: np.sqrt((1 - w) ** 2 + w ** 2 * d(x) ** 2), 0, h, epsabs=0, epsrel=1e-13, limit=500)
        assert abs(oracle.segment_length(Ea, Eb, da, db, h, w) - ref) <= 1e-12 * ref
    assert oracle.segment_length(1.0, 2.0, 3.0, 4.0, 0.7, 0.0) == 0.7  # w = 0: the geodesic distance
    # a flat segment (no slope, equal energies) has length (1 - w) h
    assert abs(oracle.segment_length(1.0, 1.0, 0.0, 0.0, 0.8, 0.4) - 0.6 * 0.8) < 1e-15


def test_energy_weighted_springs_equalise_segment_lengths():
    # with w > 0 and no climbing image, the converged chain has equal
    # energy-weighted segment lengths, measured here by an independent
    # quadrature of the spline through the chain's path data
    from scipy.integrate import quad
    from scipy.interpolate import CubicHermiteSpline
    s = _three_well_system()
    ch0, _ = _equator_chain(9, 0.0, np.pi / 2)
    a, _, _, _ = s.minimise(ch0[0], dt=0.05, tol=1e-13, max_iter=100000)
    b, _, _, _ = s.minimise(ch0[-1], dt=0.05, tol=1e-13, max_iter=100000)
    ch0[0], ch0[-1] = a, b
    w = 0.6
    ch, v, E, mf, it = s.gneb(ch0, n_iter=400000, tol=1e-10, dt=0.02, k_spring=1.0, climbing=False, energy_weight=w)
    assert mf < 1e-10
    P = s.gneb_path(ch)
    L = []
    for k in range(len(ch) - 1):
        h = P["r"][k + 1] - P["r"][k]
        d = CubicHermiteSpline([0, h], [P["E"][k], P["E"][k + 1]], [P["slope"][k], P["slope"][k + 1]]).derivative()
        L.append(quad(lambda x: np.sqrt((1 - w) ** 2 + w ** 2 * d(x) ** 2), 0, h, epsabs=0, epsrel=1e-12)[0])
    L = np.array(L)
    assert np.max(np.abs(L - L.mean())) < 1e-8
    # and they differ from the geodesic spacing: images crowd where E changes
    dr = np.diff(P["r"])
    assert np.max(dr) / np.min(dr) > 1.2


# ----------------------------------------------------------------------------
# Metropolis Monte Carlo (Sec. Monte Carlo)
# ----------------------------------------------------------------------------
def _langevin(x):
    return 1.0 / np.tanh(x) - 1.0 / x


def _mc_run(s, R, T, thermal, samples, seed, start=None):
    x0 = np.tile(I.ferromagnet(s.N)[None], (R, 1, 1)) if start is None else start
    x, cone, _ = s.mc(x0, T, thermal, seed=seed, target_accept=0.5, sample=False)
    x, cone, st = s.mc(x, T, samples, seed=seed, sweep0=thermal, target_accept=0.0, sample=True, cone=cone)
    return x, cone, st


def test_mc_single_spin_in_a_field_is_langevin():
    # one moment in B along z: <n_z> = L(x), var(n_z) = 1 - 2 L(x)/x - L(x)^2,
    # x = mu B / (k_B T); E = -mu B n_z
    mu, Bz, T = 2.0, 1.0, 1.0
    s = oracle.System(I.square(1, 1, mu_s=mu), dict(B=[0, 0, Bz]))
    assert s.mc_colours() == 1
    R = 64
    _, _, st = _mc_run(s, R, [T] * R, 200, 3000, seed=11)
    muB = mu * oracle.MU_B * Bz
    x = muB / (oracle.K_B * T)
    nz = -st[:, 3].sum() / st[:, 5].sum() / muB
    nz2 = st[:, 4].sum() / st[:, 5].sum() / muB ** 2
    L = _langevin(x)
    assert abs(nz - L) < 5e-3
    assert abs((nz2 - nz ** 2) - (1 - 2 * L / x - L ** 2)) < 5e-3


def test_mc_single_spin_anisotropy_matches_quadrature():
    # E = -K n_z^2: <n_z^2> = int u^2 exp(K u^2/kT) du / int exp(K u^2/kT) du
    from scipy.integrate import quad
    K, T = 0.1, 0.8
    s = oracle.System(I.square(1, 1, mu_s=2.0), dict(K=[K], Khat=[[0, 0, 1]]))
    R = 64
    _, _, st = _mc_run(s, R, [T] * R, 200, 3000, seed=12)
    kap = K / (oracle.K_B * T)
    ref = quad(lambda u: u * u * np.exp(kap * u * u), -1, 1)[0] / quad(lambda u: np.exp(kap * u * u), -1, 1)[0]
    assert abs(-st[:, 3].sum() / st[:, 5].sum() / K - ref) < 5e-3


def test_mc_exchange_dimer_is_langevin_in_j_over_kt():
    # two spins coupled by J: the angle between them has density ~ exp(x cos g),
    # so <n1.n2> = L(J / kT) and <E> = -J L(J / kT)
    J, T = 0.2, 1.5
    s = oracle.System(I.square(2, 1, periodic=(False, False), mu_s=2.0), dict(J=[J]))
    assert s.mc_colours() == 2
    R = 64
    _, _, st = _mc_run(s, R, [T] * R, 200, 3000, seed=13)
    x = J / (oracle.K_B * T)
    assert abs(-st[:, 3].sum() / st[:, 5].sum() / J - _langevin(x)) < 6e-3


def test_mc_heisenberg_ring_energy_is_the_transfer_matrix_value():
    # classical Heisenberg ring of 5 spins: exp(K n.m) has the eigenvalues
    # 4 pi i_l(K) (multiplicity 2l + 1, i_l the modified spherical Bessel
    # function), so Z = (4 pi)^5 sum_l (2l+1) i_l(K)^5 and
    # <E> = -J d ln Z / dK, K = J / kT.  Five colours (c0 mod 5): the sweep
    # visits the ring sequentially
    from scipy.special import spherical_in
    J, T = 1.0, 7.5
    s = oracle.System(I.square(5, 1, periodic=(True, False), mu_s=2.0), dict(J=[J]))
    assert s.mc_colours() == 5
    K = J / (oracle.K_B * T)
    ls = np.arange(0, 40)
    i_l = spherical_in(ls, K)
    di_l = spherical_in(ls, K, derivative=True)
    dlnZ = np.sum((2 * ls + 1) * 5 * i_l ** 4 * di_l) / np.sum((2 * ls + 1) * i_l ** 5)
    R = 64
    _, _, st = _mc_run(s, R, [T] * R, 200, 3000, seed=14)
    E = st[:, 3].sum() / st[:, 5].sum()
    # the standard error is ~0.006 J; the open chain (-5 J L(K)) lies 0.13 J away
    assert abs(E - (-J * dlnZ)) < 0.03 * J, (E, -J * dlnZ)


@pytest.mark.parametrize("geom,ham,ncol", [
    (I.simple_cubic(6, 4, 4), dict(J=[1.0]), 2),          # (c0 + c1 + c2) mod 2
    (I.simple_cubic(9, 3, 3), dict(J=[1.0]), 3),          # odd periodic extents: mod 3 (product: 27)
    (I.simple_cubic(5, 5, 5), dict(J=[1.0]), 5),          # no product colouring
    (I.simple_cubic(4, 4, 4), dict(J=[1.0, -0.2]), 8),    # second shell: d0 + d1 + d2 = 0 bonds
    (I.hexagonal(9, 9, periodic=(True, True), mu_s=2.0), dict(J=[1.0]), 9),
    (I.simple_cubic(7, 7, 7), dict(J=[1.0, -0.2]), 0),    # neither colouring
])
def test_mc_colour_counts(geom, ham, ncol):
    assert oracle.System(geom, ham).mc_colours() == ncol


def test_mc_random_order_sweep_visits_every_spin_once():
    # the method's sweep visits each spin once per iteration in a random
    # order.  At a temperature where every trial is accepted, one sweep moves
    # every spin exactly once: each spin's move is the trial drawn for it, so
    # the coloured order (a different visiting order) gives the same state,
    # and a permutation that missed a spin would leave it where it was
    s = oracle.System(I.simple_cubic(6, 6, 4), dict(J=[1.0], B=[0, 0, 0.5]))
    x0 = I.random_spins(s.N, 8)[None]
    x, _, st = s.mc(x0, [1e12], 1, seed=3, target_accept=0.0, sample=False, cone=[0.7])
    y, _, _ = s.mc(x0, [1e12], 1, seed=3, target_accept=0.0, sample=False, cone=[0.7], order="coloured")
    assert st[0, 6] == st[0, 7] == s.N
    assert np.all(np.linalg.norm(x[0] - x0[0], axis=1) > 0)
    assert np.abs(x - y).max() < 1e-15
    # at a finite temperature the visiting order matters (the field of a
    # spin depends on which neighbours moved before it): the two orders give
    # different chains
    x, _, _ = s.mc(x0, [3.0], 3, seed=3, target_accept=0.0, sample=False, cone=[0.7])
    y, _, _ = s.mc(x0, [3.0], 3, seed=3, target_accept=0.0, sample=False, cone=[0.7], order="coloured")
    assert np.abs(x - y).max() > 1e-3


def test_mc_cone_adapts_to_the_target_acceptance_and_limits():
    # 8^3 spins: a sweep's acceptance fluctuates by ~2% (on 4^3 by ~6%, and the
    # multiplicative feedback turns that into a random walk of the cone)
    s = oracle.System(I.simple_cubic(8, 8, 8), dict(J=[1.0], B=[0, 0, 0.5]))
    assert s.mc_colours() == 2  # nearest neighbours only: (c0 + c1 + c2) mod 2
    x0 = np.tile(I.random_spins(s.N, 3)[None], (3, 1, 1))
    x, cone, st = s.mc(x0, [5.0, 12.0, 60.0], 400, seed=5, target_accept=0.4, sample=False)
    # acceptance of the next 100 sweeps at the adapted cone
    _, _, st = s.mc(x, [5.0, 12.0, 60.0], 100, seed=5, sweep0=400, target_accept=0.0, sample=False, cone=cone)
    assert np.all(np.abs(st[:2, 6] / st[:2, 7] - 0.4) < 0.03)
    # far above Tc even whole-sphere trials are accepted more often than the
    # target: the cone stops at pi
    assert cone[2] == np.pi and st[2, 6] / st[2, 7] > 0.4
    # T = 0 accepts only moves that lower the energy: E never increases
    E0 = s.energy(x0[0])[0]
    y, _, st0 = s.mc(x0[:1], [0.0], 30, seed=6, target_accept=0.0, sample=True, cone=[0.3])
    assert st0[0, 3] / st0[0, 5] < E0 and s.energy(y[0])[0] <= E0
    # at a very high temperature every trial is accepted
    _, _, sth = s.mc(x0[:1], [1e12], 5, seed=7, target_accept=0.0, sample=False, cone=[1.0])
    assert sth[0, 6] == sth[0, 7]


# ----------------------------------------------------------------------------
# Covariant Hessian and minimum mode following (Sec. MMF, manifold appendix)
# ----------------------------------------------------------------------------
def _retract(n, z, eps):
    y = n + eps * z
    return y / np.linalg.norm(y, axis=1, keepdims=True)


def test_hessian_matches_finite_differences_of_the_riemannian_gradient():
    # Hess f(x)[z] = P_x d/de grad f(R_x(e z)) at e = 0, with grad f = -P B;
    # central differences along a retraction, projected back onto T_x
    g = I.hexagonal(3, 3, periodic=(True, True), mu_s=2.0)
    h = dict(J=[1.0], dmi_kind="interfacial", D=[0.4], K=[0.3], Khat=[[0.2, 0.3, 0.93]], B=[0.1, -0.4, 1.3])
    s = oracle.System(g, h)
    n = I.random_spins(s.N, 17)
    H, T = s.hessian_dense(n)
    assert np.abs(H - H.T).max() < 1e-12  # symmetric in the tangent basis

    def rgrad(x):
        B = s.field(x)
        return -(B - np.sum(B * x, axis=1, keepdims=True) * x)

    eps = 1e-5
    for col in range(2 * s.N):
        z = np.zeros((s.N, 3))
        z[col // 2] = T[col // 2, :, col % 2]
        d = (rgrad(_retract(n, z, eps)) - rgrad(_retract(n, z, -eps))) / (2 * eps)
        d -= np.sum(d * n, axis=1, keepdims=True) * n
        fd = np.einsum("ikc,ik->ic", T, d).reshape(-1)
        assert np.abs(fd - H[:, col]).max() < 1e-7


def test_hessian_of_the_ferromagnet_is_the_magnon_spectrum():
    # n = z on an L x L periodic square lattice with B, K along z and exchange
    # J: eigenvalues mu B + 2K + J (4 - 2 cos qx - 2 cos qy), each twice
    L, mu, Bz, K, J = 4, 2.0, 0.7, 0.15, 1.0
    s = oracle.System(I.square(L, L, periodic=(True, True), mu_s=mu), dict(J=[J], K=[K], Khat=[[0, 0, 1]], B=[0, 0, Bz]))
    H, _ = s.hessian_dense(I.ferromagnet(s.N))
    q = 2 * np.pi * np.arange(L) / L
    lam = [mu * oracle.MU_B * Bz + 2 * K + J * (4 - 2 * np.cos(a) - 2 * np.cos(b)) for a in q for b in q]
    assert np.allclose(np.sort(np.linalg.eigvalsh(H)), np.sort(lam + lam), rtol=0, atol=1e-12)


def test_mmf_single_spin_climbs_onto_a_first_order_saddle():
    # one spin: Zeeman along z, easy axis along x.  Started near the minimum,
    # minimum mode following ends on a point with zero gradient and exactly
    # one negative Hessian eigenvalue, which Newton's method confirms.
    s = oracle.System(I.square(1, 1, mu_s=2.0), dict(B=[0, 0, 2.0], K=[0.3], Khat=[[1, 0, 0]]))
    x0, _, _, _ = s.minimise(np.array([[0.9, 0.1, 0.4]]) / np.linalg.norm([0.9, 0.1, 0.4]), dt=0.1, tol=1e-12,
                             max_iter=100000)
    assert np.all(np.linalg.eigvalsh(s.hessian_dense(x0)[0]) > 0)
    start = _retract(x0, np.array([[0.0, 0.3, -0.2]]), 0.3)
    x, v, F, lam = s.mmf(start, 3000, dt=0.1)
    assert np.abs(F).max() < 1e-9
    ev = np.linalg.eigvalsh(s.hessian_dense(x)[0])
    assert ev[0] < 0 < ev[1] and abs(lam - ev[0]) < 1e-12
    # Newton on the Riemannian gradient from a perturbed start: same point
    y = _retract(x, np.array([[1e-3, -2e-3, 1e-3]]), 1.0)
    for _ in range(40):
        Hy, Ty = s.hessian_dense(y)
        B = s.field(y)
        gr = -(B - np.sum(B * y, axis=1, keepdims=True) * y)
        step = np.linalg.solve(Hy, -np.einsum("ikc,ik->ic", Ty, gr).reshape(-1))
        y = _retract(y, np.einsum("ikc,ic->ik", Ty, step.reshape(-1, 2)), 1.0)
    assert np.linalg.norm(y - x) < 1e-8
    assert s.energy(x)[0] > s.energy(x0)[0]


# ----------------------------------------------------------------------------
# Harmonic transition-state theory (Sec. HTST, appendix on the manifold)
# ----------------------------------------------------------------------------
def _single_spin_stationary(mu_s, K, Bx, Bz):
    """Stationary points of one spin with easy axis z and field (Bx, 0, Bz) on
    the great circle n = (sin psi, 0, cos psi), found here independently of
    the oracle: (psi_min, psi_saddle) and the closed-form curvatures
    lambda_psi = E''(psi), lambda_y = 2 K n_z^2 + mu (Bx n_x + Bz n_z) (the
    second derivative along the geodesic towards y, which does not couple to
    psi by the mirror symmetry y -> -y)."""
    from scipy.optimize import brentq
    mu = mu_s * oracle.MU_B
    dE = lambda p: 2 * K * math.cos(p) * math.sin(p) - mu * (Bx * math.cos(p) - Bz * math.sin(p))  # noqa: E731
    d2E = lambda p: 2 * K * math.cos(2 * p) + mu * (Bx * math.sin(p) + Bz * math.cos(p))  # noqa: E731
    grid = np.linspace(-math.pi, math.pi, 4001)
    roots = [brentq(dE, a, b, xtol=1e-15) for a, b in zip(grid[:-1], grid[1:]) if dE(a) * dE(b) < 0]

    def lam(p):
        nx, nz = math.sin(p), math.cos(p)
        return d2E(p), 2 * K * nz * nz + mu * (Bx * nx + Bz * nz)

    mins = [p for p in roots if min(lam(p)) > 0]
    sads = [p for p in roots if lam(p)[0] < 0 < lam(p)[1]]
    # the metastable minimum (the higher of the two) and the saddle
    E = lambda p: -K * math.cos(p) ** 2 - mu * (Bx * math.sin(p) + Bz * math.cos(p))  # noqa: E731
    pm = max(mins, key=E)
    return pm, sads[0], lam(pm), lam(sads[0]), mu


def test_htst_single_spin_prefactor_is_the_precession_frequency():
    # one spin: the saddle's positive curvature cancels between Omega_0 and
    # v, and the prefactor is the precession frequency at the minimum over
    # 2 pi, gamma / (2 pi mu) sqrt(lambda_1^M lambda_2^M)
    mu_s, K, Bx, Bz = 2.0, 1.0, 1.5, 3.0
    pm, ps, lm, ls, mu = _single_spin_stationary(mu_s, K, Bx, Bz)
    s = oracle.System(I.square(1, 1, mu_s=mu_s), dict(B=[Bx, 0, Bz], K=[K], Khat=[[0, 0, 1]]))
    nm = np.array([[math.sin(pm), 0.0, math.cos(pm)]])
    ns = np.array([[math.sin(ps), 0.0, math.cos(ps)]])
    r = s.htst(nm, ns, zero_tol=1e-9)
    assert r["n_neg_min"] == 0 and r["n_neg_sad"] == 1 and r["n_zero_min"] == r["n_zero_sad"] == 0
    assert np.allclose(np.sort(r["eig_min"]), np.sort(lm), rtol=1e-12)
    assert np.allclose(np.sort(r["eig_sad"]), np.sort(ls), rtol=1e-12)
    assert abs(r["omega0"] - math.sqrt(lm[0] * lm[1] / ls[1])) <= 1e-12 * r["omega0"]
    assert abs(r["v"] - oracle.GAMMA / mu * math.sqrt(ls[1])) <= 1e-12 * r["v"]
    freq = oracle.GAMMA / (2 * math.pi * mu) * math.sqrt(lm[0] * lm[1])
    assert abs(r["prefactor"] - freq) <= 1e-12 * freq
    E = lambda p: -K * math.cos(p) ** 2 - mu * (Bx * math.sin(p) + Bz * math.cos(p))  # noqa: E731
    assert abs(r["dE"] - (E(ps) - E(pm))) <= 1e-12 * abs(E(pm))


def test_htst_axial_single_spin_has_a_zero_mode_at_the_saddle():
    # field along the easy axis: the saddle is a ring (cos theta = -h), one
    # zero mode there and none at the minimum; no positive saddle mode is
    # left, so the velocity factor of the primed sum vanishes
    mu_s, K, Bz = 2.0, 1.0, 3.0
    mu = mu_s * oracle.MU_B
    h = mu * Bz / (2 * K)
    s = oracle.System(I.square(1, 1, mu_s=mu_s), dict(B=[0, 0, Bz], K=[K], Khat=[[0, 0, 1]]))
    th = math.acos(-h)
    r = s.htst(np.array([[0.0, 0.0, -1.0]]), np.array([[math.sin(th), 0.0, math.cos(th)]]), zero_tol=1e-9)
    assert r["n_zero_sad"] == 1 and r["n_neg_sad"] == 1 and r["n_zero_min"] == 0
    assert abs(r["dE"] - K * (1 - h) ** 2) < 1e-12
    assert r["v"] == 0.0


def test_htst_velocity_equals_the_turned_mode_curvature():
    # the identity the GPU path computes v with: for W antisymmetric per
    # spin, sum over positive modes of a_i^2 / lambda_i = u . H u with
    # u_i = (gamma / mu_i) n_i x e_1,i (e_1 the unstable eigenvector), when
    # no zero modes are present.  Checked on a random "saddle" of a small
    # interacting system: the lowest eigenvalue is negative there.
    g = I.hexagonal(3, 3, periodic=(True, True), mu_s=[2.0])
    g["basis"] = [[0, 0, 0], [0.5, 0.3, 0]]
    g["mu_s"] = [2.0, 1.3]
    h = dict(J=[1.0, 0.3], dmi_kind="interfacial", D=[0.4], K=[0.3, 0.1], Khat=[[0, 0, 1], [1, 0, 0]], B=[0.1, 0, 0.9])
    s = oracle.System(g, h)
    n = I.random_spins(s.N, 4)
    r = s.htst(n, n, zero_tol=1e-9)
    lam, vec, T = s.hessian_eigen(n)
    assert lam[0] < 0
    e1 = np.einsum("ikc,ic->ik", T, vec[:, 0].reshape(-1, 2))
    mu = np.array([s.mu_s[i % 2] for i in range(s.N)]) * oracle.MU_B
    u = (oracle.GAMMA / mu)[:, None] * np.cross(n, e1)
    uHu = np.sum(u * s.hessian_apply(n, u))
    neg = lam < -1e-9
    # the primed sum leaves out every non-positive mode; u.Hu keeps the
    # other negative ones, whose share is subtracted here
    a = r["a"]
    extra = np.sum(a[neg][1:] ** 2 / lam[neg][1:])
    assert abs((uHu - extra) - r["v"] ** 2) <= 1e-10 * r["v"] ** 2


def test_htst_log_determinant_of_the_ferromagnet_is_the_magnon_product():
    # ferromagnet along z on a periodic square lattice (B, K along z): the
    # Hessian's eigenvalues are mu B + 2K + J (4 - 2 cos qx - 2 cos qy), each
    # twice, so log det = 2 sum_q log(...)
    L, mu_s, Bz, K, J = 6, 2.0, 0.7, 0.2, 1.0
    s = oracle.System(I.square(L, L, periodic=(True, True), mu_s=mu_s), dict(J=[J], K=[K], Khat=[[0, 0, 1]],
                                                                              B=[0, 0, Bz]))
    n = I.ferromagnet(s.N)
    q = 2 * math.pi * np.arange(L) / L
    w = mu_s * oracle.MU_B * Bz + 2 * K + J * (4 - 2 * np.cos(q)[:, None] - 2 * np.cos(q)[None, :])
    r = s.htst(n, n, zero_tol=1e-9)
    assert abs(r["log_det_min"] - 2 * np.sum(np.log(w))) <= 1e-12 * abs(r["log_det_min"])
    assert r["n_neg_min"] == 0 and r["n_zero_min"] == 0
