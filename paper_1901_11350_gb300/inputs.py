"""Seeded synthetic inputs and the workload definitions.

This module builds lattices, parameter sets and initial spin states; it
contains none of the method's arithmetic (no fields, energies or
integrators), so both the CUDA path and the CPU oracle may take their inputs
from it.

Geometry and Hamiltonian descriptions are plain dictionaries:

* geometry: ``bravais`` (rows = lattice vectors, units of the lattice
  constant), ``basis`` (fractional), ``n_cells``, ``periodic``,
  ``lattice_constant`` (Angstrom), ``mu_s`` (Bohr magnetons per basis atom);
* hamiltonian: ``B`` (T), ``K``/``Khat`` (meV, per basis atom), ``J`` (meV per
  shell), ``dmi_kind`` + ``D`` (meV per shell), ``dipole``, ``pairs``.

Random initial spins are uniform on the sphere: cos(theta) ~ U(-1, 1),
phi ~ U(0, 2 pi), drawn from numpy's PCG64 generator seeded with the
workload's seed.
"""
import math

import numpy as np

SQRT3_2 = math.sqrt(3.0) / 2.0


# ---------------------------------------------------------------- lattices
def square(n0, n1, periodic=(False, False), mu_s=2.0, a=1.0):
    return dict(bravais=[[1, 0, 0], [0, 1, 0], [0, 0, 1]], basis=[[0, 0, 0]],
                n_cells=[n0, n1, 1], periodic=[int(periodic[0]), int(periodic[1]), 0],
                lattice_constant=a, mu_s=[mu_s])


def simple_cubic(n0, n1=None, n2=None, periodic=(True, True, True), mu_s=2.0, a=1.0):
    n1 = n0 if n1 is None else n1
    n2 = n0 if n2 is None else n2
    return dict(bravais=[[1, 0, 0], [0, 1, 0], [0, 0, 1]], basis=[[0, 0, 0]],
                n_cells=[n0, n1, n2], periodic=[int(p) for p in periodic],
                lattice_constant=a, mu_s=[mu_s])


def hexagonal(n0, n1, periodic=(False, False), mu_s=2.0, a=1.0):
    return dict(bravais=[[1, 0, 0], [0.5, SQRT3_2, 0], [0, 0, 1]], basis=[[0, 0, 0]],
                n_cells=[n0, n1, 1], periodic=[int(periodic[0]), int(periodic[1]), 0],
                lattice_constant=a, mu_s=[mu_s])


def n_spins(geometry):
    nc = geometry["n_cells"]
    return len(geometry["basis"]) * nc[0] * nc[1] * nc[2]


def site_positions(geometry):
    """Cartesian site positions r_i = a (c + basis_b) . A, index order
    i = b + n_basis (c0 + n0 (c1 + n1 c2))."""
    A = np.asarray(geometry["bravais"], dtype=np.float64)
    basis = np.asarray(geometry["basis"], dtype=np.float64)
    n0, n1, n2 = geometry["n_cells"]
    c2, c1, c0, b = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), np.arange(len(basis)),
                                indexing="ij")
    frac = np.stack([c0, c1, c2], axis=-1).reshape(-1, 3).astype(np.float64) + basis[b.reshape(-1)]
    return geometry.get("lattice_constant", 1.0) * frac @ A


# ---------------------------------------------------------------- states
def random_spins(n, seed):
    """n unit vectors uniform on the sphere, float64 (n, 3)."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def ferromagnet(n, direction=(0.0, 0.0, 1.0)):
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return np.tile(d, (n, 1))


def perturbed(spins, amplitude, seed):
    rng = np.random.default_rng(seed)
    s = spins + amplitude * rng.standard_normal(spins.shape)
    return s / np.linalg.norm(s, axis=1, keepdims=True)


def flat_spiral(positions, q, e1, e2):
    """n(r) = cos(q.r) e1 + sin(q.r) e2 (e1, e2 orthonormal)."""
    ph = positions @ np.asarray(q, dtype=np.float64)
    e1 = np.asarray(e1, dtype=np.float64)
    e2 = np.asarray(e2, dtype=np.float64)
    return np.cos(ph)[:, None] * e1 + np.sin(ph)[:, None] * e2


def neel_skyrmion(positions, centre, radius, helicity=0.0):
    """Neel-type ansatz: theta(r) = pi (1 - r / R) inside R, 0 outside, core
    pointing to -z in a +z background; in-plane angle = polar angle +
    helicity."""
    d = positions[:, :2] - np.asarray(centre, dtype=np.float64)[None, :2]
    r = np.linalg.norm(d, axis=1)
    theta = np.where(r < radius, math.pi * (1.0 - r / radius), 0.0)
    psi = np.arctan2(d[:, 1], d[:, 0]) + helicity
    return np.stack([np.sin(theta) * np.cos(psi), np.sin(theta) * np.sin(psi), np.cos(theta)], axis=1)


def slerp_chain(first, last, n_images, positions=None, centre=None):
    """Initial GNEB guess: per-spin great-circle interpolation between two
    states.  Antiparallel pairs rotate about the in-plane radial axis
    z x rhat from `centre` (x at the centre, or without positions)."""
    a = np.asarray(first, dtype=np.float64)
    b = np.asarray(last, dtype=np.float64)
    n = a.shape[0]
    c = np.clip(np.sum(a * b, axis=1), -1.0, 1.0)
    ang = np.arccos(c)
    axis = np.cross(a, b)
    an = np.linalg.norm(axis, axis=1)
    anti = an < 1e-8
    fallback = np.tile(np.array([1.0, 0.0, 0.0]), (n, 1))
    if positions is not None and centre is not None:
        d = positions[:, :2] - np.asarray(centre, dtype=np.float64)[None, :2]
        rad = np.stack([-d[:, 1], d[:, 0], np.zeros(n)], axis=1)
        rn = np.linalg.norm(rad, axis=1)
        fallback = np.where(rn[:, None] > 1e-12, rad / np.maximum(rn, 1e-300)[:, None], fallback)
    # an axis perpendicular to a for the antiparallel (or identical) case
    fb = fallback - np.sum(fallback * a, axis=1, keepdims=True) * a
    fbn = np.linalg.norm(fb, axis=1)
    fb = np.where(fbn[:, None] > 1e-12, fb / np.maximum(fbn, 1e-300)[:, None],
                  np.cross(a, np.array([0.0, 1.0, 0.0])))
    axis = np.where(anti[:, None], fb, axis / np.maximum(an, 1e-300)[:, None])
    chain = np.empty((n_images, n, 3))
    for v in range(n_images):
        t = v / (n_images - 1)
        th = ang * t
        k = axis
        kxa = np.cross(k, a)
        kda = np.sum(k * a, axis=1, keepdims=True)
        chain[v] = a * np.cos(th)[:, None] + kxa * np.sin(th)[:, None] + k * kda * (1 - np.cos(th))[:, None]
    chain[0] = a
    chain[-1] = b
    return chain


# ---------------------------------------------------------------- workloads
def cfg_square_32():
    """32x32 square lattice, open, J=1, interfacial D=0.3, K=0.1 z, B=1 T z,
    mu_s=2; random start (seed 0); Depondt LLG dt=1e-3 ps, alpha=0.3, 1000
    steps, FP64."""
    g = square(32, 32, periodic=(False, False), mu_s=2.0)
    h = dict(B=[0, 0, 1.0], K=[0.1], Khat=[[0, 0, 1]], J=[1.0], dmi_kind="interfacial", D=[0.3])
    run = dict(solver="depondt", dt=1e-3, alpha=0.3, T=0.0, n_steps=1000, seed=0)
    return dict(name="square32_depondt_fp64", geometry=g, hamiltonian=h, run=run, spin_seed=0)


def cfg_sc_128(n=128):
    """n^3 simple cubic, periodic, J1=1.0, J2=-0.2, J3=0.05, bulk D=0.2
    (first shell), K=0.05 z, B=0, mu_s=2; random start (seed 1); stochastic
    Heun at T=10 K (thermal seed 1), alpha=0.1, dt=1e-3 ps, 10k steps."""
    g = simple_cubic(n, periodic=(True, True, True), mu_s=2.0)
    h = dict(B=[0, 0, 0], K=[0.05], Khat=[[0, 0, 1]], J=[1.0, -0.2, 0.05], dmi_kind="bulk", D=[0.2])
    run = dict(solver="heun", dt=1e-3, alpha=0.1, T=10.0, n_steps=10000, seed=1)
    return dict(name="sc%d_heun_sllg" % n, geometry=g, hamiltonian=h, run=run, spin_seed=1)


def cfg_hex_dipole(n=512):
    """n x n hexagonal monolayer, open, mu_s=3, J=1, interfacial D=0.3,
    K=0.2 z, B=0, dipole-dipole by zero-padded FFT; random start (seed 2);
    Depondt, alpha=0.5, dt=1e-3 ps, 2000 steps."""
    g = hexagonal(n, n, periodic=(False, False), mu_s=3.0)
    h = dict(B=[0, 0, 0], K=[0.2], Khat=[[0, 0, 1]], J=[1.0], dmi_kind="interfacial", D=[0.3],
             dipole="fft")
    run = dict(solver="depondt", dt=1e-3, alpha=0.5, T=0.0, n_steps=2000, seed=2)
    return dict(name="hex%d_dipole_depondt" % n, geometry=g, hamiltonian=h, run=run, spin_seed=2)


# With the interfacial convention D_ij = D (z x rhat_ij) and D > 0, the
# metastable Neel skyrmion in a +z background has helicity pi (its in-plane
# part points towards the core); helicity 0 unwinds.
SKYRMION_HELICITY = math.pi


def gneb_draw(seed, index, attempt=0, sizes=(64, 96, 128), images=(12, 40)):
    """Parameters of chain `index` of the batched GNEB workload: image count
    U{12..40}, periodic hexagonal lattice side from `sizes`, skyrmion radius
    U{3..8} sites, J=1, D~U[0.25,0.4], K~U[0.05,0.1] (z), B~U[0.5,2] T (z),
    mu_s=2.  `attempt` > 0 gives the redraw used when a draw has no
    metastable isolated skyrmion."""
    rng = np.random.default_rng([seed, index, attempt])
    L = int(rng.choice(sizes))
    M = int(rng.integers(images[0], images[1] + 1))
    R = int(rng.integers(3, 9))
    D = float(rng.uniform(0.25, 0.4))
    K = float(rng.uniform(0.05, 0.1))
    B = float(rng.uniform(0.5, 2.0))
    g = hexagonal(L, L, periodic=(True, True), mu_s=2.0)
    h = dict(B=[0, 0, B], K=[K], Khat=[[0, 0, 1]], J=[1.0], dmi_kind="interfacial", D=[D])
    return dict(index=index, attempt=attempt, seed=seed, L=L, n_images=M, radius=R, geometry=g, hamiltonian=h)


def gneb_batch(n_chains=48, seed=4, sizes=(64, 96, 128), images=(12, 40)):
    """First draws of the batched GNEB workload (see gneb_draw)."""
    return [gneb_draw(seed, c, 0, sizes, images) for c in range(n_chains)]


# ---------------------------------------------------------------- warm start
WARMSTART_SEEDS = dict(train=5, heldout=6)
# the learned warm start of GNEB paths: gneb_draw chains of 128 x 128 lattices
# with 16 images, training and held-out seeds
GNEB_WARMSTART_SEEDS = dict(train=7, heldout=8)


def warmstart_draw(seed, index, L=128):
    """System `index` of the learned warm-start workload: an L x L periodic
    hexagonal monolayer, mu_s=2, J=1 meV, interfacial D~U[0.1,0.5] meV,
    K~U[0,0.2] meV along z, B~U[0,3] T along z, spins uniform on the sphere.
    Each system has its own generator (seed, index), so any subset can be
    drawn without the others."""
    rng = np.random.default_rng([seed, index])
    D = float(rng.uniform(0.1, 0.5))
    K = float(rng.uniform(0.0, 0.2))
    B = float(rng.uniform(0.0, 3.0))
    spin_seed = int(rng.integers(0, 2**62))
    g = hexagonal(L, L, periodic=(True, True), mu_s=2.0)
    h = dict(B=[0, 0, B], K=[K], Khat=[[0, 0, 1]], J=[1.0], dmi_kind="interfacial", D=[D])
    return dict(index=index, seed=seed, L=L, J=1.0, D=D, K=K, B=B, geometry=g, hamiltonian=h,
                spins=random_spins(L * L, spin_seed))


def warmstart_features(draw):
    """The 4 per-system scalars the warm-start network sees: J, D/0.5, K/0.2
    and B/3 (the workload's parameter ranges scaled to about [0, 1])."""
    return np.array([draw["J"], draw["D"] / 0.5, draw["K"] / 0.2, draw["B"] / 3.0], dtype=np.float32)


# (cin, cout) of the network's 14 convolutions, in parameter order: encoder
# 32-32, 32-64, 64-128, 128-256 (two each), decoder 384-128, 128-128,
# 192-64, 64-64, 96-32, 32-32; then the 32 -> 3 head.
UNET_LAYERS = [(32, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (128, 256), (256, 256),
               (384, 128), (128, 128), (192, 64), (64, 64), (96, 32), (32, 32)]
UNET_REAL_INPUTS = 7  # n (3) + features (4); the other input channels are zero


def unet_n_params(layers=UNET_LAYERS, head_in=32):
    return sum(co * 9 * ci + co for ci, co in layers) + 3 * head_in + 3


def unet_init(seed, layers=UNET_LAYERS, head_in=32, real_inputs=UNET_REAL_INPUTS):
    """Initial flat parameters (float32): He-normal convolution weights
    (std sqrt(2 / (9 * fan-in channels))), zero on the first layer's padding
    channels, zero biases, head weights with std sqrt(1 / head_in)."""
    rng = np.random.default_rng(seed)
    parts = []
    for l, (ci, co) in enumerate(layers):
        fan = real_inputs if l == 0 else ci
        W = rng.standard_normal((co, 9, ci)) * math.sqrt(2.0 / (9 * fan))
        if l == 0:
            W[:, :, real_inputs:] = 0.0
        parts += [W.ravel(), np.zeros(co)]
    parts += [rng.standard_normal(3 * head_in) * math.sqrt(1.0 / head_in), np.zeros(3)]
    return np.concatenate(parts).astype(np.float32)
