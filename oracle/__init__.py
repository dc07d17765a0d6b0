"""Python view of the FP64 CPU oracle (``spo.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg are the only callers.  The oracle is written from the paper's
equations (arXiv:1901.11350, Eq. 1, Eq. 3-4, Appendices A, B, D, F, G) and
shares no code with the CUDA library; it takes plain dictionaries and numpy
arrays, never anything from the product package.

Geometry dictionary keys: ``bravais`` (3x3, rows are lattice vectors in units
of the lattice constant), ``basis`` (n_basis x 3 fractional), ``n_cells``,
``periodic``, ``lattice_constant`` (Angstrom), ``mu_s`` (Bohr magnetons per
basis atom).

Hamiltonian dictionary keys (all optional): ``B`` (T), ``K`` and ``Khat`` per
basis atom, ``J`` (list per shell, meV), ``dmi_kind`` (``none``, ``bulk``,
``interfacial``), ``D`` (list per shell), ``dipole`` (``none``, ``direct``,
``fft``), ``pairs`` (list of ``(i, j, (d0, d1, d2), J, (Dx, Dy, Dz))``),
``gauss`` (rows ``(a, sigma, cx, cy, cz)``, Appendix G landscape).
"""
import ctypes as C

import numpy as np

from . import build as _build

MAX_BASIS = 8
MAX_SHELLS = 8
MAX_GAUSS = 16
DMI = {"none": 0, "bulk": 1, "interfacial": 2}
DIPOLE = {"none": 0, "direct": 1, "fft": 2}
SOLVER = {"depondt": 0, "heun": 1, "sib": 2, "rk4": 3}

# Constants as the oracle states them (CODATA 2018), for tests' closed forms.
MU_B = 0.05788381806
K_B = 0.08617333262
GAMMA = 0.176085963023
C_DIP = 0.05368151123574179


class _Pair(C.Structure):
    _fields_ = [("i", C.c_int), ("j", C.c_int), ("d", C.c_int * 3), ("J", C.c_double),
                ("D", C.c_double * 3)]


class _Ham(C.Structure):
    _fields_ = [("B", C.c_double * 3), ("K", C.c_double * MAX_BASIS),
                ("Khat", (C.c_double * 3) * MAX_BASIS), ("n_shells", C.c_int),
                ("J", C.c_double * MAX_SHELLS), ("dmi_kind", C.c_int), ("n_dmi_shells", C.c_int),
                ("D", C.c_double * MAX_SHELLS), ("dipole", C.c_int), ("n_pairs", C.c_int),
                ("pairs", C.POINTER(_Pair)), ("n_gauss", C.c_int),
                ("gauss", (C.c_double * 5) * MAX_GAUSS)]


class _LLG(C.Structure):
    _fields_ = [("solver", C.c_int), ("dt", C.c_double), ("alpha", C.c_double), ("T", C.c_double),
                ("seed", C.c_uint64), ("step0", C.c_uint64), ("replica", C.c_uint32)]


class _GNEB(C.Structure):
    _fields_ = [("dt", C.c_double), ("mass", C.c_double), ("k_spring", C.c_double),
                ("climbing", C.c_int), ("image_types", C.POINTER(C.c_int)), ("energy_weight", C.c_double)]


IMAGE = {"normal": 0, "climbing": 1, "falling": 2}


class _MC(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("sweep0", C.c_uint64), ("target_accept", C.c_double), ("sample", C.c_int)]


def segment_length(Ea, Eb, da, db, h, w):
    """Energy-weighted length of a path segment (see spo.h)."""
    return lib().spo_segment_length(float(Ea), float(Eb), float(da), float(db), float(h), float(w))


def _gneb_params(dt, mass, k_spring, climbing, image_types, energy_weight):
    """The parameter block and the int array it points to (keep both alive)."""
    types = None
    if image_types is not None:
        types = (C.c_int * len(image_types))(*[IMAGE[t] if isinstance(t, str) else int(t) for t in image_types])
    p = _GNEB(float(dt), float(mass), float(k_spring), int(bool(climbing)),
              C.cast(types, C.POINTER(C.c_int)) if types is not None else None, float(energy_weight))
    return p, types


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.POINTER
        d = P(C.c_double)
        L.spo_create.argtypes = [P(C.c_void_p)]
        L.spo_destroy.argtypes = [C.c_void_p]
        L.spo_destroy.restype = None
        L.spo_set_geometry.argtypes = [C.c_void_p, d, C.c_int, d, P(C.c_int), P(C.c_int), C.c_double, d]
        L.spo_set_hamiltonian.argtypes = [C.c_void_p, P(_Ham)]
        L.spo_n_spins.argtypes = [C.c_void_p]
        L.spo_positions.argtypes = [C.c_void_p, d]
        L.spo_n_neighbours.argtypes = [C.c_void_p, C.c_int]
        L.spo_shell_radius.argtypes = [C.c_void_p, C.c_int, d]
        L.spo_effective_field.argtypes = [C.c_void_p, d, d, C.c_int]
        L.spo_dipole_field.argtypes = [C.c_void_p, d, d, C.c_int]
        L.spo_dipole_field_direct_at.argtypes = [C.c_void_p, d, C.c_int, P(C.c_int), d]
        L.spo_energy.argtypes = [C.c_void_p, d, d]
        L.spo_llg.argtypes = [C.c_void_p, d, P(_LLG), C.c_int]
        L.spo_minimise.argtypes = [C.c_void_p, d, d, C.c_double, C.c_double, C.c_double, C.c_int,
                                   P(C.c_int), d]
        L.spo_gneb.argtypes = [C.c_void_p, d, d, C.c_int, P(_GNEB), C.c_int, C.c_double, d, d,
                               P(C.c_int)]
        L.spo_gneb_forces.argtypes = [C.c_void_p, d, C.c_int, P(_GNEB), d, d, d, P(C.c_int)]
        L.spo_gneb_path.argtypes = [C.c_void_p, d, C.c_int, C.c_int, d, d, d, d, d, d]
        L.spo_hessian_apply.argtypes = [C.c_void_p, d, d, d]
        L.spo_hessian_dense.argtypes = [C.c_void_p, d, d, d]
        L.spo_mc.argtypes = [C.c_void_p, d, C.c_int, d, P(_MC), C.c_int, d, d]
        L.spo_mc_coloured.argtypes = [C.c_void_p, d, C.c_int, d, P(_MC), C.c_int, d, d]
        L.spo_mc_colours.argtypes = [C.c_void_p]
        L.spo_segment_length.argtypes = [C.c_double] * 6
        L.spo_segment_length.restype = C.c_double
        L.spo_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
        L.spo_philox4x32_10.restype = None
        L.spo_thermal_normals.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, d]
        L.spo_thermal_normals.restype = None
        L.spo_topological_charge.argtypes = [C.c_void_p, d, d]
        L.spo_threads.argtypes = []
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, rc))


def threads():
    return lib().spo_threads()


def philox4x32_10(ctr, key):
    """Raw Philox4x32-10 block for a 4-word counter and a 2-word key."""
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().spo_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def thermal_normals(seed, step, replica, i):
    out = np.zeros(3)
    lib().spo_thermal_normals(int(seed), int(step), int(replica), int(i), _dp(out))
    return out


class System:
    """One lattice + Hamiltonian in the oracle."""

    def __init__(self, geometry, hamiltonian):
        L = lib()
        self._h = C.c_void_p()
        _check(L.spo_create(C.byref(self._h)), "create")
        g = geometry
        brav = np.ascontiguousarray(np.asarray(g["bravais"], dtype=np.float64).reshape(9))
        basis = np.ascontiguousarray(np.asarray(g.get("basis", [[0, 0, 0]]), dtype=np.float64))
        nb = basis.shape[0]
        nc = (C.c_int * 3)(*[int(x) for x in g["n_cells"]])
        per = (C.c_int * 3)(*[int(bool(x)) for x in g["periodic"]])
        mu = np.ascontiguousarray(np.broadcast_to(np.asarray(g["mu_s"], dtype=np.float64), (nb,)).copy())
        _check(L.spo_set_geometry(self._h, _dp(brav), nb, _dp(basis.reshape(-1)), nc, per,
                                  float(g.get("lattice_constant", 1.0)), _dp(mu)), "set_geometry")
        self.n_basis = nb
        self.mu_s = mu.copy()
        self.N = L.spo_n_spins(self._h)
        h = hamiltonian
        H = _Ham()
        for k, v in enumerate(h.get("B", [0, 0, 0])):
            H.B[k] = float(v)
        K = np.broadcast_to(np.asarray(h.get("K", 0.0), dtype=np.float64), (nb,))
        Kh = np.broadcast_to(np.asarray(h.get("Khat", [0, 0, 1]), dtype=np.float64), (nb, 3))
        for b in range(nb):
            H.K[b] = float(K[b])
            for k in range(3):
                H.Khat[b][k] = float(Kh[b, k])
        J = list(h.get("J", []))
        H.n_shells = len(J)
        for q, v in enumerate(J):
            H.J[q] = float(v)
        H.dmi_kind = DMI[h.get("dmi_kind", "none")]
        D = list(h.get("D", []))
        H.n_dmi_shells = len(D)
        for q, v in enumerate(D):
            H.D[q] = float(v)
        H.dipole = DIPOLE[h.get("dipole", "none")]
        pairs = list(h.get("pairs", []))
        self._pairs = (_Pair * max(1, len(pairs)))()
        for q, (i, j, d, Jp, Dp) in enumerate(pairs):
            self._pairs[q].i, self._pairs[q].j = int(i), int(j)
            for k in range(3):
                self._pairs[q].d[k] = int(d[k])
                self._pairs[q].D[k] = float(Dp[k])
            self._pairs[q].J = float(Jp)
        H.n_pairs = len(pairs)
        H.pairs = C.cast(self._pairs, C.POINTER(_Pair))
        gauss = list(h.get("gauss", []))
        H.n_gauss = len(gauss)
        for q, row in enumerate(gauss):
            for k in range(5):
                H.gauss[q][k] = float(row[k])
        _check(L.spo_set_hamiltonian(self._h, C.byref(H)), "set_hamiltonian")

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.spo_destroy(self._h)
            self._h = None

    def _spins(self, n):
        a = np.ascontiguousarray(np.asarray(n, dtype=np.float64)[..., :3]).copy()
        if a.shape != (self.N, 3):
            raise ValueError("expected %d x 3 spins, got %s" % (self.N, a.shape))
        return a

    def positions(self):
        r = np.zeros((self.N, 3))
        _check(lib().spo_positions(self._h, _dp(r)), "positions")
        return r

    def n_neighbours(self, basis=0):
        return lib().spo_n_neighbours(self._h, basis)

    def shell_radius(self, shell):
        r = C.c_double()
        _check(lib().spo_shell_radius(self._h, shell, C.byref(r)), "shell_radius")
        return r.value

    def field(self, n, dipole=None):
        n = self._spins(n)
        B = np.zeros_like(n)
        m = -1 if dipole is None else DIPOLE[dipole]
        _check(lib().spo_effective_field(self._h, _dp(n), _dp(B), m), "effective_field")
        return B

    def gradient(self, n):
        return -self.field(n)

    def dipole_field(self, n, method):
        n = self._spins(n)
        B = np.zeros_like(n)
        _check(lib().spo_dipole_field(self._h, _dp(n), _dp(B), DIPOLE[method]), "dipole_field")
        return B

    def dipole_field_direct_at(self, n, idx):
        n = self._spins(n)
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int32))
        B = np.zeros((idx.size, 3))
        _check(lib().spo_dipole_field_direct_at(self._h, _dp(n), int(idx.size),
                                                idx.ctypes.data_as(C.POINTER(C.c_int)), _dp(B)),
               "dipole_field_direct_at")
        return B

    def energy(self, n):
        """[total, Zeeman, anisotropy, exchange, DMI, dipole] in meV."""
        n = self._spins(n)
        e = np.zeros(6)
        _check(lib().spo_energy(self._h, _dp(n), _dp(e)), "energy")
        return e

    def llg(self, n, n_steps, solver="depondt", dt=1e-3, alpha=0.1, T=0.0, seed=0, step0=0, replica=0):
        n = self._spins(n)
        p = _LLG(SOLVER[solver], float(dt), float(alpha), float(T), int(seed), int(step0), int(replica))
        _check(lib().spo_llg(self._h, _dp(n), C.byref(p), int(n_steps)), "llg")
        return n

    def minimise(self, n, v=None, dt=0.1, mass=1.0, tol=1e-6, max_iter=10000):
        n = self._spins(n)
        v = np.zeros_like(n) if v is None else self._spins(v)
        it = C.c_int()
        mt = C.c_double()
        _check(lib().spo_minimise(self._h, _dp(n), _dp(v), float(dt), float(mass), float(tol),
                                  int(max_iter), C.byref(it), C.byref(mt)), "minimise")
        return n, v, it.value, mt.value

    def gneb_forces(self, chain, k_spring=1.0, climbing=True, dt=0.1, mass=1.0, image_types=None, energy_weight=0.0):
        ch = np.ascontiguousarray(np.asarray(chain, dtype=np.float64)[..., :3]).copy()
        M = ch.shape[0]
        F = np.zeros_like(ch)
        E = np.zeros(M)
        l = np.zeros(max(M - 1, 1))
        ci = C.c_int()
        p, _keep = _gneb_params(dt, mass, k_spring, climbing, image_types, energy_weight)
        _check(lib().spo_gneb_forces(self._h, _dp(ch), M, C.byref(p), _dp(F), _dp(E), _dp(l),
                                     C.byref(ci)), "gneb_forces")
        return F, E, l[:M - 1], ci.value

    def gneb(self, chain, vel=None, n_iter=100, tol=0.0, k_spring=1.0, climbing=True, dt=0.1, mass=1.0,
             image_types=None, energy_weight=0.0):
        ch = np.ascontiguousarray(np.asarray(chain, dtype=np.float64)[..., :3]).copy()
        M = ch.shape[0]
        v = np.zeros_like(ch) if vel is None else np.ascontiguousarray(
            np.asarray(vel, dtype=np.float64)[..., :3]).copy()
        E = np.zeros(M)
        mf = C.c_double()
        it = C.c_int()
        p, _keep = _gneb_params(dt, mass, k_spring, climbing, image_types, energy_weight)
        _check(lib().spo_gneb(self._h, _dp(ch), _dp(v), M, C.byref(p), int(n_iter), float(tol),
                              _dp(E), C.byref(mf), C.byref(it)), "gneb")
        return ch, v, E, mf.value, it.value

    def gneb_path(self, chain, n_interp=10, charge=False):
        """Per image (r, E, dE/dr[, Q]) and the cubic interpolation (r_i, E_i)."""
        ch = np.ascontiguousarray(np.asarray(chain, dtype=np.float64)[..., :3]).copy()
        M = ch.shape[0]
        r, E, sl = np.zeros(M), np.zeros(M), np.zeros(M)
        Q = np.zeros(M) if charge else None
        ri, Ei = np.zeros((M - 1) * n_interp + 1), np.zeros((M - 1) * n_interp + 1)
        _check(lib().spo_gneb_path(self._h, _dp(ch), M, int(n_interp), _dp(r), _dp(E), _dp(sl),
                                   _dp(Q) if charge else None, _dp(ri), _dp(Ei)), "gneb_path")
        out = dict(r=r, E=E, slope=sl, r_interp=ri, E_interp=Ei)
        if charge:
            out["Q"] = Q
        return out

    def hessian_apply(self, n, v):
        n = self._spins(n)
        v = np.ascontiguousarray(np.asarray(v, dtype=np.float64)[..., :3]).reshape(-1, 3).copy()
        out = np.zeros_like(n)
        _check(lib().spo_hessian_apply(self._h, _dp(n), _dp(v), _dp(out)), "hessian_apply")
        return out

    def hessian_dense(self, n):
        """(H [2N, 2N], T [N, 3, 2]) of the covariant Hessian in the tangent basis."""
        n = self._spins(n)
        H = np.zeros((2 * self.N, 2 * self.N))
        T = np.zeros((self.N, 3, 2))
        _check(lib().spo_hessian_dense(self._h, _dp(n), _dp(H), _dp(T)), "hessian_dense")
        return H, T

    def lowest_mode(self, n):
        """Lowest eigenvalue of the covariant Hessian and its eigenvector as
        an N x 3 unit tangent field (dense eigen-decomposition)."""
        H, T = self.hessian_dense(n)
        w, V = np.linalg.eigh(0.5 * (H + H.T))
        mode = np.einsum("ikc,ic->ik", T, V[:, 0].reshape(-1, 2))
        return w[0], mode / np.linalg.norm(mode)

    def hessian_eigen(self, n):
        """All 2N eigenvalues (ascending) and eigenvectors (columns, in the
        tangent basis T) of the covariant Hessian at n, by dense
        eigen-decomposition."""
        H, T = self.hessian_dense(n)
        lam, vec = np.linalg.eigh(0.5 * (H + H.T))
        return lam, vec, T

    def htst(self, n_min, n_sad, zero_tol=1e-6, V_min=1.0, V_sad=1.0):
        """Harmonic transition-state theory rate prefactor (Sec. HTST) of the
        transition from the minimum n_min over the first-order saddle n_sad:
        Gamma = v/(2 pi) Omega_0 exp(-dE/kB T), with
          Omega_0 = sqrt(prod' lambda^M / prod' lambda^S)   (eigenvalues above zero_tol),
          v = (2 pi kB T)^((N0^M - N0^S)/2) V^S/V^M sqrt(sum'_i a_i^2 / lambda^S_i),
        a_i the first row (the unstable mode's) of the dynamical matrix in the
        Hessian's eigenbasis, V|2N = Lambda^T T^T V|3N T Lambda.  The dynamical
        matrix is the linearisation at the saddle of the precession without
        damping, dn_i/dt = (gamma/mu_i) n_i x grad_i H, i.e. V|3N = G H|3N with
        G_ii = (gamma/mu_i) [n_i]_x; in the eigenbasis its first row is
        (Lambda^T T^T G T Lambda)_1k lambda_k.  Returns a dict with the fields
        of the C result (prefactor = v/(2 pi) Omega_0 V^S/V^M without the
        (2 pi kB T) factor) and the eigenvalues."""
        out = {}
        spec = {}
        for tag, n in (("min", n_min), ("sad", n_sad)):
            lam, vec, T = self.hessian_eigen(n)
            pos = lam > zero_tol
            spec[tag] = (lam, vec, T)
            out["log_det_" + tag] = float(np.sum(np.log(lam[pos])))
            out["n_zero_" + tag] = int(np.sum(np.abs(lam) <= zero_tol))
            out["n_neg_" + tag] = int(np.sum(lam < -zero_tol))
            out["E_" + tag] = float(self.energy(n)[0])
            out["eig_" + tag] = lam
        out["dE"] = out["E_sad"] - out["E_min"]
        lam, vec, T = spec["sad"]
        n = self._spins(n_sad)
        # G in the tangent basis, 2 x 2 per spin: T_i^T (gamma/mu_i) [n_i]_x T_i
        W = np.zeros((2 * self.N, 2 * self.N))
        for i in range(self.N):
            x = n[i]
            nx = np.array([[0.0, -x[2], x[1]], [x[2], 0.0, -x[0]], [-x[1], x[0], 0.0]])
            mu = self.mu_s[i % self.n_basis] * MU_B
            W[2 * i:2 * i + 2, 2 * i:2 * i + 2] = (GAMMA / mu) * (T[i].T @ nx @ T[i])
        Vd = (vec.T @ W @ vec) * lam[None, :]  # the dynamical matrix in the eigenbasis
        a = Vd[0, :]                            # the unstable mode's row
        pos = lam > zero_tol
        out["a"] = a
        out["lambda_unstable"] = float(lam[0])
        out["v"] = float(np.sqrt(np.sum(a[pos] ** 2 / lam[pos])))
        out["omega0"] = float(np.exp(0.5 * (out["log_det_min"] - out["log_det_sad"])))
        out["prefactor"] = out["v"] / (2.0 * np.pi) * out["omega0"] * V_sad / V_min
        return out

    def mmf(self, n, n_iter, dt=0.1, mass=1.0, vel=None):
        """Minimum mode following (Sec. MMF): velocity projection (Appendix D)
        with the effective force F - 2 (F.l) l, l the lowest mode; where the
        lowest eigenvalue is not negative, -(F.l) l (reading: climb along the
        lowest mode only).  Returns (n, v, F, lambda_min)."""
        x = self._spins(n).copy()
        v = np.zeros_like(x) if vel is None else np.asarray(vel, dtype=np.float64)[..., :3].reshape(-1, 3).copy()

        def force(x):
            B = self.field(x)
            F = B - np.sum(B * x, axis=1, keepdims=True) * x
            lam, l = self.lowest_mode(x)
            fl = np.sum(F * l)
            Fe = F - 2.0 * fl * l if lam < 0 else -fl * l
            return F, Fe, lam

        F, Fe, lam = force(x)
        for _ in range(n_iter):
            y = x + dt * v + dt * dt / (2 * mass) * Fe
            y /= np.linalg.norm(y, axis=1, keepdims=True)
            F2, Fe2, lam = force(y)
            v = v + dt / (2 * mass) * (Fe + Fe2)
            vf = np.sum(v * Fe2)
            ff = np.sum(Fe2 * Fe2)
            v = (vf / ff) * Fe2 if (vf > 0 and ff > 0) else np.zeros_like(v)
            x, F, Fe = y, F2, Fe2
        return x, v, F, lam

    def mc_colours(self):
        return lib().spo_mc_colours(self._h)

    def mc(self, spins, T, n_sweeps, seed=0, sweep0=0, target_accept=0.5, sample=True, cone=None, stats=None,
           order="random"):
        """Metropolis sweeps of replicas spins [R, N, 3] at temperatures T[R];
        returns (spins, cone[R], stats[R, 8]).  order "random": each sweep
        visits the spins in a fresh random order (the method's sweep);
        "coloured": colour by colour of the lattice colouring (a check of a
        colour-parallel decomposition)."""
        x = np.ascontiguousarray(np.asarray(spins, dtype=np.float64)[..., :3]).copy()
        R = x.shape[0]
        Tk = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(R))
        cn = np.full(R, 0.5) if cone is None else np.ascontiguousarray(np.asarray(cone, dtype=np.float64)).copy()
        st = np.zeros((R, 8)) if stats is None else np.ascontiguousarray(np.asarray(stats, dtype=np.float64)).copy()
        p = _MC(int(seed), int(sweep0), float(target_accept), int(bool(sample)))
        fn = {"random": lib().spo_mc, "coloured": lib().spo_mc_coloured}[order]
        _check(fn(self._h, _dp(x), R, _dp(Tk), C.byref(p), int(n_sweeps), _dp(cn), _dp(st)), "mc")
        return x, cn, st

    def topological_charge(self, n):
        n = self._spins(n)
        q = C.c_double()
        _check(lib().spo_topological_charge(self._h, _dp(n), C.byref(q)), "topological_charge")
        return q.value
