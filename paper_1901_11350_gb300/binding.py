"""Thin Python binding of ``libspirit_gb.so`` (include/spirit_gb.h).

Argument marshalling only: tensors are checked for device, dtype, shape and
contiguity, and their device pointers are passed to the C ABI together with
torch's current CUDA stream.  Every step of the computation runs in the
library's CUDA kernels; there is no CPU path.  The library must have been
built (``paper_1901_11350_gb300.build.build()``); loading fails loudly
otherwise.
"""
import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

MAX_BASIS = 4
MAX_SHELLS = 8
F32, F64 = 0, 1
DMI = {"none": 0, "bulk": 1, "interfacial": 2}
DIPOLE = {"none": 0, "fft": 2}
SOLVER = {"depondt": 0, "heun": 1, "sib": 2, "rk4": 3}
ERRORS = {-1: "SP_ERR_ARG", -2: "SP_ERR_STATE", -3: "SP_ERR_CUDA", -4: "SP_ERR_UNSUPPORTED",
          -5: "SP_ERR_TIMEOUT", -6: "SP_ERR_NAN"}


class SpinError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class Pair(C.Structure):
    _fields_ = [("i", C.c_int), ("j", C.c_int), ("d", C.c_int * 3), ("J", C.c_double), ("D", C.c_double * 3)]


class Hamiltonian(C.Structure):
    _fields_ = [("B", C.c_double * 3), ("K", C.c_double * MAX_BASIS), ("Khat", (C.c_double * 3) * MAX_BASIS),
                ("n_shells", C.c_int), ("J", C.c_double * MAX_SHELLS), ("dmi_kind", C.c_int),
                ("n_dmi_shells", C.c_int), ("D", C.c_double * MAX_SHELLS), ("dipole", C.c_int),
                ("n_pairs", C.c_int), ("pairs", C.POINTER(Pair))]


class LLGParams(C.Structure):
    _fields_ = [("solver", C.c_int), ("dt", C.c_double), ("alpha", C.c_double), ("T", C.c_double),
                ("seed", C.c_uint64), ("step0", C.c_uint64), ("replica", C.c_uint32)]


class GNEBParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("mass", C.c_double), ("k_spring", C.c_double), ("climbing", C.c_int),
                ("image_types", C.POINTER(C.c_int)), ("energy_weight", C.c_double)]


IMAGE_KINDS = {"normal": 0, "climbing": 1, "falling": 2}


class MMFParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("mass", C.c_double), ("krylov", C.c_int)]


class HTSTParams(C.Structure):
    _fields_ = [("zero_tol", C.c_double), ("V_min", C.c_double), ("V_sad", C.c_double)]


class HTSTResult(C.Structure):
    _fields_ = [("E_min", C.c_double), ("E_sad", C.c_double), ("dE", C.c_double), ("log_det_min", C.c_double),
                ("log_det_sad", C.c_double), ("omega0", C.c_double), ("v", C.c_double),
                ("lambda_unstable", C.c_double), ("prefactor", C.c_double), ("n_zero_min", C.c_int),
                ("n_zero_sad", C.c_int), ("n_neg_min", C.c_int), ("n_neg_sad", C.c_int)]


class MCParams(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("sweep0", C.c_uint64), ("target_accept", C.c_double), ("sample", C.c_int)]


def gneb_params(dt, mass, k_spring, climbing, image_types=None, energy_weight=0.0):
    """The parameter block and the int array it points to (keep both alive)."""
    arr = None
    if image_types is not None:
        arr = (C.c_int * len(image_types))(*[IMAGE_KINDS[t] if isinstance(t, str) else int(t) for t in image_types])
    p = GNEBParams(float(dt), float(mass), float(k_spring), int(bool(climbing)),
                   C.cast(arr, C.POINTER(C.c_int)) if arr is not None else None, float(energy_weight))
    return p, arr


_lib = None

# every entry point of include/spirit_gb.h with its ctypes signature
_vp, _i, _d = C.c_void_p, C.c_int, C.c_double
SIGNATURES = {
    "sp_create": (_i, [C.POINTER(_vp), _i]),
    "sp_destroy": (_i, [_vp]),
    "sp_last_error": (C.c_char_p, [_vp]),
    "sp_sync_status": (_i, [_vp]),
    "sp_set_geometry": (_i, [_vp, C.POINTER(_d), _i, C.POINTER(_d), C.POINTER(_i), C.POINTER(_i), _d, C.POINTER(_d)]),
    "sp_set_hamiltonian": (_i, [_vp, C.POINTER(Hamiltonian)]),
    "sp_n_spins": (_i, [_vp, C.POINTER(_i)]),
    "sp_effective_field": (_i, [_vp, _vp, _vp, _vp]),
    "sp_gradient": (_i, [_vp, _vp, _vp, _vp]),
    "sp_energy": (_i, [_vp, _vp, _vp, _vp]),
    "sp_max_torque": (_i, [_vp, _vp, _vp, _vp]),
    "sp_topological_charge": (_i, [_vp, _vp, _vp, _vp]),
    "sp_llg_step": (_i, [_vp, _vp, C.POINTER(LLGParams), _i, _vp]),
    "sp_llg_step_replicas": (_i, [_vp, _vp, _i, C.POINTER(_d), C.POINTER(LLGParams), _i, _vp]),
    "sp_sample": (_i, [_vp, _vp, _i, _vp, _vp]),
    "sp_llg_step_batch": (_i, [C.POINTER(_vp), _i, _vp, C.POINTER(C.c_longlong), C.POINTER(_d), C.POINTER(LLGParams),
                              _i, _vp]),
    "sp_minimise": (_i, [_vp, _vp, _vp, _d, _d, _d, _i, _i, C.POINTER(_i), C.POINTER(_d), _vp]),
    "sp_gneb_step": (_i, [_vp, _vp, _vp, _i, C.POINTER(GNEBParams), _i, _vp, _vp, _vp]),
    "sp_gneb_batch_step": (_i, [C.POINTER(_vp), _i, _vp, _vp, C.POINTER(C.c_longlong), C.POINTER(_i),
                               C.POINTER(GNEBParams), _i, _vp, _vp, _vp]),
    "sp_hessian_apply": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "sp_lowest_mode": (_i, [_vp, _vp, _vp, _i, C.POINTER(_d), _vp]),
    "sp_mmf": (_i, [_vp, _vp, _vp, _vp, C.POINTER(MMFParams), _i, C.POINTER(_d), C.POINTER(_d), _vp]),
    "sp_hessian_spectrum": (_i, [_vp, _vp, _vp, _vp]),
    "sp_htst": (_i, [_vp, _vp, _vp, C.POINTER(HTSTParams), C.POINTER(HTSTResult), _vp]),
    "sp_mc_colours": (_i, [_vp, C.POINTER(_i)]),
    "sp_mc_sweeps": (_i, [_vp, _vp, _i, C.POINTER(_d), C.POINTER(MCParams), _i, _vp, _vp, _vp]),
    "sp_gneb_path": (_i, [_vp, _vp, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sp_minimise_batch": (_i, [C.POINTER(_vp), _i, _vp, _vp, C.POINTER(C.c_longlong), _d, _d, _d, _i, _i,
                              C.POINTER(_i), C.POINTER(_d), _vp]),
    "sp_llg_step_static": (_i, [_vp, _vp, C.POINTER(LLGParams), _i, _vp]),
    "sp_gneb_batch_autotune": (_i, [C.POINTER(_vp), _i, _vp, _vp, C.POINTER(C.c_longlong), C.POINTER(_i),
                                   C.POINTER(GNEBParams), _i, C.POINTER(_i), C.POINTER(_d), _vp]),
    "sp_set_option": (_i, [_vp, _i, _i]),
    "sp_get_option": (_i, [_vp, _i, C.POINTER(_i)]),
    "sp_autotune": (_i, [_vp, _vp, C.POINTER(_i), _vp]),
    "sp_profile_enable": (_i, [_vp, _i]),
    "sp_profile_read": (_i, [_vp, _i, C.POINTER(_d), C.POINTER(C.c_longlong)]),
    # warm-start network (spirit_gb_unet.h)
    "sp_unet_n_params": (C.c_longlong, []),
    "sp_unet_layer": (_i, [_i, C.POINTER(_i), C.POINTER(_i), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "sp_unet_create": (_i, [C.POINTER(_vp), _i, _i]),
    "sp_unet_destroy": (None, [_vp]),
    "sp_unet_last_error": (C.c_char_p, [_vp]),
    "sp_unet_set_params": (_i, [_vp, _vp, C.c_longlong]),
    "sp_unet_get_params": (_i, [_vp, _vp, C.c_longlong]),
    "sp_unet_predict": (_i, [_vp, _vp, _vp, _i, _vp, _vp]),
    "sp_unet_loss_grad": (_i, [_vp, _vp, _vp, _vp, _i, _vp, _vp, _vp]),
    "sp_unet_adam": (_i, [_vp, _d, _d, _d, _d, _i, _vp]),
    "sp_conv3x3_forward": (_i, [_vp, _i, _i, _vp, _i, _vp, _vp, _i, _vp, _i, _i, _i, _i, _vp, _vp]),
    "sp_conv3x3_transpose": (_i, [_vp, _i, _i, _vp, _vp]),
    "sp_conv3x3_wgrad_workspace": (C.c_longlong, [_i, _i, _i, _i, _i]),
    "sp_conv3x3_set_kernel": (_i, [_i]),
    "sp_conv3x3_get_kernel": (_i, []),
    "sp_unet_device_error": (_i, []),
    "sp_conv3x3_set_wait_limit": (_i, [C.c_longlong]),
    "sp_conv3x3_wgrad": (_i, [_vp, _i, _i, _vp, _i, _vp, _i, _i, _i, _i, _vp, _vp, _vp, C.c_longlong, _vp]),
}
PROFILE_KINDS = {"llg_predictor": 0, "llg_corrector": 1, "dipole": 2}
OPTIONS = {"generic_stencil": 1, "planes_per_cta": 2, "has_cubic_path": 3, "generic_fft": 4, "small_path": 5,
           "planes_per_cta_corr": 6, "mc_resident": 7, "scratch_kib": 8, "gneb_persistent": 9,
           "wait_limit": 10, "cubic_rows": 11, "cubic_rows_corr": 12, "cubic_lean": 13}


def library_path():
    return _build.LIB


def lib():
    """Load the C-ABI library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("CUDA library %s is missing: build it with "
                               "paper_1901_11350_gb300.build.build() (nvcc, sm_103a)" % path)
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class Context:
    """A lattice + Hamiltonian on the GPU, computing in FP32 or FP64."""

    def __init__(self, geometry, hamiltonian, precision="f32"):
        self.precision = precision
        self.dtype = torch.float32 if precision == "f32" else torch.float64
        L = lib()
        self._h = C.c_void_p()
        rc = L.sp_create(C.byref(self._h), F32 if precision == "f32" else F64)
        if rc:
            raise SpinError(rc, "sp_create")
        g = geometry
        brav = np.ascontiguousarray(np.asarray(g["bravais"], dtype=np.float64).reshape(9))
        basis = np.ascontiguousarray(np.asarray(g.get("basis", [[0, 0, 0]]), dtype=np.float64))
        nb = basis.shape[0]
        mu = np.ascontiguousarray(np.broadcast_to(np.asarray(g["mu_s"], dtype=np.float64), (nb,)).copy())
        nc = (C.c_int * 3)(*[int(x) for x in g["n_cells"]])
        per = (C.c_int * 3)(*[int(bool(x)) for x in g["periodic"]])
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        self._check(L.sp_set_geometry(self._h, dp(brav), nb, dp(basis.reshape(-1)), nc, per,
                                      float(g.get("lattice_constant", 1.0)), dp(mu)))
        h = hamiltonian
        H = Hamiltonian()
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
        self._pairs = (Pair * max(1, len(pairs)))()
        for q, (i, j, d, Jp, Dp) in enumerate(pairs):
            self._pairs[q].i, self._pairs[q].j, self._pairs[q].J = int(i), int(j), float(Jp)
            for k in range(3):
                self._pairs[q].d[k] = int(d[k])
                self._pairs[q].D[k] = float(Dp[k])
        H.n_pairs = len(pairs)
        H.pairs = C.cast(self._pairs, C.POINTER(Pair))
        self._check(L.sp_set_hamiltonian(self._h, C.byref(H)))
        n = C.c_int()
        self._check(L.sp_n_spins(self._h, C.byref(n)))
        self.N = n.value

    def _check(self, rc):
        if rc:
            raise SpinError(rc, lib().sp_last_error(self._h).decode())

    def sync_status(self):
        """Wait for the device and return (code, message) of the context's
        status word, cleared (code 0 when nothing was flagged)."""
        rc = lib().sp_sync_status(self._h)
        return rc, (lib().sp_last_error(self._h).decode() if rc else "")

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.sp_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    # ------------------------------------------------------------ buffers
    def spins(self, arr, device="cuda"):
        """(N, 3) or (M, N, 3) array -> contiguous 4-wide device tensor."""
        a = torch.as_tensor(np.asarray(arr, dtype=np.float64))
        out = torch.zeros(a.shape[:-1] + (4,), dtype=self.dtype)
        out[..., :3] = a[..., :3].to(self.dtype)
        return out.to(device)

    def _spin_arg(self, t, name, images=None):
        shape = (self.N, 4) if images is None else (images, self.N, 4)
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == self.dtype and tuple(t.shape) == shape
                and t.is_contiguous()):
            raise ValueError("%s must be a contiguous CUDA %s tensor of shape %s" % (name, self.dtype, shape))
        return _ptr(t)

    # ------------------------------------------------------------ calls
    def effective_field(self, n, out=None):
        out = torch.empty_like(n) if out is None else out
        self._check(lib().sp_effective_field(self._h, self._spin_arg(n, "n"), self._spin_arg(out, "out"), _stream()))
        return out

    def gradient(self, n, out=None):
        out = torch.empty_like(n) if out is None else out
        self._check(lib().sp_gradient(self._h, self._spin_arg(n, "n"), self._spin_arg(out, "out"), _stream()))
        return out

    def energy(self, n, out=None):
        """Device tensor of 6 doubles: total, Zeeman, anisotropy, exchange, DMI, dipole (meV)."""
        out = torch.empty(6, dtype=torch.float64, device=n.device) if out is None else out
        self._check(lib().sp_energy(self._h, self._spin_arg(n, "n"), _ptr(out), _stream()))
        return out

    def max_torque(self, n, out=None):
        out = torch.empty(1, dtype=torch.float64, device=n.device) if out is None else out
        self._check(lib().sp_max_torque(self._h, self._spin_arg(n, "n"), _ptr(out), _stream()))
        return out

    def gneb_path(self, chain, n_interp=10, charge=False):
        """Per image (r, E, dE/dr[, Q]) and the cubic interpolation (r_i, E_i), as numpy arrays."""
        M = chain.shape[0]
        r, E, sl = (np.zeros(M) for _ in range(3))
        Q = np.zeros(M) if charge else None
        ri, Ei = np.zeros((M - 1) * n_interp + 1), np.zeros((M - 1) * n_interp + 1)
        dp = lambda a: a.ctypes.data_as(C.c_void_p) if a is not None else None  # noqa: E731
        self._check(lib().sp_gneb_path(self._h, self._spin_arg(chain, "chain", M), M, int(n_interp), dp(r), dp(E),
                                       dp(sl), dp(Q), dp(ri), dp(Ei), _stream()))
        out = dict(r=r, E=E, slope=sl, r_interp=ri, E_interp=Ei)
        if charge:
            out["Q"] = Q
        return out

    def hessian_apply(self, n, v, out=None):
        out = torch.empty_like(n) if out is None else out
        self._check(lib().sp_hessian_apply(self._h, self._spin_arg(n, "n"), self._spin_arg(v, "v"),
                                           self._spin_arg(out, "out"), _stream()))
        return out

    def lowest_mode(self, n, mode=None, krylov=64):
        """(lowest eigenvalue, unit mode [N, 4]); `mode` (updated in place) is the start vector."""
        mode = torch.zeros_like(n) if mode is None else mode
        lam = C.c_double()
        self._check(lib().sp_lowest_mode(self._h, self._spin_arg(n, "n"), self._spin_arg(mode, "mode"), int(krylov),
                                         C.byref(lam), _stream()))
        return lam.value, mode

    def hessian_spectrum(self, n):
        """All 2N eigenvalues of the covariant Hessian at n (FP64 contexts), ascending."""
        eig = np.zeros(2 * self.N)
        self._check(lib().sp_hessian_spectrum(self._h, self._spin_arg(n, "n"), eig.ctypes.data_as(C.c_void_p),
                                              _stream()))
        return eig

    def htst(self, n_min, n_sad, zero_tol=1e-6, V_min=1.0, V_sad=1.0):
        """HTST rate prefactor of the transition n_min -> over n_sad, as a dict."""
        p = HTSTParams(float(zero_tol), float(V_min), float(V_sad))
        r = HTSTResult()
        self._check(lib().sp_htst(self._h, self._spin_arg(n_min, "n_min"), self._spin_arg(n_sad, "n_sad"),
                                  C.byref(p), C.byref(r), _stream()))
        return {name: getattr(r, name) for name, _ in HTSTResult._fields_}

    def mmf(self, n, vel, mode, n_iter, dt=0.1, mass=1.0, krylov=64):
        """Minimum mode following in place; returns (max |F|, lowest eigenvalue)."""
        p = MMFParams(float(dt), float(mass), int(krylov))
        mf, lam = C.c_double(), C.c_double()
        self._check(lib().sp_mmf(self._h, self._spin_arg(n, "n"), self._spin_arg(vel, "vel"),
                                 self._spin_arg(mode, "mode"), C.byref(p), int(n_iter), C.byref(mf), C.byref(lam),
                                 _stream()))
        return mf.value, lam.value

    def mc_colours(self):
        n = C.c_int()
        self._check(lib().sp_mc_colours(self._h, C.byref(n)))
        return n.value

    def mc_sweeps(self, spins, T, n_sweeps, seed=0, sweep0=0, target_accept=0.5, sample=True, cone=None, stats=None):
        """Metropolis sweeps of replicas spins [R, N, 4] (CUDA, this context's
        dtype) at temperatures T[R]; cone [R] and stats [R, 8] are float64
        CUDA tensors, updated in place (created when None).  Returns (cone, stats)."""
        R = spins.shape[0]
        if spins.dim() != 3 or spins.shape[1] != self.N:
            raise ValueError("spins must be [replicas, N, 4]")
        self._spin_arg(spins, "spins", R)
        cone = torch.full((R,), 0.5, dtype=torch.float64, device=spins.device) if cone is None else cone
        stats = torch.zeros((R, 8), dtype=torch.float64, device=spins.device) if stats is None else stats
        Th = (C.c_double * R)(*[float(t) for t in T])
        p = MCParams(int(seed), int(sweep0), float(target_accept), int(bool(sample)))
        self._check(lib().sp_mc_sweeps(self._h, _ptr(spins), R, Th, C.byref(p), int(n_sweeps), _ptr(cone), _ptr(stats),
                                       _stream()))
        return cone, stats

    def topological_charge(self, n, out=None):
        out = torch.empty(1, dtype=torch.float64, device=n.device) if out is None else out
        self._check(lib().sp_topological_charge(self._h, self._spin_arg(n, "n"), _ptr(out), _stream()))
        return out

    def llg_step(self, n, n_steps=1, solver="depondt", dt=1e-3, alpha=0.1, T=0.0, seed=0, step0=0, replica=0):
        p = LLGParams(SOLVER[solver], float(dt), float(alpha), float(T), int(seed), int(step0), int(replica))
        self._check(lib().sp_llg_step(self._h, self._spin_arg(n, "n"), C.byref(p), int(n_steps), _stream()))
        return n

    def llg_step_replicas(self, spins, T, n_steps=1, solver="heun", dt=1e-3, alpha=0.1, seed=0, step0=0, replica=0):
        """LLG steps of replicas spins [R, N, 4] (CUDA, this context's dtype)
        at temperatures T[R], replica r on the thermal stream replica + r."""
        R = spins.shape[0]
        if spins.dim() != 3 or spins.shape[1] != self.N:
            raise ValueError("spins must be [replicas, N, 4]")
        self._spin_arg(spins, "spins", R)
        if len(T) != R:
            raise ValueError("one temperature per replica")
        Th = (C.c_double * R)(*[float(t) for t in T])
        p = LLGParams(SOLVER[solver], float(dt), float(alpha), 0.0, int(seed), int(step0), int(replica))
        self._check(lib().sp_llg_step_replicas(self._h, _ptr(spins), R, Th, C.byref(p), int(n_steps), _stream()))
        return spins

    def sample(self, spins, stats=None):
        """Accumulate per-replica observables of spins [R, N, 4] into stats
        [R, 8] (float64 CUDA, created when None): sums of m, m^2, m^4, E, E^2
        and the sample count."""
        R = spins.shape[0]
        if spins.dim() != 3 or spins.shape[1] != self.N:
            raise ValueError("spins must be [replicas, N, 4]")
        self._spin_arg(spins, "spins", R)
        stats = torch.zeros((R, 8), dtype=torch.float64, device=spins.device) if stats is None else stats
        if not (stats.is_cuda and stats.dtype == torch.float64 and tuple(stats.shape) == (R, 8) and stats.is_contiguous()):
            raise ValueError("stats must be a contiguous float64 CUDA tensor [R, 8]")
        self._check(lib().sp_sample(self._h, _ptr(spins), R, _ptr(stats), _stream()))
        return stats

    def minimise(self, n, v, dt=0.1, mass=1.0, tol=1e-6, max_iter=10000, check_every=64):
        it = C.c_int()
        mt = C.c_double()
        self._check(lib().sp_minimise(self._h, self._spin_arg(n, "n"), self._spin_arg(v, "v"), float(dt), float(mass),
                                      float(tol), int(max_iter), int(check_every), C.byref(it), C.byref(mt),
                                      _stream()))
        return it.value, mt.value

    def set_option(self, name, value):
        self._check(lib().sp_set_option(self._h, OPTIONS[name], int(value)))

    def get_option(self, name):
        v = C.c_int()
        self._check(lib().sp_get_option(self._h, OPTIONS[name], C.byref(v)))
        return v.value

    def autotune(self, n):
        """Pick the planes-per-CTA of the 27-point path by timing (spins unchanged)."""
        v = C.c_int()
        self._check(lib().sp_autotune(self._h, self._spin_arg(n, "n"), C.byref(v), _stream()))
        return v.value

    def profile(self, on=True):
        self._check(lib().sp_profile_enable(self._h, int(bool(on))))

    def profile_read(self, kind):
        """(summed device ms, launches) of a kernel class since the last read."""
        ms, n = C.c_double(), C.c_longlong()
        self._check(lib().sp_profile_read(self._h, PROFILE_KINDS[kind], C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def gneb_step(self, chain, vel, n_iter=1, k_spring=1.0, climbing=True, dt=0.1, mass=1.0, energies=None,
                  max_force=None, image_types=None, energy_weight=0.0):
        M = chain.shape[0]
        E = torch.empty(M, dtype=torch.float64, device=chain.device) if energies is None else energies
        F = torch.empty(1, dtype=torch.float64, device=chain.device) if max_force is None else max_force
        p, _keep = gneb_params(dt, mass, k_spring, climbing, image_types, energy_weight)
        self._check(lib().sp_gneb_step(self._h, self._spin_arg(chain, "chain", M), self._spin_arg(vel, "vel", M), M,
                                       C.byref(p), int(n_iter), _ptr(E), _ptr(F), _stream()))
        return E, F


def gneb_batch_step(ctxs, chains, vel, offsets, n_images, n_iter=1, k_spring=1.0, climbing=True, dt=0.1, mass=1.0,
                    energies=None, max_force=None, image_types=None, energy_weight=0.0):
    """Step many chains (one context each) together; `chains` and `vel` are
    one flat CUDA tensor of 4-wide records each, chain c starting at record
    offsets[c].  Returns (energies, max_force) device tensors."""
    L = lib()
    n = len(ctxs)
    dtype = ctxs[0].dtype
    for t, name in ((chains, "chains"), (vel, "vel")):
        if not (t.is_cuda and t.dtype == dtype and t.is_contiguous() and t.shape[-1] == 4):
            raise ValueError("%s must be a contiguous CUDA %s tensor of 4-wide records" % (name, dtype))
    E = torch.empty(int(sum(n_images)), dtype=torch.float64, device=chains.device) if energies is None else energies
    F = torch.empty(n, dtype=torch.float64, device=chains.device) if max_force is None else max_force
    handles = (C.c_void_p * n)(*[c._h for c in ctxs])
    offs = (C.c_longlong * n)(*[int(x) for x in offsets])
    ims = (C.c_int * n)(*[int(x) for x in n_images])
    p, _keep = gneb_params(dt, mass, k_spring, climbing, image_types, energy_weight)
    rc = L.sp_gneb_batch_step(handles, n, _ptr(chains), _ptr(vel), offs, ims, C.byref(p), int(n_iter), _ptr(E),
                              _ptr(F), _stream())
    if rc:
        raise SpinError(rc, L.sp_last_error(ctxs[0]._h).decode())
    return E, F


def llg_step_batch(ctxs, spins, offsets, T, n_steps=1, solver="heun", dt=1e-3, alpha=0.1, seed=0, step0=0,
                   replica=0):
    """LLG steps of many systems of different lattices (one context each)
    together; `spins` is one flat CUDA tensor of 4-wide records, system k
    starting at record offsets[k], at temperature T[k] on the thermal stream
    replica + k."""
    L = lib()
    n = len(ctxs)
    dtype = ctxs[0].dtype
    if not (spins.is_cuda and spins.dtype == dtype and spins.is_contiguous() and spins.shape[-1] == 4):
        raise ValueError("spins must be a contiguous CUDA %s tensor of 4-wide records" % dtype)
    if len(T) != n or len(offsets) != n:
        raise ValueError("one offset and one temperature per system")
    handles = (C.c_void_p * n)(*[c._h for c in ctxs])
    offs = (C.c_longlong * n)(*[int(x) for x in offsets])
    Th = (C.c_double * n)(*[float(t) for t in T])
    p = LLGParams(SOLVER[solver], float(dt), float(alpha), 0.0, int(seed), int(step0), int(replica))
    rc = L.sp_llg_step_batch(handles, n, _ptr(spins), offs, Th, C.byref(p), int(n_steps), _stream())
    if rc:
        raise SpinError(rc, L.sp_last_error(ctxs[0]._h).decode())
    return spins


def gneb_batch_autotune(ctxs, chains, vel, offsets, n_images, n_trial=16, k_spring=1.0, climbing=True, dt=0.1,
                        mass=1.0, image_types=None, energy_weight=0.0):
    """Time the batch with one launch per pass and with the persistent kernel
    (on copies; the tensors are not changed) and keep the faster on
    ctxs[0].  Returns (persistent, ms_per_pass, ms_persistent)."""
    L = lib()
    n = len(ctxs)
    handles = (C.c_void_p * n)(*[c._h for c in ctxs])
    offs = (C.c_longlong * n)(*[int(x) for x in offsets])
    ims = (C.c_int * n)(*[int(x) for x in n_images])
    p, _keep = gneb_params(dt, mass, k_spring, climbing, image_types, energy_weight)
    choice = C.c_int()
    ms = (C.c_double * 2)()
    rc = L.sp_gneb_batch_autotune(handles, n, _ptr(chains), _ptr(vel), offs, ims, C.byref(p), int(n_trial),
                                  C.byref(choice), ms, _stream())
    if rc:
        raise SpinError(rc, L.sp_last_error(ctxs[0]._h).decode())
    return choice.value, ms[0], ms[1]


def minimise_batch(ctxs, spins, vel, offsets, dt=0.1, mass=1.0, tol=1e-6, max_iter=10000, check_every=64):
    """Relax many systems (one context each) together; `spins` and `vel` are
    one flat CUDA tensor of 4-wide records each.  Returns (iters, max_torque)
    as numpy arrays."""
    L = lib()
    n = len(ctxs)
    dtype = ctxs[0].dtype
    for t, name in ((spins, "spins"), (vel, "vel")):
        if not (t.is_cuda and t.dtype == dtype and t.is_contiguous() and t.shape[-1] == 4):
            raise ValueError("%s must be a contiguous CUDA %s tensor of 4-wide records" % (name, dtype))
    handles = (C.c_void_p * n)(*[c._h for c in ctxs])
    offs = (C.c_longlong * n)(*[int(x) for x in offsets])
    it = (C.c_int * n)()
    mt = (C.c_double * n)()
    rc = L.sp_minimise_batch(handles, n, _ptr(spins), _ptr(vel), offs, float(dt), float(mass), float(tol),
                             int(max_iter), int(check_every), it, mt, _stream())
    if rc:
        raise SpinError(rc, L.sp_last_error(ctxs[0]._h).decode())
    return np.array(it[:], dtype=np.int64), np.array(mt[:])
