"""Python binding of libparo.so (include/paro.h): argument marshalling only.

Every numerical step runs in the library's CUDA kernels; this module only converts NumPy / torch
arguments to pointers and sizes. Device arrays are torch CUDA tensors (complex128 / complex64 are
interleaved (re, im), the layout the C ABI expects). Work is enqueued on torch's current CUDA stream,
so library calls and torch operations stay ordered. There is no CPU fallback: without a CUDA device
or without the built library every entry point raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libparo.so")

PARO_OK, PARO_ERR_ARG, PARO_ERR_CUDA, PARO_ERR_BREAKDOWN, PARO_ERR_NOT_CONVERGED, PARO_ERR_STATE = 0, -1, -2, -3, -4, -6
PARO_FP64, PARO_MIXED = 0, 1
PARO_C64, PARO_C32 = 0, 1
PARO_ALG1, PARO_ALG2, PARO_ALG3 = 1, 2, 3
PARO_VNL_ACCURATE, PARO_VNL_TENSOR = 0, 1
ENERGY_TERMS = ("kinetic", "nonlocal", "local", "hartree", "xc", "ewald", "total")

# Every symbol include/paro.h declares.
EXPORTS = (
    "paro_create", "paro_set_local_pp", "paro_set_kb", "paro_set_positions", "paro_set_veff", "paro_set_veff_rest",
    "paro_get_veff",
    "paro_get_vloc", "paro_set_density", "paro_set_ecut", "paro_set_gamma_real", "paro_set_smearing", "paro_get_occupations", "paro_grid", "paro_npw", "paro_miller", "paro_sigma", "paro_apply_h",
    "paro_apply_h_noalloc", "paro_apply_vnl", "paro_apply_h_adjoint", "paro_orthonormalize", "paro_solve_source", "paro_batch_create", "paro_batch_apply_h",
    "paro_batch_step", "paro_batch_info", "paro_batch_tuning", "paro_batch_destroy",
    "paro_set_orbitals", "paro_get_orbitals", "paro_get_eigenvalues", "paro_get_residuals", "paro_step",
    "paro_eigh", "paro_density", "paro_energy", "paro_scf_step", "paro_scf", "paro_set_state", "paro_profile",
    "paro_profile_read", "paro_profile_names", "paro_launch_count", "paro_last_error", "paro_destroy",
)

_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_dbl_p = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


class ScfOpts(ctypes.Structure):
    _fields_ = [("alg", ctypes.c_int), ("tol_per_atom", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("inner_rel_tol", ctypes.c_double), ("inner_max_it", ctypes.c_int), ("pulay_depth", ctypes.c_int),
                ("pulay_beta", ctypes.c_double)]


class ScfResult(ctypes.Structure):
    _fields_ = [("n_iter", ctypes.c_int), ("converged", ctypes.c_int), ("energy", ctypes.c_double * 7),
                ("max_resid", ctypes.c_double)]


_SIGS = {
    "paro_create": (ctypes.c_int, [ctypes.POINTER(_vp), _c_dbl_p, ctypes.c_int, _c_dbl_p,
                                   ctypes.c_double, ctypes.c_int, _c_dbl_p, _c_dbl_p, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, _vp]),
    "paro_set_local_pp": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "paro_set_kb": (ctypes.c_int, [_vp, ctypes.c_double, _c_dbl_p]),
    "paro_set_veff": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "paro_set_veff_rest": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "paro_get_veff": (ctypes.c_int, [_vp, _c_dbl_p]),
    "paro_set_density": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "paro_set_smearing": (ctypes.c_int, [_vp, ctypes.c_double]),
    "paro_set_ecut": (ctypes.c_int, [_vp, ctypes.c_double]),
    "paro_set_gamma_real": (ctypes.c_int, [_vp, ctypes.c_int]),
    "paro_get_occupations": (ctypes.c_int, [_vp, _c_dbl_p, _c_dbl_p, _c_dbl_p]),
    "paro_grid": (ctypes.c_int, [_vp, _c_int_p]),
    "paro_npw": (ctypes.c_int, [_vp, ctypes.c_int, _c_int_p]),
    "paro_miller": (ctypes.c_int, [_vp, ctypes.c_int, _c_int_p]),
    "paro_sigma": (ctypes.c_int, [_vp, _c_dbl_p]),
    "paro_apply_h": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "paro_apply_h_noalloc": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "paro_apply_vnl": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_int]),
    "paro_apply_h_adjoint": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp,
                                            _vp]),
    "paro_set_positions": (ctypes.c_int, [_vp, _c_dbl_p]),
    "paro_orthonormalize": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "paro_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int]),
    "paro_batch_apply_h": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
    "paro_batch_step": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int, _c_dbl_p]),
    "paro_batch_info": (ctypes.c_int, [_vp, _c_int_p, _c_int_p, _c_int_p, _c_int_p,
                                       ctypes.POINTER(ctypes.c_longlong)]),
    "paro_batch_tuning": (ctypes.c_int, [_vp, ctypes.c_int, _c_int_p, _c_dbl_p]),
    "paro_batch_destroy": (None, [_vp]),
    "paro_get_vloc": (ctypes.c_int, [_vp, _c_dbl_p]),
    "paro_solve_source": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _c_dbl_p, _vp, _vp,
                                         ctypes.c_double, ctypes.c_int, _c_int_p]),
    "paro_set_orbitals": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int]),
    "paro_get_orbitals": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int]),
    "paro_get_eigenvalues": (ctypes.c_int, [_vp, _c_dbl_p]),
    "paro_get_residuals": (ctypes.c_int, [_vp, _c_dbl_p]),
    "paro_step": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, _c_dbl_p]),
    "paro_eigh": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
    "paro_density": (ctypes.c_int, [_vp, _vp]),
    "paro_energy": (ctypes.c_int, [_vp, _c_dbl_p]),
    "paro_scf_step": (ctypes.c_int, [_vp, ctypes.POINTER(ScfOpts), _c_dbl_p, _c_dbl_p]),
    "paro_scf": (ctypes.c_int, [_vp, ctypes.POINTER(ScfOpts), ctypes.POINTER(ScfResult)]),
    "paro_set_state": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _c_dbl_p, ctypes.c_int]),
    "paro_profile": (ctypes.c_int, [_vp, ctypes.c_int]),
    "paro_profile_read": (ctypes.c_int, [_vp, ctypes.c_char_p, _c_int_p, _c_dbl_p]),
    "paro_profile_names": (ctypes.c_int, [_vp, ctypes.c_char_p, ctypes.c_int]),
    "paro_launch_count": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_longlong)]),
    "paro_last_error": (ctypes.c_char_p, [_vp]),
    "paro_destroy": (None, [_vp]),
}

_LIB = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libparo.so and declares every entry point; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -m paper_1702_04045_gb300.build`")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


class ParoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libparo status {status}: {msg}")
        self.status = status


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_c_dbl_p)


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(_c_int_p)


class ScfOptions:
    def __init__(self, alg=1, tol_per_atom=1e-8, max_iter=200, inner_rel_tol=0.25, inner_max_it=8, pulay_depth=8,
                 pulay_beta=0.7):
        self.s = ScfOpts(alg, tol_per_atom, max_iter, inner_rel_tol, inner_max_it, pulay_depth, pulay_beta)


class Context:
    """One libparo context: cell, basis per k-point, potentials and orbitals on the current CUDA device."""

    def __init__(self, lattice, pos, ecut, n_bands, n_occ, precision="fp64", kpts=None, kweights=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libparo needs a CUDA device; there is no CPU path")
        self.torch = torch
        self.lib = load_library()
        lat = np.ascontiguousarray(np.asarray(lattice, dtype=np.float64).reshape(9))
        p = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
        self.n_atoms = p.shape[0]
        if kpts is None:
            kp, nk = None, 1
        else:
            kp = np.ascontiguousarray(np.asarray(kpts, dtype=np.float64).reshape(-1, 3))
            nk = kp.shape[0]
        kw = None if kweights is None else np.ascontiguousarray(np.asarray(kweights, dtype=np.float64))
        self.prec = {"fp64": PARO_FP64, "mixed": PARO_MIXED}[precision]
        self.n_bands, self.n_occ, self.nk = int(n_bands), int(n_occ), nk
        h = _vp()
        stream = torch.cuda.current_stream().cuda_stream
        st = self.lib.paro_create(ctypes.byref(h), _dptr(lat), self.n_atoms, _dptr(p), float(ecut), nk,
                                  _dptr(kp) if kp is not None else None, _dptr(kw) if kw is not None else None,
                                  self.n_bands, self.n_occ, self.prec, _vp(stream))
        if st != 0:
            raise ParoError(st, self.lib.paro_last_error(None).decode())
        self.h = h
        self._keep = []

    # -- helpers ------------------------------------------------------------------------------
    def _check(self, st):
        if st != 0:
            raise ParoError(st, self.lib.paro_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.paro_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- setup --------------------------------------------------------------------------------
    def set_local_pp(self, Z, rc, A, a):
        self._check(self.lib.paro_set_local_pp(self.h, Z, rc, A, a))

    def set_kb(self, rc, D):
        d = np.ascontiguousarray(np.asarray(D, dtype=np.float64).reshape(-1))
        self._check(self.lib.paro_set_kb(self.h, rc, _dptr(d)))

    def set_veff(self, v):
        if hasattr(v, "is_cuda") and v.is_cuda:
            t = v.contiguous().to(self.torch.float64)
            self._check(self.lib.paro_set_veff(self.h, _vp(t.data_ptr()), 1))
        else:
            a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(-1))
            self._check(self.lib.paro_set_veff(self.h, _vp(a.ctypes.data), 0))

    def set_veff_rest(self, v_rest):
        """V_eff = V_loc(current positions) + v_rest, formed by the library (host array or CUDA tensor)."""
        if hasattr(v_rest, "is_cuda") and v_rest.is_cuda:
            t = v_rest.detach().contiguous().to(self.torch.float64)
            self._check(self.lib.paro_set_veff_rest(self.h, _vp(t.data_ptr()), 1))
        else:
            a = np.ascontiguousarray(np.asarray(v_rest, dtype=np.float64).reshape(-1))
            self._check(self.lib.paro_set_veff_rest(self.h, _vp(a.ctypes.data), 0))

    def get_veff(self):
        out = np.empty(self.grid, dtype=np.float64)
        self._check(self.lib.paro_get_veff(self.h, _dptr(out)))
        return out

    def set_density(self, rho):
        """Input density of the SCF (host array or CUDA tensor, the grid's shape, electrons / Bohr^3)."""
        if hasattr(rho, "is_cuda") and rho.is_cuda:
            t = rho.detach().contiguous().to(self.torch.float64)
            self._check(self.lib.paro_set_density(self.h, _vp(t.data_ptr()), 1))
        else:
            a = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(-1))
            self._check(self.lib.paro_set_density(self.h, _vp(a.ctypes.data), 0))

    def set_ecut(self, ecut):
        """One step of the cutoff ladder (Algorithm 1 step 2): the basis and grid of the larger cutoff, the
        orbitals embedded in it."""
        self._check(self.lib.paro_set_ecut(self.h, float(ecut)))

    def set_gamma_real(self, enable=True):
        """Gamma-point real-wavefunction mode: two real orbitals per complex H application and density
        transform in the ParO iteration (k = 0 contexts only)."""
        self._check(self.lib.paro_set_gamma_real(self.h, 1 if enable else 0))

    def set_smearing(self, kT):
        """Fermi-Dirac occupations of width kT (Ha); 0 restores integer occupations of the n_occ lowest bands."""
        self._check(self.lib.paro_set_smearing(self.h, float(kT)))

    def occupations(self):
        """(f of shape (n_k, n_bands), mu, -T S) of the current orbitals."""
        f = np.empty((self.nk, self.n_bands), dtype=np.float64)
        mu, mts = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.paro_get_occupations(self.h, _dptr(f), ctypes.byref(mu), ctypes.byref(mts)))
        return f, mu.value, mts.value

    @property
    def grid(self):
        n = np.zeros(3, dtype=np.int32)
        self._check(self.lib.paro_grid(self.h, _iptr(n)))
        return tuple(int(x) for x in n)

    def npw(self, ik=0):
        n = ctypes.c_int()
        self._check(self.lib.paro_npw(self.h, ik, ctypes.byref(n)))
        return n.value

    def miller(self, ik=0):
        out = np.zeros((self.npw(ik), 3), dtype=np.int32)
        self._check(self.lib.paro_miller(self.h, ik, _iptr(out)))
        return out

    def sigma(self):
        s = ctypes.c_double()
        self._check(self.lib.paro_sigma(self.h, ctypes.byref(s)))
        return s.value

    # -- H psi and source problems --------------------------------------------------------------
    def apply_h(self, psi, ik=0, out=None):
        torch = self.torch
        dt = PARO_C64 if psi.dtype == torch.complex128 else PARO_C32
        psi = psi.contiguous()
        nb = psi.shape[0]
        if out is None:
            out = torch.empty_like(psi)
        self._check(self.lib.paro_apply_h(self.h, ik, nb, dt, _vp(psi.data_ptr()), _vp(out.data_ptr())))
        return out

    def apply_h_noalloc(self, psi, out, ik=0):
        """H psi into a caller-provided output through the library's allocation-free entry point.
        psi and out: CUDA tensors of the same shape (nb, npw(ik)) and dtype (complex128 or complex64);
        out must be contiguous (it is written in place)."""
        torch = self.torch
        if psi.dtype not in (torch.complex128, torch.complex64):
            raise ParoError(PARO_ERR_ARG, "apply_h_noalloc: psi must be complex128 or complex64")
        if psi.dim() != 2 or psi.shape[1] != self.npw(ik):
            raise ParoError(PARO_ERR_ARG, f"apply_h_noalloc: psi must have shape (nb, {self.npw(ik)})")
        if (not (psi.is_cuda and out.is_cuda) or out.dtype != psi.dtype or tuple(out.shape) != tuple(psi.shape)
                or not out.is_contiguous() or out.device != psi.device):
            raise ParoError(PARO_ERR_ARG, "apply_h_noalloc: out must be a contiguous CUDA tensor of psi's shape, "
                                          "dtype and device")
        dt = PARO_C64 if psi.dtype == torch.complex128 else PARO_C32
        psi = psi.contiguous()
        self._check(self.lib.paro_apply_h_noalloc(self.h, ik, psi.shape[0], dt, _vp(psi.data_ptr()),
                                                  _vp(out.data_ptr())))
        return out

    def apply_vnl(self, psi, form=PARO_VNL_ACCURATE, ik=0):
        """The nonlocal term V_nl psi alone (device tensor of psi's shape and dtype); form PARO_VNL_TENSOR
        (complex64 only) is the tensor-core product of the inner solves."""
        torch = self.torch
        dt = PARO_C64 if psi.dtype == torch.complex128 else PARO_C32
        psi = psi.contiguous()
        out = torch.empty_like(psi)
        self._check(self.lib.paro_apply_vnl(self.h, ik, psi.shape[0], dt, _vp(psi.data_ptr()), _vp(out.data_ptr()),
                                            int(form)))
        return out

    def apply_h_adjoint(self, psi, w, ik=0, grads=("psi", "v", "pos")):
        """Vector-Jacobian product of Y = H Psi for cotangent W: (dL/dPsi, dL/dV_eff(r), dL/dR) as device
        tensors (None where not asked for); dL/dV has the grid's shape, dL/dR is (n_atoms, 3)."""
        torch = self.torch
        dt = PARO_C64 if psi.dtype == torch.complex128 else PARO_C32
        psi = psi.contiguous()
        w = w.to(psi.dtype).contiguous()
        dev = psi.device
        g_psi = torch.empty_like(psi) if "psi" in grads else None
        g_v = torch.empty(self.grid, dtype=torch.float64, device=dev) if "v" in grads else None
        g_pos = torch.empty((self.n_atoms, 3), dtype=torch.float64, device=dev) if "pos" in grads else None

        def p(t):
            return _vp(t.data_ptr()) if t is not None else None

        self._check(self.lib.paro_apply_h_adjoint(self.h, ik, psi.shape[0], dt, p(psi), p(w), p(g_psi), p(g_v),
                                                  p(g_pos)))
        return g_psi, g_v, g_pos

    def set_positions(self, pos):
        pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1))
        if pos.size != 3 * self.n_atoms:
            raise ValueError("positions must be n_atoms x 3")
        self._check(self.lib.paro_set_positions(self.h, _dptr(pos)))

    def get_vloc(self):
        v = np.empty(self.grid, dtype=np.float64)
        self._check(self.lib.paro_get_vloc(self.h, _dptr(v)))
        return v

    def orthonormalize(self, x, ik=0, out=None):
        """Rows x -> orthonormal rows spanning the same nested subspaces (Cholesky of the Gram matrix);
        out may be x itself (in place)."""
        torch = self.torch
        dt = PARO_C64 if x.dtype == torch.complex128 else PARO_C32
        x = x.contiguous()
        if out is None:
            out = torch.empty_like(x)
        self._check(self.lib.paro_orthonormalize(self.h, ik, x.shape[0], dt, _vp(x.data_ptr()),
                                                 _vp(out.data_ptr())))
        return out

    def solve_source(self, eps, psi, rel_tol, max_it, ik=0):
        torch = self.torch
        dt = PARO_C64 if psi.dtype == torch.complex128 else PARO_C32
        psi = psi.contiguous()
        nb = psi.shape[0]
        e = np.ascontiguousarray(np.asarray(eps, dtype=np.float64))
        x = torch.empty_like(psi)
        its = np.zeros(nb, dtype=np.int32)
        self._check(self.lib.paro_solve_source(self.h, ik, nb, dt, _dptr(e), _vp(psi.data_ptr()), _vp(x.data_ptr()),
                                               float(rel_tol), int(max_it), _iptr(its)))
        return x, its

    # -- orbitals and the ParO iteration --------------------------------------------------------
    def set_orbitals(self, psi, ik=0):
        if hasattr(psi, "is_cuda") and psi.is_cuda:
            t = psi.contiguous().to(self.torch.complex128)
            self._check(self.lib.paro_set_orbitals(self.h, ik, _vp(t.data_ptr()), 1))
        else:
            a = np.ascontiguousarray(np.asarray(psi, dtype=np.complex128))
            self._check(self.lib.paro_set_orbitals(self.h, ik, _vp(a.ctypes.data), 0))

    def get_orbitals(self, ik=0, device=False):
        if device:
            out = self.torch.empty((self.n_bands, self.npw(ik)), dtype=self.torch.complex128, device="cuda")
            self._check(self.lib.paro_get_orbitals(self.h, ik, _vp(out.data_ptr()), 1))
            return out
        out = np.empty((self.n_bands, self.npw(ik)), dtype=np.complex128)
        self._check(self.lib.paro_get_orbitals(self.h, ik, _vp(out.ctypes.data), 0))
        return out

    def eigenvalues(self):
        out = np.empty((self.nk, self.n_bands), dtype=np.float64)
        self._check(self.lib.paro_get_eigenvalues(self.h, _dptr(out)))
        return out

    def residuals(self):
        out = np.empty((self.nk, self.n_bands), dtype=np.float64)
        self._check(self.lib.paro_get_residuals(self.h, _dptr(out)))
        return out

    def step(self, alg=1, rel_tol=0.25, max_it=8):
        r = ctypes.c_double()
        self._check(self.lib.paro_step(self.h, alg, float(rel_tol), int(max_it), ctypes.byref(r)))
        return r.value

    def eigh(self, a):
        torch = self.torch
        a = a.contiguous().to(torch.complex128)
        n = a.shape[0]
        w = torch.empty(n, dtype=torch.float64, device=a.device)
        v = torch.empty_like(a)
        self._check(self.lib.paro_eigh(self.h, n, _vp(a.data_ptr()), _vp(w.data_ptr()), _vp(v.data_ptr())))
        return w, v

    def density(self):
        out = self.torch.empty(self.grid, dtype=self.torch.float64, device="cuda")
        self._check(self.lib.paro_density(self.h, _vp(out.data_ptr())))
        return out

    def energy(self):
        t = np.zeros(7)
        self._check(self.lib.paro_energy(self.h, _dptr(t)))
        return dict(zip(ENERGY_TERMS, t.tolist()))

    def scf_step(self, opts: ScfOptions | None = None):
        o = (opts or ScfOptions()).s
        t = np.zeros(7)
        r = ctypes.c_double()
        self._check(self.lib.paro_scf_step(self.h, ctypes.byref(o), _dptr(t), ctypes.byref(r)))
        return dict(zip(ENERGY_TERMS, t.tolist())), r.value

    def set_state(self, psi, eps, ik=0):
        """Restore orthonormal orbitals and their Ritz values verbatim (host array or CUDA tensor)."""
        e = np.ascontiguousarray(np.asarray(eps, dtype=np.float64))
        if hasattr(psi, "is_cuda") and psi.is_cuda:
            self._check(self.lib.paro_set_state(self.h, ik, _vp(psi.data_ptr()), _dptr(e), 1))
        else:
            a = np.ascontiguousarray(np.asarray(psi, dtype=np.complex128))
            self._check(self.lib.paro_set_state(self.h, ik, _vp(a.ctypes.data), _dptr(e), 0))

    def profile(self, enable=True):
        self._check(self.lib.paro_profile(self.h, 1 if enable else 0))

    def profile_read(self, name="*"):
        n = ctypes.c_int()
        t = ctypes.c_double()
        self._check(self.lib.paro_profile_read(self.h, name.encode(), ctypes.byref(n), ctypes.byref(t)))
        return n.value, t.value

    def profile_names(self):
        buf = ctypes.create_string_buffer(4096)
        self._check(self.lib.paro_profile_names(self.h, buf, 4096))
        return [s for s in buf.value.decode().split(",") if s]

    def launch_count(self):
        n = ctypes.c_longlong()
        self._check(self.lib.paro_launch_count(self.h, ctypes.byref(n)))
        return n.value

    def scf(self, opts: ScfOptions | None = None):
        o = (opts or ScfOptions()).s
        res = ScfResult()
        st = self.lib.paro_scf(self.h, ctypes.byref(o), ctypes.byref(res))
        out = dict(n_iter=res.n_iter, converged=bool(res.converged),
                   energy=dict(zip(ENERGY_TERMS, list(res.energy))), max_resid=res.max_resid)
        if st != 0:
            err = ParoError(st, self.lib.paro_last_error(self.h).decode())
            err.result = out
            raise err
        return out


class Batch:
    """Batched ParO over the k-points of several contexts (uneven plane-wave counts and grids): one
    persistent H psi launch over all orbitals, one CUDA graph per ParO step."""

    def __init__(self, ctxs):
        self.ctxs = list(ctxs)
        self.lib = self.ctxs[0].lib
        arr = (_vp * len(self.ctxs))(*[c.h for c in self.ctxs])
        h = _vp()
        st = self.lib.paro_batch_create(ctypes.byref(h), arr, len(self.ctxs))
        if st != 0:
            raise ParoError(st, self.lib.paro_last_error(self.ctxs[0].h).decode())
        self.h = h
        self.problems = [(i, k) for i, c in enumerate(self.ctxs) for k in range(c.nk)]

    def _check(self, st):
        if st != 0:
            raise ParoError(st, self.lib.paro_last_error(self.ctxs[0].h).decode())

    def apply_h(self, psis):
        """H psi of every problem; psis: one device tensor (n_bands, npw) per problem, context-major."""
        torch = self.ctxs[0].torch
        psis = [p.contiguous() for p in psis]
        outs = [torch.empty_like(p) for p in psis]
        dt = PARO_C64 if psis[0].dtype == torch.complex128 else PARO_C32
        a = (_vp * len(psis))(*[_vp(p.data_ptr()) for p in psis])
        o = (_vp * len(outs))(*[_vp(p.data_ptr()) for p in outs])
        self._check(self.lib.paro_batch_apply_h(self.h, dt, a, o))
        return outs

    def step(self, rel_tol=0.25, max_it=8):
        r = ctypes.c_double()
        self._check(self.lib.paro_batch_step(self.h, float(rel_tol), int(max_it), ctypes.byref(r)))
        return r.value

    def info(self):
        v = [ctypes.c_int() for _ in range(4)]
        k = ctypes.c_longlong()
        self._check(self.lib.paro_batch_info(self.h, *[ctypes.byref(x) for x in v], ctypes.byref(k)))
        return dict(problems=v[0].value, items=v[1].value, launches_per_apply=v[2].value, grid=v[3].value,
                    kernels_per_step=k.value)

    def tuning(self):
        """The autotuner's table: rows (launches per apply, grid, sticks per unit, plane points per unit, ms)."""
        n = ctypes.c_int()
        self._check(self.lib.paro_batch_tuning(self.h, 0, ctypes.byref(n), None))
        rows = np.zeros((max(n.value, 1), 5))
        self._check(self.lib.paro_batch_tuning(self.h, n.value, ctypes.byref(n), _dptr(rows)))
        return rows[: n.value]

    def close(self):
        if self.h:
            self.lib.paro_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_HPSI_FN = None


def hpsi(ctx: Context, psi, v_rest, pos, ik=0):
    """Differentiable Y = H Psi with H built from V_eff = V_loc(pos) + v_rest and the KB projectors at
    pos (torch.autograd): the backward pass is the library's adjoint (dL/dPsi, dL/dv_rest, dL/dpos).
    psi: device complex (nb, npw); v_rest: float64 tensor of the grid's shape; pos: float64 (n_atoms, 3)."""
    global _HPSI_FN
    torch = ctx.torch
    if _HPSI_FN is None:
        class _HPsi(torch.autograd.Function):
            @staticmethod
            def forward(fctx, psi_, v_rest_, pos_, c, k):
                c.set_positions(pos_.detach().cpu().numpy())
                c.set_veff_rest(v_rest_)
                y = c.apply_h(psi_.detach(), ik=k)
                fctx.save_for_backward(psi_.detach())
                fctx.c, fctx.k = c, k
                return y

            @staticmethod
            def backward(fctx, gy):
                (psi_,) = fctx.saved_tensors
                g_psi, g_v, g_pos = fctx.c.apply_h_adjoint(psi_, gy, ik=fctx.k)
                return g_psi, g_v, g_pos, None, None

        _HPSI_FN = _HPsi
    return _HPSI_FN.apply(psi, v_rest, pos, ctx, ik)


def context_from_config(name: str, precision: str = "fp64", **kw) -> Context:
    """Context for a named synthetic workload of paper_1702_04045_gb300.inputs (pseudopotentials set)."""
    from . import inputs
    lat, pos, d, c = inputs.config_inputs(name)
    ctx = Context(lat, pos, c["ecut"], c["n_bands"], c["n_occ"], precision, **kw)
    ctx.set_local_pp(**inputs.LOCAL_PP)
    if d is not None:
        ctx.set_kb(inputs.KB_RC, d)
    if c.get("kT"):
        ctx.set_smearing(c["kT"])
    return ctx
