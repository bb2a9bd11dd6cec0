"""CPU FP64 oracle: the Gamma-point real-wavefunction trick (not in the paper; the standard companion of a
plane-wave method at k = 0).

TEST INFRASTRUCTURE ONLY (see oracle/pw.py). Plain NumPy in float64/complex128.

At k = 0 the local potential V_eff(r) and the Kleinman-Bylander projectors beta_j(r) are real, so H maps
real functions to real functions. A real orbital has coefficients with c(-G) = conj(c(G)). Two real
orbitals a, b are carried by one complex function phi = a + i b:
  * H phi = H a + i H b, and (H a)(G) = [y(G) + conj(y(-G))]/2, (H b)(G) = [y(G) - conj(y(-G))]/(2i) with
    y = H phi, so one complex H application serves two orbitals (half the FFT and projector work);
  * |phi(r)|^2 = a(r)^2 + b(r)^2, so one inverse transform gives the density of two orbitals (weights
    enter as sqrt(f) on each before packing);
  * Gram and Rayleigh-Ritz matrices of real orbitals are real symmetric: their imaginary parts are
    dropped, and the orbitals are kept real by taking the real part c(G) <- [c(G) + conj(c(-G))]/2.
An odd orbital count packs the last orbital with zero.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import paro, pw


def minus_g(basis: pw.Basis) -> np.ndarray:
    """Index of -G in the basis for every G (the Gamma-point sphere is symmetric)."""
    if np.any(basis.kfrac != 0):
        raise ValueError("the real-wavefunction trick needs k = 0")
    index = {tuple(m): i for i, m in enumerate(basis.miller.tolist())}
    return np.array([index[tuple(-x for x in m)] for m in basis.miller.tolist()], dtype=np.int64)


def real_part(basis: pw.Basis, c: np.ndarray) -> np.ndarray:
    """Coefficients of Re psi(r): [c(G) + conj(c(-G))]/2 for every row."""
    mg = minus_g(basis)
    return 0.5 * (c + np.conj(c[:, mg]))


def pack(c: np.ndarray) -> np.ndarray:
    """Rows (a0, b0, a1, b1, ...) -> a_j + i b_j; an odd last row is packed with zero."""
    nb = c.shape[0]
    out = c[0::2].astype(np.complex128).copy()
    out[: nb // 2] += 1j * c[1::2]
    return out


def unpack(basis: pw.Basis, y: np.ndarray, nb: int) -> np.ndarray:
    """Packed rows y_j = H(a_j + i b_j) -> rows H a_j, H b_j."""
    mg = minus_g(basis)
    yc = np.conj(y[:, mg])
    out = np.empty((nb, y.shape[1]), dtype=np.complex128)
    out[0::2] = 0.5 * (y + yc)[: (nb + 1) // 2]
    out[1::2] = (-0.5j * (y - yc))[: nb // 2]
    return out


def apply_h(basis: pw.Basis, v_r, psi, beta=None, dvec=None) -> np.ndarray:
    """H psi of real orbitals, two per complex application of pw.apply_h."""
    return unpack(basis, pw.apply_h(basis, v_r, pack(psi), beta, dvec), psi.shape[0])


def density_weighted(basis: pw.Basis, psi, occ, weight=1.0) -> np.ndarray:
    """sum_i occ_i psi_i(r)^2 * weight / Omega of real orbitals, two per inverse transform."""
    fr = pw.to_real_space(basis, pack(np.sqrt(np.asarray(occ))[:, None] * psi))
    return weight * np.sum(np.abs(fr) ** 2, axis=0) / basis.omega


class GammaProblem(paro.ParoProblem):
    """The fixed-potential problem at k = 0 with H applied two real orbitals at a time."""

    def h(self, psi):
        return apply_h(self.basis, self.v_r, psi, self.beta, self.dvec)


def cholesky_orthonormalize(basis, x):
    """Cholesky orthonormalisation of real rows with the real Gram matrix."""
    s = np.real(np.conj(x) @ x.T)
    s = 0.5 * (s + s.T)
    low = np.linalg.cholesky(s)
    return real_part(basis, sla.solve_triangular(low, x, lower=True))


def rayleigh_ritz(basis, y, hy):
    """Rayleigh-Ritz of real rows with the real symmetric H_sub (real eigenvectors)."""
    hsub = np.real(np.conj(y) @ hy.T)
    eps, c = np.linalg.eigh(0.5 * (hsub + hsub.T))
    return eps, real_part(basis, c.T @ y), real_part(basis, c.T @ hy)


def initial_state(prob: GammaProblem, c0):
    y = cholesky_orthonormalize(prob.basis, real_part(prob.basis, c0))
    return rayleigh_ritz(prob.basis, y, prob.h(y))


def paro_step_alg1(prob: GammaProblem, psi, eps, tol, max_it):
    """Algorithm 1 on real orbitals: the source solves (real operator and preconditioner keep them real),
    real Cholesky, real Rayleigh-Ritz."""
    x, its = paro.source_solve(prob, psi, eps, tol, max_it)
    y = cholesky_orthonormalize(prob.basis, real_part(prob.basis, x))
    eps1, psi1, hpsi1 = rayleigh_ritz(prob.basis, y, prob.h(y))
    return eps1, psi1, hpsi1, its
