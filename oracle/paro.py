"""CPU FP64 oracle: source problems and the ParO projection step (Algorithms 1 and 2).

TEST INFRASTRUCTURE ONLY (see oracle/pw.py). Plain NumPy/SciPy in float64/complex128.

Readings of points the paper leaves open:
  * Source problem of Algorithm 1, step 3: a(rho; psi^{n+1/2}, phi) = (eps_i psi_i, phi), i.e.
    H x = eps_i psi_i, which is singular or indefinite whenever H has a zero or negative
    eigenvalue. It is solved shifted: (H - sigma) x_i = (eps_i - sigma) psi_i with sigma a rigorous
    lower bound of the spectrum minus delta. The Rayleigh-Ritz step only sees span{x_i}, so the
    fixed point does not depend on sigma; sigma = 0 recovers the printed problem when H > 0.
  * Algorithm 2, step 3: H e_i = -(H psi_i - eps_i psi_i), solved as (H - sigma) e_i = -r_i.
  * The inner solver is preconditioned CG with diag(|k+G|^2/2 + mean V - sigma)^{-1}, started from
    x = psi_i (Algorithm 1) or e = 0 (Algorithm 2), stopped once its residual has dropped by a
    factor tol or after max_it steps (the paper only asks for the source problems to be solved).
  * Orthonormality (Algorithm 1 step 4) is imposed by Cholesky of the Gram matrix in band order.
  * Algorithm 3 (MParO II), step 3: the projected correction equation
    (I - P_i)(H - lambda_i)(I - P_i) e_i = (eps_i - H) psi_i, P_i = |psi_i><psi_i|, with lambda_i^n,
    which the paper never defines, read as eps_i^n. The operator is Hermitian and indefinite on the
    complement of psi_i, so it is solved there by preconditioned MINRES (Paige and Saunders), with
    the projected preconditioner (I - P_i) D (I - P_i), D the PCG preconditioner (positive definite on
    that complement), started at e = 0 and stopped like the PCG (residual estimate reduced by tol, or
    max_it steps). The Rayleigh-Ritz step then works as in Algorithm 2.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import pw


def sigma_shift(v_r: np.ndarray, beta=None, dstr=None, delta: float = 0.5) -> float:
    """sigma = sigma_LB - delta, sigma_LB a lower bound of the grid Hamiltonian's spectrum.

    T >= 0; psi^H V psi = N^{-1} sum_r V(r)|psi(r)|^2 >= min V (discrete Parseval); for an
    attractive channel D_{I,l} < 0,  D sum_j |beta_j><beta_j| >= D sum_j ||beta_j||^2
    >= D (2l+1) max_j ||beta_j||^2.
    """
    lb = float(np.min(v_r))
    if beta is not None:
        nat = dstr.shape[0]
        bn = np.sum(np.abs(beta) ** 2, axis=1).reshape(nat, 4)
        for i in range(nat):
            if dstr[i, 0] < 0:
                lb += dstr[i, 0] * bn[i, 0]
            if dstr[i, 1] < 0:
                lb += dstr[i, 1] * 3.0 * np.max(bn[i, 1:])
    return lb - delta


def pcg(apply_a, b, x0, precond, tol, max_it):
    """Preconditioned CG, one independent system per row of b (Hermitian positive definite A).

    Each row stops when ||r_i|| <= tol ||r_i^0|| (its initial residual; checked after every
    update) or after max_it iterations. Returns (x, iterations per row).
    """
    x = x0.astype(np.complex128).copy()
    r = b - apply_a(x)
    z = precond[None, :] * r
    p = z.copy()
    rz = np.real(np.sum(np.conj(r) * z, axis=1))
    r0norm = np.linalg.norm(r, axis=1)
    active = r0norm > 0.0
    its = np.zeros(b.shape[0], dtype=np.int64)
    for _ in range(max_it):
        if not np.any(active):
            break
        ap = apply_a(p)
        pap = np.real(np.sum(np.conj(p) * ap, axis=1))
        alpha = np.where(active, rz / np.where(active, pap, 1.0), 0.0)
        x = x + alpha[:, None] * p
        r = r - alpha[:, None] * ap
        its += active
        still = active & (np.linalg.norm(r, axis=1) > tol * r0norm)
        z = precond[None, :] * r
        rz_new = np.real(np.sum(np.conj(r) * z, axis=1))
        beta = np.where(still, rz_new / np.where(active, rz, 1.0), 0.0)
        p = np.where(still[:, None], z + beta[:, None] * p, p)
        rz = np.where(still, rz_new, rz)
        active = still
    return x, its


def cholesky_orthonormalize(x: np.ndarray) -> np.ndarray:
    """Rows x_i -> orthonormal rows spanning the same nested subspaces (Gram-Schmidt in band order).

    Column form: S = X^H X = L L^H, Y = X L^{-H}. With vectors as rows, y = conj(L)^{-1} x.
    """
    s = np.conj(x) @ x.T                             # S_ij = <x_i, x_j>
    s = 0.5 * (s + np.conj(s.T))
    low = np.linalg.cholesky(s)
    return sla.solve_triangular(np.conj(low), x, lower=True)


def rayleigh_ritz(y: np.ndarray, hy: np.ndarray):
    """Algorithm 1 step 4 on orthonormal rows y with hy = H y: H_sub = Y^H H Y, H_sub C = C diag(eps);
    returns (eps ascending, psi = rows of Y C, H psi = rows of (HY) C)."""
    hsub = np.conj(y) @ hy.T                         # (Y^H H Y)_ij = <y_i, H y_j>
    hsub = 0.5 * (hsub + np.conj(hsub.T))
    eps, c = np.linalg.eigh(hsub)
    return eps, c.T @ y, c.T @ hy


def residuals(psi: np.ndarray, hpsi: np.ndarray, eps: np.ndarray) -> np.ndarray:
    """||H psi_i - eps_i psi_i||_2 per band (Algorithm 1 step 5)."""
    return np.linalg.norm(hpsi - eps[:, None] * psi, axis=1)


class ParoProblem:
    """Fixed-potential eigenproblem for one k-point: basis, V_eff(r), optional KB projectors."""

    def __init__(self, basis: pw.Basis, v_r, beta=None, dstr=None, delta=0.5):
        self.basis = basis
        self.v_r = np.asarray(v_r, dtype=np.float64)
        self.beta = beta
        self.dstr = dstr
        self.dvec = pw.kb_dvec(dstr) if dstr is not None else None
        self.sigma = sigma_shift(self.v_r, beta, dstr, delta)
        self.precond = 1.0 / (basis.kin + float(np.mean(self.v_r)) - self.sigma)

    def h(self, psi):
        return pw.apply_h(self.basis, self.v_r, psi, self.beta, self.dvec)

    def a(self, x):
        return self.h(x) - self.sigma * x


def initial_state(prob: ParoProblem, c0: np.ndarray):
    """Algorithm 1 step 1: orthonormalise the start vectors and take Ritz pairs in their span."""
    y = cholesky_orthonormalize(c0)
    eps, psi, hpsi = rayleigh_ritz(y, prob.h(y))
    return eps, psi, hpsi


def source_solve(prob: ParoProblem, psi, eps, tol, max_it):
    """Algorithm 1 step 3: (H - sigma) x_i = (eps_i - sigma) psi_i for all i, started at x = psi."""
    b = (eps - prob.sigma)[:, None] * psi
    return pcg(prob.a, b, psi, prob.precond, tol, max_it)


def paro_step_alg1(prob: ParoProblem, psi, eps, tol, max_it):
    """One iteration of Algorithm 1 at a fixed potential: source solves, Cholesky, Rayleigh-Ritz."""
    x, its = source_solve(prob, psi, eps, tol, max_it)
    y = cholesky_orthonormalize(x)
    eps1, psi1, hpsi1 = rayleigh_ritz(y, prob.h(y))
    return eps1, psi1, hpsi1, its


def paro_step_alg2(prob: ParoProblem, psi, hpsi, eps, tol, max_it, drop=1e-10):
    """One iteration of Algorithm 2 (MParO I): (H - sigma) e_i = -(H psi_i - eps_i psi_i), then
    Rayleigh-Ritz in span{psi, e} (dimension up to 2N). Corrections are projected out of span{psi}
    and a correction whose remaining norm is below drop * ||e_i|| is left out (it adds nothing to the
    span and would make the 2N Gram matrix singular). Returns the lowest N Ritz pairs."""
    nb = psi.shape[0]
    b = -(hpsi - eps[:, None] * psi)
    e, its = pcg(prob.a, b, np.zeros_like(psi), prob.precond, tol, max_it)
    e = e - (e @ np.conj(psi).T) @ psi               # e_i -= sum_j <psi_j, e_i> psi_j
    keep = np.linalg.norm(e, axis=1) > drop
    y = cholesky_orthonormalize(np.concatenate([psi, e[keep]], axis=0))
    eps2, psi2, hpsi2 = rayleigh_ritz(y, prob.h(y))
    return eps2[:nb], psi2[:nb], hpsi2[:nb], its


def minres(apply_a, b, apply_minv, tol, max_it):
    """Preconditioned MINRES, one independent Hermitian system A_i e_i = b_i per row of b, started at 0,
    with a Hermitian positive definite preconditioner M^{-1} (apply_minv). Lanczos in the M^{-1} inner
    product, the tridiagonal reduced by Givens rotations; eta_i estimates ||b_i - A_i e_i||_{M^{-1}}.
    Row i stops once |eta_i| <= tol |eta_i^0| or after max_it steps. Returns (e, steps per row)."""
    b = b.astype(np.complex128)
    n = b.shape[0]
    x = np.zeros_like(b)
    v_old = np.zeros_like(b)
    v = b.copy()
    z = apply_minv(v)
    gamma = np.sqrt(np.maximum(np.real(np.sum(np.conj(z) * v, axis=1)), 0.0))
    gamma_old = np.ones(n)
    eta = gamma.copy()
    eta0 = gamma.copy()
    c_old, c = np.ones(n), np.ones(n)
    s_old, s = np.zeros(n), np.zeros(n)
    w_old = np.zeros_like(b)
    w = np.zeros_like(b)
    active = gamma > 0.0
    its = np.zeros(n, dtype=np.int64)
    for _ in range(max_it):
        if not np.any(active):
            break
        g = np.where(active, gamma, 1.0)
        zn = z / g[:, None]
        az = apply_a(zn)
        delta = np.real(np.sum(np.conj(az) * zn, axis=1))
        v_new = az - (delta / g)[:, None] * v - (g / gamma_old)[:, None] * v_old
        z_new = apply_minv(v_new)
        gamma_new = np.sqrt(np.maximum(np.real(np.sum(np.conj(z_new) * v_new, axis=1)), 0.0))
        a0 = c * delta - c_old * s * g
        a1 = np.sqrt(a0 * a0 + gamma_new * gamma_new)
        a2 = s * delta + c_old * c * g
        a3 = s_old * g
        a1s = np.where(a1 > 0.0, a1, 1.0)
        c_new, s_new = a0 / a1s, gamma_new / a1s
        w_new = (zn - a3[:, None] * w_old - a2[:, None] * w) / a1s[:, None]
        upd = active[:, None]
        x = np.where(upd, x + (c_new * eta)[:, None] * w_new, x)
        eta_new = -s_new * eta
        # advance the recurrences of the active rows
        v_old, v = np.where(upd, v, v_old), np.where(upd, v_new, v)
        z = np.where(upd, z_new, z)
        w_old, w = np.where(upd, w, w_old), np.where(upd, w_new, w)
        gamma_old, gamma = np.where(active, g, gamma_old), np.where(active, gamma_new, gamma)
        c_old, c = np.where(active, c, c_old), np.where(active, c_new, c)
        s_old, s = np.where(active, s, s_old), np.where(active, s_new, s)
        eta = np.where(active, eta_new, eta)
        its += active
        active = active & (np.abs(eta) > tol * eta0) & (gamma > 0.0)
    return x, its


def correction_alg3(prob: "ParoProblem", psi, hpsi, eps, tol, max_it):
    """Algorithm 3 step 3 for every orbital: (I - P_i)(H - eps_i)(I - P_i) e_i = -(H psi_i - eps_i psi_i)
    on the complement of psi_i, by preconditioned MINRES with M^{-1} = (I - P_i) D (I - P_i)."""
    def proj(v):
        return v - np.sum(np.conj(psi) * v, axis=1)[:, None] * psi

    def apply_a(v):
        pv = proj(v)
        return proj(prob.h(pv) - eps[:, None] * pv)

    def apply_minv(v):
        return proj(prob.precond[None, :] * proj(v))

    return minres(apply_a, proj(-(hpsi - eps[:, None] * psi)), apply_minv, tol, max_it)


def paro_step_alg3(prob: "ParoProblem", psi, hpsi, eps, tol, max_it, drop=1e-10):
    """One iteration of Algorithm 3 (MParO II): the projected corrections e_i (correction_alg3), then
    Rayleigh-Ritz in span{psi, e} exactly as in Algorithm 2. Returns the lowest N Ritz pairs."""
    nb = psi.shape[0]
    e, its = correction_alg3(prob, psi, hpsi, eps, tol, max_it)
    e = e - (e @ np.conj(psi).T) @ psi               # out of span{psi} (each e_i is already out of psi_i)
    keep = np.linalg.norm(e, axis=1) > drop
    y = cholesky_orthonormalize(np.concatenate([psi, e[keep]], axis=0))
    eps3, psi3, hpsi3 = rayleigh_ritz(y, prob.h(y))
    return eps3[:nb], psi3[:nb], hpsi3[:nb], its


# Inexact inner solves: each PCG reduces its own residual by INNER_RTOL, in at most INNER_MAX_IT
# steps. More inner work barely changes the outer rate, which is that of subspace inverse iteration.
INNER_RTOL = 0.25
INNER_MAX_IT = 8


def paro_fixed_potential(prob: ParoProblem, c0, n_occ, tol=1e-8, max_iter=2000,
                         eta=INNER_RTOL, max_inner=INNER_MAX_IT, alg=1):
    """Iterate Algorithm 1 (2, 3) at a fixed potential until max_{i<n_occ} ||H psi_i - eps_i psi_i|| < tol."""
    eps, psi, hpsi = initial_state(prob, c0)
    res = residuals(psi, hpsi, eps)
    hist = []
    for it in range(max_iter):
        if np.max(res[:n_occ]) < tol:
            return eps, psi, res, it, hist
        if alg == 1:
            eps, psi, hpsi, _ = paro_step_alg1(prob, psi, eps, eta, max_inner)
        elif alg == 2:
            eps, psi, hpsi, _ = paro_step_alg2(prob, psi, hpsi, eps, eta, max_inner)
        else:
            eps, psi, hpsi, _ = paro_step_alg3(prob, psi, hpsi, eps, eta, max_inner)
        res = residuals(psi, hpsi, eps)
        hist.append(float(np.max(res[:n_occ])))
    raise RuntimeError("ParO did not converge")
