"""CPU FP64 oracle: the adjoint (vector-Jacobian product) of H psi.

TEST INFRASTRUCTURE ONLY. Only tests, the smoke check and the bench's CPU-baseline leg may import
this package; the product path never does.

The paper defines H (Eq. e5, with the local pseudopotential and the Kleinman-Bylander projectors of
Section 2.2) but never differentiates it; this module is the derivative of that operator written out
term by term, for a loss L that is a real function of Y = H Psi.

Convention for complex arrays: the cotangent of Y is W = dL/dRe(Y) + i dL/dIm(Y), so that
dL = Re sum conj(W) dY; the returned gradient of Psi follows the same convention.

Dependence on the atom positions R_I: V_eff = V_loc(R) + V_rest with V_rest held fixed, and the
projectors beta_Ij(k+G) = Omega^{-1/2} exp(-i (k+G).R_I) p~_j(k+G).
"""
from __future__ import annotations

import numpy as np

from . import pw


def hamiltonian_parts(basis: pw.Basis, v_rest, pos, pp, kb=None):
    """V_eff(r) = V_loc(r; R) + V_rest(r), beta(R) and D per projector (None without KB)."""
    v_r = pw.vloc_real(basis.lat, pos, basis.grid, basis.ecut, pp["Z"], pp["rc"], pp["A"], pp["a"]) + v_rest
    if kb is None:
        return v_r, None, None
    rc, dstr = kb
    return v_r, pw.kb_beta(basis.lat, pos, basis.q, rc), pw.kb_dvec(dstr)


def loss(basis: pw.Basis, v_rest, pos, pp, psi, w, kb=None) -> float:
    """L = Re sum conj(W) (H Psi): the linear functional whose gradients hpsi_vjp returns."""
    v_r, beta, dvec = hamiltonian_parts(basis, v_rest, pos, pp, kb)
    return float(np.real(np.sum(np.conj(w) * pw.apply_h(basis, v_r, psi, beta, dvec))))


def grad_psi(basis: pw.Basis, v_r, w, beta=None, dvec=None) -> np.ndarray:
    """dL/dPsi = H^H W from the explicit matrix of the grid operator (no use of H = H^H)."""
    h = pw.dense_h(basis, v_r, beta, dvec)
    return (np.conj(h).T @ np.atleast_2d(w).T).T


def grad_v(basis: pw.Basis, psi, w) -> np.ndarray:
    """dL/dV(r): Y_b(G_m) holds N^{-1} sum_r exp(-i G_m.r) V(r) psi~_b(r), so
    dL/dV(r) = N^{-1} Re sum_b conj(W~_b(r)) psi~_b(r), both unnormalised inverse DFTs of the
    coefficients scattered on the grid."""
    pr = pw.to_real_space(basis, psi)
    wr = pw.to_real_space(basis, w)
    return np.real(np.sum(np.conj(wr) * pr, axis=0)) / basis.ngrid


def grad_pos_local(basis: pw.Basis, pos, pp, g_v) -> np.ndarray:
    """dL/dR_I through V_loc(r) = sum_G V_loc(G) exp(i G.r), V_loc(G) = Omega^{-1} sum_I exp(-i G.R_I) v(G):
    dV_loc(r)/dR_Ia = sum_G (-i G_a) Omega^{-1} exp(-i G.R_I) v(G) exp(i G.r), contracted with dL/dV(r)."""
    lat = basis.lat
    grid = basis.grid
    nmil = pw.grid_miller(grid).reshape(-1, 3)
    g = nmil.astype(np.float64) @ pw.reciprocal(lat)
    g2 = np.sum(g * g, axis=1)
    keep = (0.5 * g2 <= 4.0 * basis.ecut) & np.all(2 * np.abs(nmil) < np.array(grid), axis=1)
    form = np.zeros(nmil.shape[0])
    form[keep] = pw.vloc_form(g2[keep], pp["Z"], pp["rc"], pp["A"], pp["a"]) / basis.omega
    pos = np.asarray(pos, dtype=np.float64)
    out = np.zeros_like(pos)
    for i_at, r in enumerate(pos):
        sf = np.exp(-1j * (g @ r))
        for al in range(3):
            dvg = (-1j * g[:, al]) * sf * form
            dv_r = np.real(np.fft.ifftn(dvg.reshape(grid)) * basis.ngrid)
            out[i_at, al] = float(np.sum(g_v * dv_r))
    return out


def grad_pos_kb(basis: pw.Basis, pos, kb, psi, w, atoms=None) -> np.ndarray:
    """dL/dR_I through the projectors, by the product rule on Y_b += sum_p beta_p D_p (beta_p^H psi_b)
    with d beta_p / dR_Ia = -i (k+G)_a beta_p for the projectors p of atom I (rows of the atoms listed
    in `atoms` only, the others left zero, when given)."""
    rc, dstr = kb
    beta = pw.kb_beta(basis.lat, pos, basis.q, rc)
    dvec = pw.kb_dvec(dstr)
    psi = np.atleast_2d(psi)
    w = np.atleast_2d(w)
    pos = np.asarray(pos, dtype=np.float64)
    out = np.zeros_like(pos)
    proj = np.conj(beta) @ psi.T
    for i_at in (range(pos.shape[0]) if atoms is None else atoms):
        sel = np.zeros(beta.shape[0], dtype=bool)
        sel[4 * i_at:4 * i_at + 4] = True
        for al in range(3):
            dbeta = np.where(sel[:, None], -1j * basis.q[None, :, al] * beta, 0.0)
            dproj = np.conj(dbeta) @ psi.T
            dy = (dbeta.T @ (dvec[:, None] * proj) + beta.T @ (dvec[:, None] * dproj)).T
            out[i_at, al] = float(np.real(np.sum(np.conj(w) * dy)))
    return out


def hpsi_vjp(basis: pw.Basis, v_rest, pos, pp, psi, w, kb=None):
    """(dL/dPsi, dL/dV_eff(r), dL/dR) for L = Re sum conj(W) H Psi, H built from (V_rest, R, pp, kb)."""
    psi = np.atleast_2d(np.asarray(psi, dtype=np.complex128))
    w = np.atleast_2d(np.asarray(w, dtype=np.complex128))
    v_r, beta, dvec = hamiltonian_parts(basis, v_rest, pos, pp, kb)
    g_psi = grad_psi(basis, v_r, w, beta, dvec)
    g_v = grad_v(basis, psi, w)
    g_pos = grad_pos_local(basis, pos, pp, g_v)
    if kb is not None:
        g_pos = g_pos + grad_pos_kb(basis, pos, kb, psi, w)
    return g_psi, g_v, g_pos
