"""CPU FP64 oracle: the cutoff ladder of Algorithm 1 (step 2): E_cut is raised from one level to the next
and the iteration goes on in the larger plane-wave space V_{N_G^{n+1}}, which contains the old one.

TEST INFRASTRUCTURE ONLY (see oracle/pw.py). Plain NumPy in float64/complex128.

Readings of points the paper leaves open (it never ran the ladder and has no estimator for it):
  * the schedule of cutoffs is fixed by the caller;
  * the orbitals psi_i^n of the old level enter the source problems of the new level unchanged: their
    coefficients are embedded in the larger basis (new coefficients zero), so they stay orthonormal,
    and the eigenvalue estimates eps_i^n are kept (step 3 uses eps_i^n psi_i^n as the right-hand side);
  * the FFT grid follows the alias-free rule at the new cutoff, and the local pseudopotential is rebuilt
    on it (its density-sphere cutoff 4 E_cut moves with E_cut);
  * every other grid function (the rest V_eff - V_loc of a given potential, the SCF input density) is
    carried to the new grid by Fourier interpolation: its Fourier coefficients with |n_i| < N_i/2 on
    the old grid are placed at the same n on the new grid (exact for a function band-limited to the old
    grid); the Pulay history starts afresh at each level.
"""
from __future__ import annotations

import numpy as np

from . import paro, pw


def prolong(b_old: pw.Basis, b_new: pw.Basis, psi: np.ndarray) -> np.ndarray:
    """Embeds coefficient rows of the basis b_old into the larger basis b_new of the same k-point."""
    index = {tuple(m): i for i, m in enumerate(b_new.miller.tolist())}
    where = np.array([index[tuple(m)] for m in b_old.miller.tolist()], dtype=np.int64)
    out = np.zeros((psi.shape[0], b_new.npw), dtype=np.complex128)
    out[:, where] = psi
    return out


def fourier_interpolate(f: np.ndarray, grid_new) -> np.ndarray:
    """Real grid function f on grid f.shape -> the trigonometric polynomial through it, sampled on
    grid_new: coefficients F(n) = N^{-1} sum_j f_j exp(-2 pi i n.j/N) for |n_i| < N_i/2 (the Nyquist
    planes are dropped), then f_new(j') = sum_n F(n) exp(2 pi i n.j'/N')."""
    grid_old = f.shape
    coef = np.fft.fftn(f) / f.size
    out = np.zeros(grid_new, dtype=np.complex128)
    mil = pw.grid_miller(grid_old).reshape(-1, 3)
    keep = np.all(2 * np.abs(mil) < np.array(grid_old), axis=1)
    src = pw.grid_index(mil[keep], grid_old)
    dst = pw.grid_index(mil[keep], grid_new)
    out.reshape(-1)[dst] = coef.reshape(-1)[src]
    return np.real(np.fft.ifftn(out) * out.size)


def level_problem(lat, pos, ecut, kfrac, pp, beta_rc=None, dstr=None, v_rest=None, delta=0.5):
    """The fixed-potential problem of one ladder level: basis and grid of ecut, V_eff = V_loc + v_rest
    (v_rest already on this level's grid), KB projectors if dstr is given."""
    grid = pw.fft_grid(lat, ecut, [kfrac])
    b = pw.Basis(lat, ecut, grid, kfrac)
    v = pw.vloc_real(lat, pos, grid, ecut, **pp)
    if v_rest is not None:
        v = v + v_rest
    beta = pw.kb_beta(lat, pos, b.q, beta_rc) if dstr is not None else None
    return paro.ParoProblem(b, v, beta, dstr, delta)


def ladder_fixed_potential(lat, pos, schedule, c0, pp, kfrac=(0.0, 0.0, 0.0), beta_rc=None, dstr=None,
                           eta=paro.INNER_RTOL, max_inner=paro.INNER_MAX_IT, alg=1):
    """Algorithm 1 (or 2) with a fixed cutoff schedule [(ecut, steps), ...] at the fixed potential V_loc:
    start vectors c0 on the first level (step 1), each later level starts from the embedded orbitals and
    the kept eigenvalue estimates (step 2). Returns (problem of the last level, eps, psi, list of the
    Ritz values after every step)."""
    hist = []
    prob = None
    for lev, (ecut, steps) in enumerate(schedule):
        new = level_problem(lat, pos, ecut, kfrac, pp, beta_rc, dstr)
        if lev == 0:
            eps, psi, hpsi = paro.initial_state(new, c0)
        else:
            psi = prolong(prob.basis, new.basis, psi)
            hpsi = new.h(psi)
        prob = new
        for _ in range(steps):
            if alg == 1:
                eps, psi, hpsi, _ = paro.paro_step_alg1(prob, psi, eps, eta, max_inner)
            else:
                eps, psi, hpsi, _ = paro.paro_step_alg2(prob, psi, hpsi, eps, eta, max_inner)
            hist.append(eps.copy())
    return prob, eps, psi, hist
