"""Pins of the oracle's cutoff ladder (Algorithm 1 step 2): exact embedding of the orbitals in the
larger basis (checked by summing the plane waves directly at arbitrary points), exact Fourier
interpolation of band-limited grid functions (checked against closed forms and against the density of
the embedded orbitals computed on the new grid), and the ladder's fixed point against dense
diagonalisation at the final cutoff.
"""
import math

import numpy as np

from oracle import ladder, paro, pw
from paper_1702_04045_gb300 import inputs


def _psi_at(basis, c, r):
    # psi(r) * Omega^{1/2} = sum_G c_G exp(i (k+G).r), summed directly
    return np.exp(1j * (r @ basis.q.T)) @ c.T


def test_prolong_is_an_exact_embedding():
    lat, _ = inputs.diamond_cell(1, 10.26, 5)
    k = (0.25, -1 / 3, 0.125)
    b4 = pw.Basis(lat, 4.0, pw.fft_grid(lat, 4.0, [k]), k)
    b7 = pw.Basis(lat, 7.0, pw.fft_grid(lat, 7.0, [k]), k)
    assert b7.npw > b4.npw and b7.grid != b4.grid
    psi = paro.cholesky_orthonormalize(inputs.start_vectors(6, b4.npw, 9))
    big = ladder.prolong(b4, b7, psi)
    r = np.random.default_rng(10).uniform(0, 10.26, size=(17, 3))
    assert np.abs(_psi_at(b7, big, r) - _psi_at(b4, psi, r)).max() < 1e-10
    assert np.abs(np.conj(big) @ big.T - np.eye(6)).max() < 1e-13
    assert np.count_nonzero(np.abs(big).sum(axis=0)) == b4.npw


def test_fourier_interpolation_of_band_limited_functions():
    # a sum of cosines with |n_i| < N_i/2 on the 18^3 grid, interpolated to 32^3 and 27 x 36 x 24
    n_list = [(0, 0, 0), (1, -2, 3), (4, 0, -8), (-8, 7, 1)]
    amp = [0.3, 1.1, -0.4, 0.25]
    ph = [0.0, 0.7, -1.3, 2.0]

    def f(grid):
        j = np.stack(np.meshgrid(*[np.arange(g) / g for g in grid], indexing="ij"), axis=-1)
        return sum(a * np.cos(2 * math.pi * (j @ np.array(n, dtype=float)) + p) for a, n, p in zip(amp, n_list, ph))

    for new in ((32, 32, 32), (27, 36, 24)):
        assert np.abs(ladder.fourier_interpolate(f((18, 18, 18)), new) - f(new)).max() < 1e-12
    # the density of orbitals on the alias-free grid of the low cutoff, interpolated, equals the density of
    # the embedded orbitals computed on the grid of the high cutoff
    lat, _ = inputs.diamond_cell(1, 10.26, 5)
    b4 = pw.Basis(lat, 4.0, pw.fft_grid(lat, 4.0), (0, 0, 0))
    b7 = pw.Basis(lat, 7.0, pw.fft_grid(lat, 7.0), (0, 0, 0))
    psi = paro.cholesky_orthonormalize(inputs.start_vectors(5, b4.npw, 11))
    occ = np.full(5, 2.0)
    from oracle import scf
    rho4 = scf.density(b4, psi, occ)
    rho7 = scf.density(b7, ladder.prolong(b4, b7, psi), occ)
    assert np.abs(ladder.fourier_interpolate(rho4, b7.grid) - rho7).max() < 1e-13


def test_ladder_fixed_point_is_the_dense_spectrum_of_the_final_cutoff():
    lat, pos = inputs.diamond_cell(1, 10.26, 1001)
    c0 = inputs.start_vectors(12, pw.Basis(lat, 3.0, pw.fft_grid(lat, 3.0)).npw, 12)
    prob, eps, psi, hist = ladder.ladder_fixed_potential(lat, pos, [(3.0, 6), (5.0, 4)], c0, inputs.LOCAL_PP, alg=2)
    assert len(hist) == 10
    hpsi = prob.h(psi)
    for _ in range(300):
        if np.max(paro.residuals(psi, hpsi, eps)[:8]) < 1e-9:
            break
        eps, psi, hpsi, _ = paro.paro_step_alg2(prob, psi, hpsi, eps, paro.INNER_RTOL, paro.INNER_MAX_IT)
    ev = np.linalg.eigvalsh(pw.dense_h(prob.basis, prob.v_r))
    assert np.abs(eps[:8] - ev[:8]).max() < 1e-10
