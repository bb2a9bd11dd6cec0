"""Pins of the oracle's SCF pieces: Ewald, LDA-PZ, Hartree, Pulay, density, SCF fixed point."""
import math

import numpy as np
import pytest

from oracle import pw, scf
from paper_1702_04045_gb300 import inputs


def test_ewald_independent_of_eta():
    lat, pos = inputs.diamond_cell(1, 10.26, 31)
    e = [scf.ewald(lat, pos, 4.0, eta=x) for x in (0.2, 0.35, 0.6)]
    assert max(e) - min(e) < 1e-10


def test_ewald_nacl_madelung_constant():
    # Rock salt of unit charges, conventional cube a: E = -8 M / a per cell (4 pairs, r0 = a/2),
    # Madelung constant M = 1.747564594633 (textbook value).
    a = 7.3
    lat = np.eye(3) * a
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    pos = np.concatenate([fcc, fcc + [0.5, 0, 0]]) * a
    z = np.array([1.0] * 4 + [-1.0] * 4)
    assert abs(scf.ewald(lat, pos, z) - (-8 * 1.747564594633 / a)) < 1e-10


def test_lda_potential_is_derivative_of_energy_density():
    rho = np.array([1e-4, 3e-3, 0.02, 0.1, 0.5, 2.0, 30.0])   # both r_s branches
    h = 1e-6 * rho
    ep, _ = scf.lda_pz(rho + h)
    em, _ = scf.lda_pz(rho - h)
    _, v = scf.lda_pz(rho)
    fd = ((rho + h) * ep - (rho - h) * em) / (2 * h)
    assert np.abs(fd - v).max() < 1e-8


def test_lda_branches_meet_at_rs_one_and_exchange_closed_form():
    rho1 = 3.0 / (4 * math.pi)                          # r_s = 1
    e_lo, _ = scf.lda_pz(np.array([rho1 * (1 + 1e-12)]))
    e_hi, _ = scf.lda_pz(np.array([rho1 * (1 - 1e-12)]))
    assert abs(e_lo[0] - e_hi[0]) < 5e-4                # the fit is continuous to its printed digits
    ex = -0.75 * (3 / math.pi) ** (1 / 3) * rho1 ** (1 / 3)   # exchange at r_s = 1: -0.458165 Ha
    assert abs(ex + 0.4581652932831429) < 1e-12
    e0, v0 = scf.lda_pz(np.array([0.0, 1e-31]))
    assert np.all(e0 == 0) and np.all(v0 == 0)


def test_hartree_of_a_cosine_density():
    # rho = rho0 + c cos(G0 . r): V_H = 4 pi c cos(G0 . r) / G0^2, E_H = (Omega/2) 4 pi c^2 / (2 G0^2).
    a = 9.0
    lat = np.eye(3) * a
    grid = (24, 24, 24)
    x = np.arange(24) / 24 * a
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    g0 = np.array([2, -1, 3]) * 2 * math.pi / a
    c = 0.013
    rho = 0.05 + c * np.cos(g0[0] * X + g0[1] * Y + g0[2] * Z)
    vh, eh = scf.hartree(lat, grid, rho)
    g2 = float(g0 @ g0)
    ref = 4 * math.pi * c / g2 * np.cos(g0[0] * X + g0[1] * Y + g0[2] * Z)
    assert np.abs(vh - ref).max() < 1e-13
    assert abs(eh - a ** 3 / 2 * 4 * math.pi * c * c / (2 * g2)) < 1e-12
    # E_H = 1/2 int V_H rho
    assert abs(eh - 0.5 * a ** 3 / rho.size * float(np.sum(vh * rho))) < 1e-12


def test_pulay_solves_linear_fixed_point():
    # Anderson/Pulay mixing on rho_out = A rho_in + b with full history behaves like GMRES and
    # reaches the fixed point of a 5-dimensional problem within dimension + 2 steps.
    rng = np.random.default_rng(5)
    q, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    amat = q @ np.diag([0.9, 0.5, -0.3, 0.2, 0.7]) @ q.T
    bvec = rng.standard_normal(5)
    x_star = np.linalg.solve(np.eye(5) - amat, bvec)
    mixer = scf.Pulay(depth=8, beta=0.7)
    x = np.zeros(5)
    for _ in range(7):
        x = mixer.mix(x, amat @ x + bvec)
    assert np.abs(x - x_star).max() < 1e-10


def _tiny_system(ecut=3.0, kb=True, shift=(0, 0, 0), n_bands=12, n_occ=8):
    # 8 occupied bands: this synthetic cell has a 0.1 Ha gap above band 8, while band 16 sits in a
    # near-degenerate cluster where fixed-occupation SCF oscillates without converging.
    lat, pos = inputs.diamond_cell(1, 10.26, 41)
    d = inputs.kb_strengths(len(pos), 42) if kb else None
    return scf.ScfSystem(lat, pos + np.array(shift), ecut, n_bands, n_occ, inputs.LOCAL_PP, d, inputs.KB_RC)


def test_density_integrates_to_electron_count():
    sys_ = _tiny_system(n_bands=20, n_occ=16)
    c0 = inputs.start_vectors(20, sys_.bases[0].npw, 1)
    from oracle import paro
    psi = paro.cholesky_orthonormalize(c0)
    rho = sys_.density([psi])
    assert abs(rho.sum() * sys_.omega / rho.size - 32.0) < 1e-10
    assert rho.min() >= 0


@pytest.mark.slow
def test_paro_scf_fixed_point_equals_dense_scf():
    # The SCF fixed point does not depend on the eigensolver: ParO (Algorithm 1) reaches the one
    # found with dense diagonalisation, in total energy and occupied eigenvalues.
    sys_ = _tiny_system()
    t_dense, eps_dense, _, _ = scf.dense_scf(sys_, tol=1e-11)
    c0 = inputs.start_vectors(12, sys_.bases[0].npw, 2)
    t_paro, eps_paro, _, _ = scf.paro_scf(sys_, [c0], tol=1e-11)
    assert abs(t_paro["total"] - t_dense["total"]) / 8 < 1e-8
    assert np.abs(eps_paro[0][:8] - eps_dense[0][:8]).max() < 1e-6


def test_dense_scf_energy_translation_invariant():
    # A rigid shift by whole grid steps leaves every term unchanged (an off-grid shift changes the
    # grid sampling of the nonlinear E_xc by ~1e-7 Ha here, the usual egg-box effect).
    s1 = _tiny_system(ecut=2.5)
    step = 10.26 / np.array(s1.grid)
    e1 = scf.dense_scf(s1, tol=1e-10)[0]["total"]
    e2 = scf.dense_scf(_tiny_system(ecut=2.5, shift=step * np.array([3, -5, 7])), tol=1e-10)[0]["total"]
    assert abs(e1 - e2) < 1e-9
