"""Pins of the oracle's total-energy assembly (ScfSystem.energy) and of its LDA-PZ constants.

The energy functional (Section 2.1, with the nonlocal and ion-ion terms the printed functional omits)
is checked against two facts that do not use ScfSystem.energy's own arithmetic:
  * its variational derivative: for every coefficient c_iG of an occupied orbital,
    dE/d conj(c_iG) = w_k f_i (H[rho] psi_i)_G, with H[rho] = T + V_loc + V_H[rho] + V_xc[rho] + V_nl
    applied by the FFT (pw.apply_h, itself pinned to the closed-form Galerkin matrix) and rho the
    density of the orbitals themselves. A dropped occupation factor, a wrong volume element or a
    wrong factor on E_H or E_xc changes one side only;
  * the double-counting identity E = sum_i f_i <psi_i|H[rho]|psi_i> - E_H + (Omega/N) sum_r rho
    (eps_xc - v_xc) + E_Ewald, which holds for any orbitals (H built from their own density) and,
    at the SCF fixed point, with the band energies f_i eps_i.
The Perdew-Zunger fit is checked against the exact high-density coefficient of the correlation
energy, (1 - ln 2)/pi^2 (random-phase approximation, Gell-Mann and Brueckner), and against a second,
independent fit of the same Ceperley-Alder data: Perdew and Wang, Phys. Rev. B 45, 13244 (1992).
"""
import math

import numpy as np
import pytest

from oracle import paro, pw, scf
from paper_1702_04045_gb300 import inputs


def _system(kb=True, n_bands=12, n_occ=8, ecut=3.0):
    lat, pos = inputs.diamond_cell(1, 10.26, 41)
    d = inputs.kb_strengths(len(pos), 42) if kb else None
    return scf.ScfSystem(lat, pos, ecut, n_bands, n_occ, inputs.LOCAL_PP, d, inputs.KB_RC)


def _h_of_own_density(sys_, psis):
    """H[rho] psi for each k, rho the density of psis (the Kohn-Sham Hamiltonian of these orbitals)."""
    rho = sys_.density(psis)
    v, _, _ = sys_.veff(rho)
    out = []
    for b, beta, psi in zip(sys_.bases, sys_.betas, psis):
        dvec = pw.kb_dvec(sys_.dstr) if beta is not None else None
        out.append(pw.apply_h(b, v, psi, beta, dvec))
    return out, rho


@pytest.mark.parametrize("kb", [False, True])
def test_energy_derivative_is_kohn_sham_hamiltonian(kb):
    sys_ = _system(kb=kb)
    npw = sys_.bases[0].npw
    psi = paro.cholesky_orthonormalize(inputs.start_vectors(12, npw, 71))
    hpsi, _ = _h_of_own_density(sys_, [psi])
    rng = np.random.default_rng(72)
    h = 1e-5
    checked = 0
    for i in (0, 3, 7):                      # occupied bands (f = 2)
        for g in rng.choice(npw, 4, replace=False):
            for unit in (1.0, 1j):           # d/dRe c and d/dIm c
                pp, pm = psi.copy(), psi.copy()
                pp[i, g] += h * unit
                pm[i, g] -= h * unit
                fd = (sys_.energy([pp])[0]["total"] - sys_.energy([pm])[0]["total"]) / (2 * h)
                # E depends on c through |c|^2-type forms: dE/dRe c = 2 Re(f H psi), dE/dIm c = 2 Im(f H psi)
                an = 2.0 * 2.0 * (hpsi[0][i, g].real if unit == 1.0 else hpsi[0][i, g].imag)
                assert abs(fd - an) < 2e-7 * max(1.0, abs(an)), (i, g, unit, fd, an)
                checked += 1
    assert checked == 24
    # an unoccupied band does not enter the energy
    pp = psi.copy()
    pp[10, 5] += 1e-3
    assert sys_.energy([pp])[0]["total"] == sys_.energy([psi])[0]["total"]


def test_energy_double_counting_identity_any_orbitals():
    sys_ = _system()
    psi = paro.cholesky_orthonormalize(inputs.start_vectors(12, sys_.bases[0].npw, 73))
    terms, rho = sys_.energy([psi])
    hpsi, rho2 = _h_of_own_density(sys_, [psi])
    assert np.array_equal(rho, rho2)
    n = sys_.n_occ
    band = float(np.sum(sys_.occ[:n] * np.real(np.sum(np.conj(psi[:n]) * hpsi[0][:n], axis=1))))
    _, e_h = scf.hartree(sys_.lat, sys_.grid, rho)
    exc_d, vxc = scf.lda_pz(rho)
    dv = sys_.omega / rho.size
    e = band - e_h + dv * float(np.sum(rho * (exc_d - vxc))) + scf.ewald(sys_.lat, sys_.pos, 4.0)
    assert abs(e - terms["total"]) < 1e-10 * max(1.0, abs(e))


def test_energy_double_counting_at_scf_fixed_point():
    # at self-consistency (rho_out = rho_in) the occupied orbitals are eigenvectors of H[rho(psi)], so
    # sum f <psi|H|psi> becomes the band energy sum f eps. Dense SCF with Pulay mixing, run until the
    # density itself (not only the energy) has converged to 1e-10.
    sys_ = _system()
    rho_in = np.full(sys_.grid, sys_.n_el / sys_.omega)
    mixer = scf.Pulay(8, 0.7)
    for _ in range(200):
        v, _, _ = sys_.veff(rho_in)
        b, beta = sys_.bases[0], sys_.betas[0]
        eps, vec = np.linalg.eigh(pw.dense_h(b, v, beta, pw.kb_dvec(sys_.dstr)))
        psi = vec[:, : sys_.n_bands].T.copy()
        rho_out = sys_.density([psi])
        if np.abs(rho_out - rho_in).max() < 1e-10:
            break
        rho_in = mixer.mix(rho_in, rho_out)
    assert np.abs(rho_out - rho_in).max() < 1e-10
    terms, rho = sys_.energy([psi])
    _, e_h = scf.hartree(sys_.lat, sys_.grid, rho)
    exc_d, vxc = scf.lda_pz(rho)
    dv = sys_.omega / rho.size
    n = sys_.n_occ
    e = (float(np.sum(sys_.occ[:n] * eps[:n])) - e_h + dv * float(np.sum(rho * (exc_d - vxc)))
         + sys_.e_ewald)
    assert abs(e - terms["total"]) < 1e-9


def _ec_pz(rs):
    """Correlation part of the oracle's LDA: eps_xc minus the closed-form exchange -(3/4)(3/pi)^{1/3}/r_s."""
    rs = np.asarray(rs, dtype=np.float64)
    rho = 3.0 / (4.0 * math.pi * rs ** 3)
    exc, _ = scf.lda_pz(rho)
    return exc + 0.75 * (9.0 / (4.0 * math.pi ** 2)) ** (1.0 / 3.0) / rs


def test_pz_correlation_high_density_coefficient():
    # eps_c -> A ln r_s + B as r_s -> 0 with A = (1 - ln 2)/pi^2 exactly (RPA)
    r1, r2 = 1e-7, 1e-6
    slope = float((_ec_pz(r2) - _ec_pz(r1)) / math.log(r2 / r1))
    assert abs(slope - (1.0 - math.log(2.0)) / math.pi ** 2) < 2e-5


def test_pz_correlation_agrees_with_perdew_wang_fit():
    # PW92, unpolarised: eps_c = -2A(1 + a1 r_s) ln(1 + 1/(2A(b1 r_s^1/2 + b2 r_s + b3 r_s^3/2 + b4 r_s^2)))
    A, a1, b1, b2, b3, b4 = 0.031091, 0.21370, 7.5957, 3.5876, 1.6382, 0.49294
    rs = np.array([0.1, 0.3, 0.5, 0.8, 1.0, 1.5, 2.0, 3.0, 5.0, 10.0, 20.0, 50.0])
    pw92 = -2 * A * (1 + a1 * rs) * np.log(1 + 1 / (2 * A * (b1 * rs ** 0.5 + b2 * rs + b3 * rs ** 1.5 + b4 * rs ** 2)))
    pz = _ec_pz(rs)
    # the two fits of the same Monte Carlo data agree to better than 1 mHa over both PZ branches
    assert np.abs(pz - pw92).max() < 1e-3
    assert np.all(pz < 0) and np.all(np.diff(pz) > 0)
