"""Pins of the oracle's Fermi-Dirac occupations and smeared SCF (fractional occupations for cells whose
highest occupied and lowest empty levels cross; the paper is silent on occupations).

  * the occupations hold the electron count and, for a gapped spectrum as kT -> 0, reduce to the
    integer occupations of the lowest n_occ bands;
  * Mermin stationarity: at the Fermi-Dirac occupations G(f) = sum_k w_k sum_i f_i eps_i - T S(f)
    changes at first order only through the electron count, dG = mu sum w df, so a wrong sign or
    factor of the entropy, of kT or of the spin factor fails;
  * the free energy's derivative with respect to the orbital coefficients at fixed fractional
    occupations is w f (H[rho] psi) (the Kohn-Sham Hamiltonian of the weighted density);
  * the smeared SCF reaches a fixed point on a cell where integer occupations do not, and its
    ParO-merged iteration reaches the dense-diagonalisation fixed point.
"""
import math

import numpy as np
import pytest

from oracle import paro, pw, scf
from paper_1702_04045_gb300 import inputs


def _entropy_term(occs, kw, kT):
    # -T S written out: g = f / 2 per spin state, S = -sum w 2 (g ln g + (1 - g) ln(1 - g))
    s = 0.0
    for f, w in zip(occs, kw):
        for x in f:
            g = x / 2.0
            for y in (g, 1.0 - g):
                if y > 0:
                    s -= w * 2.0 * y * math.log(y)
    return -kT * s


def test_fermi_occupations_count_and_zero_width_limit():
    rng = np.random.default_rng(3)
    eps = [np.sort(rng.uniform(-1, 1, 20)) for _ in range(3)]
    kw = np.array([0.5, 0.25, 0.25])
    occ, mu, mts = scf.fermi_occupations(eps, kw, 17.0, 0.01)
    assert abs(sum(w * f.sum() for f, w in zip(occ, kw)) - 17.0) < 1e-12
    assert all(np.all((f >= 0) & (f <= 2)) and np.all(np.diff(f) <= 0) for f in occ)
    assert abs(mts - _entropy_term(occ, kw, 0.01)) < 1e-12
    # one k-point, gap of 0.1 above band 8: integer occupations as kT -> 0, mu inside the gap
    e1 = np.concatenate([np.linspace(-1, 0, 8), np.linspace(0.1, 1, 12)])
    occ, mu, mts = scf.fermi_occupations([e1], [1.0], 16.0, 1e-4)
    ref = np.zeros(20)
    ref[:8] = 2.0
    assert np.abs(occ[0] - ref).max() < 1e-12 and 0.0 < mu < 0.1 and abs(mts) < 1e-12


def test_mermin_stationarity():
    rng = np.random.default_rng(4)
    eps = [np.sort(rng.uniform(-0.5, 0.5, 16)) for _ in range(2)]
    kw = np.array([0.75, 0.25])
    kT = 0.02
    occ, mu, _ = scf.fermi_occupations(eps, kw, 12.0, kT)

    def g(o):
        return sum(w * float(np.dot(f, e)) for f, e, w in zip(o, eps, kw)) + _entropy_term(o, kw, kT)

    h = 1e-6
    # directions scaled by f (2 - f), so that f +- h d stays inside (0, 2) where S is defined
    u = [f * (2.0 - f) for f in occ]
    for _ in range(3):
        r = [rng.standard_normal(16) for _ in kw]
        c = sum(w * float(np.dot(a, b)) for a, b, w in zip(u, r, kw)) / sum(w * a.sum() for a, w in zip(u, kw))
        d = [a * (b - c) for a, b in zip(u, r)]    # sum_k w_k sum_i d_ik = 0: the count is kept
        gp = g([f + h * x for f, x in zip(occ, d)])
        gm = g([f - h * x for f, x in zip(occ, d)])
        assert abs((gp - gm) / (2 * h)) < 1e-7
    d = u                                            # changes the count by dN = sum w sum u: dG = mu dN
    dn = sum(w * a.sum() for a, w in zip(u, kw))
    gp = g([f + h * x for f, x in zip(occ, d)])
    gm = g([f - h * x for f, x in zip(occ, d)])
    assert abs((gp - gm) / (2 * h) - mu * dn) < 1e-7 * max(1.0, abs(mu * dn))


def test_free_energy_derivative_with_fractional_occupations():
    lat, pos = inputs.diamond_cell(1, 10.26, 41)
    d = inputs.kb_strengths(len(pos), 42)
    sys_ = scf.ScfSystem(lat, pos, 3.0, 12, 8, inputs.LOCAL_PP, d, inputs.KB_RC, kT=0.01)
    npw = sys_.bases[0].npw
    psi = paro.cholesky_orthonormalize(inputs.start_vectors(12, npw, 75))
    occ = [np.sort(np.random.default_rng(76).uniform(0, 2, 12))[::-1].copy()]
    rho = sys_.density([psi], occ)
    v, _, _ = sys_.veff(rho)
    hpsi = pw.apply_h(sys_.bases[0], v, psi, sys_.betas[0], pw.kb_dvec(d))
    h = 1e-5
    for i, g in ((0, 5), (6, 40), (11, 77)):
        pp, pm = psi.copy(), psi.copy()
        pp[i, g] += h
        pm[i, g] -= h
        fd = (sys_.energy([pp], occ)[0]["total"] - sys_.energy([pm], occ)[0]["total"]) / (2 * h)
        an = 2.0 * occ[0][i] * hpsi[i, g].real
        assert abs(fd - an) < 2e-7 * max(1.0, abs(an)), (i, g, fd, an)


def test_smearing_reduces_to_integer_occupations_on_a_gapped_cell():
    lat, pos = inputs.diamond_cell(1, 10.26, 41)
    d = inputs.kb_strengths(len(pos), 42)
    fixed = scf.ScfSystem(lat, pos, 3.0, 12, 8, inputs.LOCAL_PP, d, inputs.KB_RC)
    smeared = scf.ScfSystem(lat, pos, 3.0, 12, 8, inputs.LOCAL_PP, d, inputs.KB_RC, kT=1e-4)
    t0 = scf.dense_scf(fixed, tol=1e-11)[0]
    t1 = scf.dense_scf(smeared, tol=1e-11)[0]
    assert abs(t1["smearing"]) < 1e-12
    assert abs(t0["total"] - t1["total"]) < 1e-9


def _crossing_cell(kT):
    # 16 occupied bands of the 8-atom cell: bands 16 and 17 cross (gap ~1e-5 Ha)
    lat, pos = inputs.diamond_cell(1, 10.26, 41)
    d = inputs.kb_strengths(len(pos), 42)
    return scf.ScfSystem(lat, pos, 3.0, 20, 16, inputs.LOCAL_PP, d, inputs.KB_RC, kT=kT)


def test_smeared_scf_converges_where_integer_occupations_do_not():
    with pytest.raises(RuntimeError):
        scf.dense_scf(_crossing_cell(0.0), tol=1e-10, max_iter=100)
    terms, eps, psis, it = scf.dense_scf(_crossing_cell(0.002), tol=1e-10, max_iter=100)
    assert it < 60


@pytest.mark.slow
def test_smeared_paro_scf_fixed_point_equals_dense():
    sys_ = _crossing_cell(0.002)
    t_dense, eps_dense, _, _ = scf.dense_scf(sys_, tol=1e-11)
    c0 = inputs.start_vectors(20, sys_.bases[0].npw, 2)
    t_paro, eps_paro, _, _ = scf.paro_scf(sys_, [c0], tol=1e-11, alg=2)
    assert abs(t_paro["total"] - t_dense["total"]) / 8 < 1e-8
    assert np.abs(eps_paro[0][:18] - eps_dense[0][:18]).max() < 1e-6
