"""Pins of the oracle's Gamma-point real-wavefunction trick against the plain complex path: two real
orbitals per complex H application equal H applied to each (KB projectors included, odd counts), the
packed density equals the per-orbital density, and a ParO step on real orbitals equals the complex step.
The trick's precondition is real orbitals: on a general complex row it gives H of the row's real part.
"""
import numpy as np

from oracle import gamma, paro, pw, scf
from paper_1702_04045_gb300 import inputs


def _problem(ecut=4.0, kb=True):
    lat, pos = inputs.diamond_cell(1, 10.26, 51)
    d = inputs.kb_strengths(len(pos), 52) if kb else None
    grid = pw.fft_grid(lat, ecut)
    b = pw.Basis(lat, ecut, grid)
    v = pw.vloc_real(lat, pos, grid, ecut, **inputs.LOCAL_PP)
    beta = pw.kb_beta(lat, pos, b.q, inputs.KB_RC) if kb else None
    return b, v, beta, d


def test_minus_g_is_an_involution():
    b, _, _, _ = _problem()
    mg = gamma.minus_g(b)
    assert np.array_equal(mg[mg], np.arange(b.npw))
    assert np.array_equal(b.miller[mg], -b.miller)


def test_two_real_orbitals_per_h_application():
    b, v, beta, d = _problem()
    dvec = pw.kb_dvec(d)
    psi = gamma.real_part(b, inputs.start_vectors(7, b.npw, 53))    # odd count
    ref = pw.apply_h(b, v, psi, beta, dvec)
    got = gamma.apply_h(b, v, psi, beta, dvec)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.abs(gamma.real_part(b, ref) - ref).max() < 1e-12 * np.abs(ref).max()   # H keeps orbitals real
    # on complex rows the packed apply returns H of the real parts, not H psi
    z = inputs.start_vectors(2, b.npw, 54)
    assert np.abs(gamma.apply_h(b, v, z, beta, dvec) - pw.apply_h(b, v, z, beta, dvec)).max() > 1e-3


def test_packed_density_equals_the_orbital_density():
    b, _, _, _ = _problem(kb=False)
    psi = gamma.real_part(b, inputs.start_vectors(9, b.npw, 55))
    occ = np.linspace(2.0, 0.3, 9)
    assert np.abs(gamma.density_weighted(b, psi, occ, 0.5) - scf.density(b, psi, occ, 0.5)).max() < 1e-13


def test_real_paro_step_equals_the_complex_step():
    b, v, beta, d = _problem()
    prob = paro.ParoProblem(b, v, beta, d)
    gprob = gamma.GammaProblem(b, v, beta, d)
    c0 = gamma.real_part(b, inputs.start_vectors(12, b.npw, 56))
    eps, psi, _ = paro.initial_state(prob, c0)
    geps, gpsi, _ = gamma.initial_state(gprob, c0)
    assert np.abs(eps - geps).max() < 1e-11
    for _ in range(3):
        eps, psi, _, _ = paro.paro_step_alg1(prob, psi, eps, 0.0, 4)
        geps, gpsi, _, _ = gamma.paro_step_alg1(gprob, gpsi, geps, 0.0, 4)
        assert np.abs(eps - geps).max() < 1e-10
    assert np.abs(gamma.real_part(b, gpsi) - gpsi).max() == 0.0
    assert np.abs(np.conj(gpsi) @ gpsi.T - np.eye(12)).max() < 1e-12
