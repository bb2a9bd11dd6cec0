"""Pins of the oracle's source solves, projection step and ParO iteration (Algorithms 1, 2)."""
import numpy as np
import pytest

from oracle import paro, pw
from paper_1702_04045_gb300 import inputs


def _problem(ecut=4.0, kb=True, kfrac=(0, 0, 0), seed=21):
    lat, pos = inputs.diamond_cell(1, 10.26, seed)
    grid = pw.fft_grid(lat, ecut, [kfrac])
    b = pw.Basis(lat, ecut, grid, kfrac)
    v = pw.vloc_real(lat, pos, grid, ecut, **inputs.LOCAL_PP)
    beta = pw.kb_beta(lat, pos, b.q, inputs.KB_RC) if kb else None
    d = inputs.kb_strengths(len(pos), seed + 1) if kb else None
    return paro.ParoProblem(b, v, beta, d), lat, pos


def test_sigma_is_below_spectrum():
    prob, _, _ = _problem()
    ev = np.linalg.eigvalsh(pw.dense_h(prob.basis, prob.v_r, prob.beta, prob.dvec))
    assert prob.sigma < ev[0] - 0.5 + 1e-12


def test_pcg_solves_shifted_system():
    prob, _, _ = _problem()
    h = pw.dense_h(prob.basis, prob.v_r, prob.beta, prob.dvec)
    a = h - prob.sigma * np.eye(prob.basis.npw)
    rng = np.random.default_rng(1)
    b = rng.standard_normal((3, prob.basis.npw)) + 1j * rng.standard_normal((3, prob.basis.npw))
    x, its = paro.pcg(prob.a, b, np.zeros_like(b), prob.precond, 1e-12, 500)
    ref = np.linalg.solve(a, b.T).T
    assert np.abs(x - ref).max() < 1e-9 * np.abs(ref).max()
    assert np.all(its > 0) and np.all(its < 500)


def test_pcg_fixed_iterations_reduce_energy_norm_error():
    # CG minimises the A-norm error over the Krylov space: it decreases monotonically.
    prob, _, _ = _problem()
    h = pw.dense_h(prob.basis, prob.v_r, prob.beta, prob.dvec)
    a = h - prob.sigma * np.eye(prob.basis.npw)
    rng = np.random.default_rng(2)
    b = rng.standard_normal((1, prob.basis.npw)) + 0j
    ref = np.linalg.solve(a, b.T).T
    errs = []
    for k in range(1, 8):
        x, _ = paro.pcg(prob.a, b, np.zeros_like(b), prob.precond, 0.0, k)
        e = (x - ref)[0]
        errs.append(np.real(np.vdot(e, a @ e)))
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))


def test_cholesky_orthonormalize_nested_spans():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((6, 50)) + 1j * rng.standard_normal((6, 50))
    y = paro.cholesky_orthonormalize(x)
    assert np.abs(np.conj(y) @ y.T - np.eye(6)).max() < 1e-13
    for k in range(1, 7):
        # span{y_1..y_k} == span{x_1..x_k}: projecting x_k onto the y's recovers it
        proj = (x[k - 1] @ np.conj(y[:k]).T) @ y[:k]
        assert np.abs(proj - x[k - 1]).max() < 1e-12 * np.abs(x[k - 1]).max()


def test_ritz_values_bound_eigenvalues_from_above():
    prob, _, _ = _problem()
    ev = np.linalg.eigvalsh(pw.dense_h(prob.basis, prob.v_r, prob.beta, prob.dvec))
    rng = np.random.default_rng(4)
    c0 = rng.standard_normal((8, prob.basis.npw)) + 1j * rng.standard_normal((8, prob.basis.npw))
    eps, psi, hpsi = paro.initial_state(prob, c0)
    assert np.all(eps >= ev[:8] - 1e-12)                 # Courant-Fischer
    assert np.abs(hpsi - prob.h(psi)).max() < 1e-11


@pytest.mark.parametrize("alg", [1, 2])
@pytest.mark.parametrize("kb,kfrac", [(False, (0, 0, 0)), (True, (0, 0, 0)), (True, (0.25, 0, -1 / 3))])
def test_paro_converges_to_dense_diagonalisation(alg, kb, kfrac):
    # The paper's own validation (ParO eigenvalues converge to those of a standard solver), with
    # brute-force dense diagonalisation as the standard.
    prob, _, _ = _problem(ecut=3.0, kb=kb, kfrac=kfrac)
    ev = np.linalg.eigvalsh(pw.dense_h(prob.basis, prob.v_r, prob.beta, prob.dvec))
    nb, nocc = 10, 8
    c0 = inputs.start_vectors(nb, prob.basis.npw, 7)
    eps, psi, res, n_it, _ = paro.paro_fixed_potential(prob, c0, nocc, tol=1e-8, alg=alg)
    assert np.abs(eps[:nocc] - ev[:nocc]).max() < 1e-10
    assert np.abs(np.conj(psi) @ psi.T - np.eye(nb)).max() < 1e-12
    assert np.max(res[:nocc]) < 1e-8


def test_alg2_ritz_values_monotone():
    # span{psi^n, e} contains psi^n, so Algorithm 2's Ritz values never increase.
    prob, _, _ = _problem(ecut=3.0)
    c0 = inputs.start_vectors(10, prob.basis.npw, 8)
    eps, psi, hpsi = paro.initial_state(prob, c0)
    for _ in range(6):
        eps2, psi, hpsi, _ = paro.paro_step_alg2(prob, psi, hpsi, eps, 0.1, 20)
        assert np.all(eps2 <= eps + 1e-12)
        eps = eps2


def test_free_electron_paro_fixed_point():
    # V = 0 at Gamma: the occupied eigenvalues are 0, then six times g, then twelve times 2g.
    lat = np.eye(3) * 10.26
    b = pw.Basis(lat, 3.0, pw.fft_grid(lat, 3.0))
    prob = paro.ParoProblem(b, np.zeros(b.grid))
    c0 = inputs.start_vectors(7, b.npw, 9)
    eps, psi, res, _, _ = paro.paro_fixed_potential(prob, c0, 7, tol=1e-9)
    g = (2 * np.pi / 10.26) ** 2 / 2
    assert abs(eps[0]) < 1e-12 and np.abs(eps[1:7] - g).max() < 1e-12
