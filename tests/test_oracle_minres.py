"""Pins of the oracle's preconditioned MINRES and of Algorithm 3 (MParO II):
  * MINRES's iterate after k steps minimises ||b - A x||_{M^{-1}} over the Krylov space
    K_k(M^{-1} A, M^{-1} b) (brute force: an explicit Krylov basis and a least-squares solve), and its
    residual estimate |eta_k| equals that norm; after n steps it is the exact solution of the n x n system;
  * the projected correction equation of Algorithm 3 is solved on the complement of psi_i: the result is
    orthogonal to psi_i and equals the dense solve Q (Q^H (H - eps_i) Q)^{-1} Q^H b with Q an orthonormal
    basis of that complement;
  * Algorithm 3's fixed point is the dense spectrum of the grid Hamiltonian.
"""
import numpy as np
import pytest

from oracle import paro, pw
from paper_1702_04045_gb300 import inputs


def _system(n, seed):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    lam = np.concatenate([rng.uniform(-3, -0.5, n // 3), rng.uniform(0.5, 4, n - n // 3)])  # indefinite
    a = (q * lam) @ q.conj().T
    a = 0.5 * (a + a.conj().T)
    mdiag = rng.uniform(0.5, 2.0, n)                 # M^{-1} = diag(mdiag), positive definite
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return a, mdiag, b


def _mnorm(r, mdiag):
    return float(np.sqrt(np.real(np.sum(np.conj(r) * mdiag * r))))


@pytest.mark.parametrize("k", [1, 2, 4, 7])
def test_minres_minimises_the_preconditioned_residual_over_the_krylov_space(k):
    a, mdiag, b = _system(24, 7)
    x, its = paro.minres(lambda v: v @ a.T, b[None, :], lambda v: v * mdiag[None, :], 0.0, k)
    assert its[0] == k
    # explicit Krylov basis of M^{-1} A applied to M^{-1} b, least squares in the M^{-1} norm
    kb = [mdiag * b]
    for _ in range(k - 1):
        kb.append(mdiag * (a @ kb[-1]))
    kmat = np.stack(kb, axis=1)
    w = np.sqrt(mdiag)
    y, *_ = np.linalg.lstsq(w[:, None] * (a @ kmat), w * b, rcond=None)
    ref = kmat @ y
    assert np.abs(x[0] - ref).max() < 1e-9 * np.abs(ref).max()


def test_minres_residual_estimate_and_exact_solution():
    a, mdiag, b = _system(16, 8)
    prev = None
    for k in range(1, 17):
        x, _ = paro.minres(lambda v: v @ a.T, b[None, :], lambda v: v * mdiag[None, :], 0.0, k)
        r = _mnorm(b - a @ x[0], mdiag)
        if prev is not None:
            assert r <= prev * (1 + 1e-10)            # non-increasing
        prev = r
    assert np.abs(x[0] - np.linalg.solve(a, b)).max() < 1e-8 * np.abs(np.linalg.solve(a, b)).max()
    # the stopping rule: |eta| <= tol |eta_0| with the true residual norm behind eta
    x, its = paro.minres(lambda v: v @ a.T, b[None, :], lambda v: v * mdiag[None, :], 1e-3, 100)
    assert _mnorm(b - a @ x[0], mdiag) <= 1e-3 * _mnorm(b, mdiag) * (1 + 1e-8)
    x1, _ = paro.minres(lambda v: v @ a.T, b[None, :], lambda v: v * mdiag[None, :], 0.0, int(its[0]) - 1)
    assert _mnorm(b - a @ x1[0], mdiag) > 1e-3 * _mnorm(b, mdiag)


def test_alg3_correction_solves_the_projected_equation():
    lat, pos = inputs.diamond_cell(1, 10.26, 1001)
    grid = pw.fft_grid(lat, 1.5)
    b = pw.Basis(lat, 1.5, grid)
    v = pw.vloc_real(lat, pos, grid, 1.5, **inputs.LOCAL_PP)
    prob = paro.ParoProblem(b, v)
    eps, psi, hpsi = paro.initial_state(prob, inputs.start_vectors(4, b.npw, 3))
    e, its = paro.correction_alg3(prob, psi, hpsi, eps, 1e-13, 400)
    h = pw.dense_h(b, v)
    for i in range(4):
        assert abs(np.vdot(psi[i], e[i])) < 1e-12 * np.linalg.norm(e[i])
        # Q: orthonormal basis of the complement of psi_i
        u, _, _ = np.linalg.svd(np.eye(b.npw) - np.outer(psi[i], psi[i].conj()))
        q = u[:, : b.npw - 1]
        rhs = -(hpsi[i] - eps[i] * psi[i])
        ref = q @ np.linalg.solve(q.conj().T @ (h - eps[i] * np.eye(b.npw)) @ q, q.conj().T @ rhs)
        assert np.abs(e[i] - ref).max() < 1e-9 * np.abs(ref).max(), i


def test_alg3_fixed_point_is_the_dense_spectrum():
    lat, pos = inputs.diamond_cell(1, 10.26, 1001)
    grid = pw.fft_grid(lat, 3.0)
    b = pw.Basis(lat, 3.0, grid)
    v = pw.vloc_real(lat, pos, grid, 3.0, **inputs.LOCAL_PP)
    prob = paro.ParoProblem(b, v)
    eps, _, res, it, _ = paro.paro_fixed_potential(prob, inputs.start_vectors(12, b.npw, 4), 8, tol=1e-9, alg=3)
    ev = np.linalg.eigvalsh(pw.dense_h(b, v))
    assert np.abs(eps[:8] - ev[:8]).max() < 1e-10
