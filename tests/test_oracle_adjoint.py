"""Pins of the oracle's adjoint of H psi (oracle/adjoint.py) against finite differences of the
forward operator, a sum rule, the translation identity and the Hellmann-Feynman theorem."""
import numpy as np
import pytest

from oracle import adjoint, pw
from paper_1702_04045_gb300 import inputs

ECUT = 3.0


@pytest.fixture(scope="module")
def case():
    lat, pos = inputs.diamond_cell(1, 10.26, seed=4242)
    grid = pw.fft_grid(lat, ECUT)
    basis = pw.Basis(lat, ECUT, grid)
    rng = np.random.default_rng(77)
    nb = 3
    psi = rng.standard_normal((nb, basis.npw)) + 1j * rng.standard_normal((nb, basis.npw))
    w = rng.standard_normal((nb, basis.npw)) + 1j * rng.standard_normal((nb, basis.npw))
    v_rest = 0.3 * rng.standard_normal(grid)
    kb = (inputs.KB_RC, inputs.kb_strengths(len(pos), 4343))
    return basis, pos, psi, w, v_rest, kb


def test_case_is_small_and_nontrivial(case):
    basis, pos, psi, *_ = case
    assert 100 < basis.npw < 600 and len(pos) == 8


def test_grad_psi_matches_directional_difference(case):
    # L is linear in Psi: L(Psi + d) - L(Psi - d) = 2 Re sum conj(g_psi) d exactly (up to rounding).
    basis, pos, psi, w, v_rest, kb = case
    g_psi, _, _ = adjoint.hpsi_vjp(basis, v_rest, pos, inputs.LOCAL_PP, psi, w, kb)
    d = np.random.default_rng(5).standard_normal(psi.shape) * (1 + 1j)
    lp = adjoint.loss(basis, v_rest, pos, inputs.LOCAL_PP, psi + d, w, kb)
    lm = adjoint.loss(basis, v_rest, pos, inputs.LOCAL_PP, psi - d, w, kb)
    want = np.real(np.sum(np.conj(g_psi) * d))
    assert abs((lp - lm) / 2 - want) <= 1e-10 * (abs(want) + abs(lp))


def test_grad_v_matches_directional_difference(case):
    # L is linear in V(r) as well.
    basis, pos, psi, w, v_rest, kb = case
    _, g_v, _ = adjoint.hpsi_vjp(basis, v_rest, pos, inputs.LOCAL_PP, psi, w, kb)
    dv = np.random.default_rng(6).standard_normal(v_rest.shape)
    lp = adjoint.loss(basis, v_rest + dv, pos, inputs.LOCAL_PP, psi, w, kb)
    lm = adjoint.loss(basis, v_rest - dv, pos, inputs.LOCAL_PP, psi, w, kb)
    want = float(np.sum(g_v * dv))
    assert abs((lp - lm) / 2 - want) <= 1e-10 * (abs(want) + abs(lp))


def test_grad_v_sum_rule(case):
    # a constant shift c of V adds c Psi to H Psi: sum_r dL/dV(r) = Re sum conj(W) Psi
    basis, pos, psi, w, v_rest, kb = case
    _, g_v, _ = adjoint.hpsi_vjp(basis, v_rest, pos, inputs.LOCAL_PP, psi, w, kb)
    assert np.sum(g_v) == pytest.approx(np.real(np.sum(np.conj(w) * psi)), rel=1e-12)


@pytest.mark.parametrize("with_kb", [False, True])
def test_grad_pos_matches_central_difference(case, with_kb):
    basis, pos, psi, w, v_rest, kb = case
    kbx = kb if with_kb else None
    _, _, g_pos = adjoint.hpsi_vjp(basis, v_rest, pos, inputs.LOCAL_PP, psi, w, kbx)
    h = 1e-4
    scale = np.max(np.abs(g_pos))
    for i_at, al in [(0, 0), (3, 1), (6, 2), (7, 0)]:
        pp, pm = pos.copy(), pos.copy()
        pp[i_at, al] += h
        pm[i_at, al] -= h
        fd = (adjoint.loss(basis, v_rest, pp, inputs.LOCAL_PP, psi, w, kbx)
              - adjoint.loss(basis, v_rest, pm, inputs.LOCAL_PP, psi, w, kbx)) / (2 * h)
        assert abs(fd - g_pos[i_at, al]) <= 1e-6 * scale


def test_grad_pos_total_is_momentum_commutator(case):
    # With V_rest = 0, moving every atom by t gives H(R + t) = T H T^H, T = diag exp(-i (k+G).t), so
    # sum_I dL/dR_Ia = Re sum conj(W) (i [H, Q_a]) Psi with Q_a = diag (k+G)_a.
    basis, pos, psi, w, v_rest, kb = case
    zero = np.zeros_like(v_rest)
    _, _, g_pos = adjoint.hpsi_vjp(basis, zero, pos, inputs.LOCAL_PP, psi, w, kb)
    v_r, beta, dvec = adjoint.hamiltonian_parts(basis, zero, pos, inputs.LOCAL_PP, kb)
    for al in range(3):
        q = basis.q[:, al][None, :]
        hp = pw.apply_h(basis, v_r, psi, beta, dvec)
        hqp = pw.apply_h(basis, v_r, q * psi, beta, dvec)
        want = np.real(np.sum(np.conj(w) * (-1j * q * hp + 1j * hqp)))
        assert g_pos[:, al].sum() == pytest.approx(want, rel=1e-9, abs=1e-11 * np.abs(g_pos).max())


def test_grad_pos_is_hellmann_feynman_force(case):
    # W = Psi = a normalised non-degenerate eigenvector: dL/dR is d(eps)/dR (Hellmann-Feynman),
    # checked against central differences of the eigenvalue of the dense matrix.
    basis, pos, _, _, v_rest, kb = case

    def lowest(p):
        v_r, beta, dvec = adjoint.hamiltonian_parts(basis, v_rest, p, inputs.LOCAL_PP, kb)
        e, vec = np.linalg.eigh(pw.dense_h(basis, v_r, beta, dvec))
        return e, vec[:, 0]

    e, c0 = lowest(pos)
    assert e[1] - e[0] > 1e-3
    _, _, g_pos = adjoint.hpsi_vjp(basis, v_rest, pos, inputs.LOCAL_PP, c0[None], c0[None], kb)
    h = 1e-4
    for i_at, al in [(1, 2), (5, 0)]:
        pp, pm = pos.copy(), pos.copy()
        pp[i_at, al] += h
        pm[i_at, al] -= h
        fd = (lowest(pp)[0][0] - lowest(pm)[0][0]) / (2 * h)
        assert abs(fd - g_pos[i_at, al]) <= 1e-6 * max(1.0, np.abs(g_pos).max())


def test_grad_v_is_hellmann_feynman_density(case):
    # W = Psi = a normalised non-degenerate eigenvector: dL/dV(r) = d(eps)/dV(r) = |psi~(r)|^2 / N,
    # checked against central differences of the dense eigenvalue in V at single grid points.
    basis, pos, _, _, v_rest, kb = case

    def lowest(v):
        v_r, beta, dvec = adjoint.hamiltonian_parts(basis, v, pos, inputs.LOCAL_PP, kb)
        e, vec = np.linalg.eigh(pw.dense_h(basis, v_r, beta, dvec))
        return e[0], vec[:, 0]

    _, c0 = lowest(v_rest)
    _, g_v, _ = adjoint.hpsi_vjp(basis, v_rest, pos, inputs.LOCAL_PP, c0[None], c0[None], kb)
    dens = np.abs(pw.to_real_space(basis, c0[None])[0]) ** 2 / basis.ngrid
    assert np.allclose(g_v, dens, rtol=0, atol=1e-14)
    h = 1e-4
    flat = v_rest.reshape(-1)
    for j in [0, 777, flat.size // 2 + 13]:
        vp, vm = flat.copy(), flat.copy()
        vp[j] += h
        vm[j] -= h
        fd = (lowest(vp.reshape(v_rest.shape))[0] - lowest(vm.reshape(v_rest.shape))[0]) / (2 * h)
        assert abs(fd - g_v.reshape(-1)[j]) <= 1e-8 * g_v.max()
