"""GPU parity of the Gamma-point real-wavefunction mode (paro_set_gamma_real: two real orbitals per packed
complex H application and density transform, real Gram and Rayleigh-Ritz matrices) against the oracle's
real-wavefunction path and the complex path: ParO steps (FP64 and mixed, KB projectors, odd band count),
realness of the orbitals, the SCF fixed point of the 8-atom KB cell, and calls on general complex vectors,
which keep the complex path.
"""
import json
import os

import numpy as np
import pytest

from oracle import gamma, paro as opar, pw
from paper_1702_04045_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "scf_si8kb_ecut10.json")


def _setup(precision, nb=11, ecut=4.0, gamma_mode=True):
    from paper_1702_04045_gb300 import paro
    lat, pos = inputs.diamond_cell(1, 10.26, 51)
    d = inputs.kb_strengths(len(pos), 52)
    ctx = paro.Context(lat, pos, ecut, nb, 8, precision)
    ctx.set_local_pp(**inputs.LOCAL_PP)
    ctx.set_kb(inputs.KB_RC, d)
    if gamma_mode:
        ctx.set_gamma_real(True)
    grid = pw.fft_grid(lat, ecut)
    b = pw.Basis(lat, ecut, grid)
    v = pw.vloc_real(lat, pos, grid, ecut, **inputs.LOCAL_PP)
    prob = gamma.GammaProblem(b, v, pw.kb_beta(lat, pos, b.q, inputs.KB_RC), d)
    return ctx, prob


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 2e-6)])
def test_gamma_steps_match_oracle(precision, tol):
    ctx, prob = _setup(precision)
    c0 = inputs.start_vectors(11, prob.basis.npw, 57)
    eps, psi, _ = gamma.initial_state(prob, c0)
    ctx.set_orbitals(c0)
    assert np.abs(ctx.eigenvalues()[0] - eps).max() < tol
    err = 0.0
    for _ in range(3):
        eps, psi, _, _ = gamma.paro_step_alg1(prob, psi, eps, 0.0, 4)
        ctx.step(1, 0.0, 4)
        err = max(err, float(np.abs(ctx.eigenvalues()[0] - eps).max()))
    print(f"{precision} real-wavefunction steps: max eigenvalue difference {err:.2e} Ha")
    assert err < tol
    got = ctx.get_orbitals()
    assert np.abs(gamma.real_part(prob.basis, got) - got).max() < (1e-15 if precision == "fp64" else 1e-7)


def test_gamma_steps_equal_complex_steps():
    ctx_g, prob = _setup("fp64")
    ctx_c, _ = _setup("fp64", gamma_mode=False)
    c0 = gamma.real_part(prob.basis, inputs.start_vectors(11, prob.basis.npw, 58))
    ctx_g.set_orbitals(c0)
    ctx_c.set_orbitals(c0)
    for alg in (1, 2, 3):
        ctx_g.step(alg, 0.0, 4)
        ctx_c.step(alg, 0.0, 4)
        assert np.abs(ctx_g.eigenvalues()[0] - ctx_c.eigenvalues()[0]).max() < 1e-10, alg


def test_gamma_mode_keeps_the_complex_path_for_general_vectors():
    ctx, prob = _setup("fp64")
    rng = np.random.default_rng(59)
    z = rng.standard_normal((5, prob.basis.npw)) + 1j * rng.standard_normal((5, prob.basis.npw))
    ref = pw.apply_h(prob.basis, prob.v_r, z, prob.beta, prob.dvec)
    got = ctx.apply_h(torch.from_numpy(z).cuda()).cpu().numpy()
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("precision,alg,tol_e,tol_eig", [("fp64", 3, 1e-10, 1e-9), ("mixed", 1, 1e-6, 1e-6)])
def test_gamma_scf_fixed_point_matches_dense_oracle(precision, alg, tol_e, tol_eig):
    from paper_1702_04045_gb300 import paro
    with open(GOLDEN) as f:
        ref = json.load(f)
    lat, pos = inputs.diamond_cell(1, 10.26, 41)
    ctx = paro.Context(lat, pos, 10.0, 12, 8, precision)
    ctx.set_local_pp(**inputs.LOCAL_PP)
    ctx.set_kb(inputs.KB_RC, inputs.kb_strengths(len(pos), 42))
    ctx.set_gamma_real(True)
    ctx.set_orbitals(inputs.start_vectors(12, ctx.npw(), 2))
    opts = paro.ScfOptions(alg=alg, tol_per_atom=0.0)
    eps_prev, small = None, 0
    thr = 1e-12 if precision == "fp64" else 1e-8
    for it in range(4000):
        terms, _ = ctx.scf_step(opts)
        eps = ctx.eigenvalues()[0][:8]
        small = small + 1 if eps_prev is not None and np.abs(eps - eps_prev).max() < thr else 0
        eps_prev = eps
        if small >= (10 if precision == "fp64" else 50):
            break
    e_err = abs(terms["total"] - ref["energy"]["total"]) / 8
    eig_err = float(np.abs(eps - np.array(ref["eigenvalues"][:8])).max())
    print(f"{precision} real-wavefunction Algorithm {alg} SCF, {it + 1} iterations: energy error {e_err:.2e} "
          f"Ha/atom, eigenvalue error {eig_err:.2e} Ha")
    assert e_err < tol_e
    assert eig_err < tol_eig
