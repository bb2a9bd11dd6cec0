"""GPU parity of Algorithm 3 (MParO II: projected correction equations by batched preconditioned MINRES,
then Rayleigh-Ritz in span{psi, e}) against the FP64 CPU oracle: ParO steps at fixed inner iteration
counts (FP64 and mixed, with KB projectors, at k != 0), the fixed point against dense diagonalisation,
and the merged SCF fixed point on a register-FFT grid.
"""
import json
import os

import numpy as np
import pytest

from oracle import paro as opar
from oracle import pw
from paper_1702_04045_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "scf_si8kb_ecut10.json")


def _small(precision, kfrac=(0.25, -1 / 3, 0.125), ecut=4.0):
    from paper_1702_04045_gb300 import paro
    lat, pos = inputs.diamond_cell(1, 10.26, 61)
    d = inputs.kb_strengths(len(pos), 62)
    ctx = paro.Context(lat, pos, ecut, 12, 8, precision, kpts=[kfrac])
    ctx.set_local_pp(**inputs.LOCAL_PP)
    ctx.set_kb(inputs.KB_RC, d)
    grid = pw.fft_grid(lat, ecut, [kfrac])
    b = pw.Basis(lat, ecut, grid, kfrac)
    v = pw.vloc_real(lat, pos, grid, ecut, **inputs.LOCAL_PP)
    prob = opar.ParoProblem(b, v, pw.kb_beta(lat, pos, b.q, inputs.KB_RC), d)
    return ctx, prob


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 2e-6)])
def test_alg3_steps_match_oracle(precision, tol):
    ctx, prob = _small(precision)
    c0 = inputs.start_vectors(12, prob.basis.npw, 31)
    eps, psi, hpsi = opar.initial_state(prob, c0)
    ctx.set_orbitals(c0)
    err = 0.0
    for _ in range(4):
        eps, psi, hpsi, _ = opar.paro_step_alg3(prob, psi, hpsi, eps, 0.0, 4)
        ctx.step(3, 0.0, 4)
        err = max(err, float(np.abs(ctx.eigenvalues()[0] - eps).max()))
    print(f"{precision} Algorithm 3 steps: max eigenvalue difference {err:.2e} Ha")
    assert err < tol
    if precision == "fp64":  # occupied subspace projectors agree
        g = ctx.get_orbitals()[:8]
        assert np.abs(g.T @ g.conj() - psi[:8].T @ psi[:8].conj()).max() < 1e-9


def test_alg3_converges_to_dense_eigenvalues():
    ctx, prob = _small("fp64", kfrac=(0, 0, 0), ecut=5.0)
    ctx.set_orbitals(inputs.start_vectors(12, prob.basis.npw, 32))
    for it in range(500):
        r = ctx.step(3, 0.25, 8)
        if r < 1e-9:
            break
    assert r < 1e-9
    ev = np.linalg.eigvalsh(pw.dense_h(prob.basis, prob.v_r, prob.beta, prob.dvec))
    print(f"Algorithm 3 to residual 1e-9 in {it + 1} iterations")
    assert np.abs(ctx.eigenvalues()[0][:8] - ev[:8]).max() < 1e-10


@pytest.mark.parametrize("precision,tol_e,tol_eig", [("fp64", 1e-10, 1e-9), ("mixed", 1e-6, 1e-6)])
def test_alg3_scf_fixed_point_matches_dense_oracle(precision, tol_e, tol_eig):
    # the 8-atom KB cell at 10 Ha (32^3 grid), 12 bands, 8 occupied: the oracle's dense SCF fixed point
    # (tests/golden/scf_si8kb_ecut10.json, written by tests/golden/make_scf_golden.py)
    from paper_1702_04045_gb300 import paro
    with open(GOLDEN) as f:
        ref = json.load(f)
    lat, pos = inputs.diamond_cell(1, 10.26, 41)
    ctx = paro.Context(lat, pos, 10.0, 12, 8, precision)
    ctx.set_local_pp(**inputs.LOCAL_PP)
    ctx.set_kb(inputs.KB_RC, inputs.kb_strengths(len(pos), 42))
    ctx.set_orbitals(inputs.start_vectors(12, ctx.npw(), 2))
    opts = paro.ScfOptions(alg=3, tol_per_atom=0.0)
    eps_prev, small = None, 0
    thr = 1e-12 if precision == "fp64" else 1e-8
    for it in range(1500):
        terms, _ = ctx.scf_step(opts)
        eps = ctx.eigenvalues()[0][:8]
        small = small + 1 if eps_prev is not None and np.abs(eps - eps_prev).max() < thr else 0
        eps_prev = eps
        if small >= 10:
            break
    e_err = abs(terms["total"] - ref["energy"]["total"]) / 8
    eig_err = float(np.abs(eps - np.array(ref["eigenvalues"][:8])).max())
    print(f"{precision} Algorithm 3 SCF, {it + 1} iterations: energy error {e_err:.2e} Ha/atom, "
          f"eigenvalue error {eig_err:.2e} Ha")
    assert e_err < tol_e
    assert eig_err < tol_eig
