"""GPU parity of the cutoff ladder (paro_set_ecut, Algorithm 1 step 2) against the FP64 CPU oracle:
the rebuilt basis, grid and potential, the embedded orbitals (exact copies), ParO steps across a ladder
step (Algorithms 1 and 2, FP64 and mixed), the SCF iteration after a ladder step (input density carried
by Fourier interpolation), and the ladder's fixed point against dense diagonalisation at the final cutoff.
"""
import numpy as np
import pytest

from oracle import ladder, paro as opar, pw, scf
from paper_1702_04045_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

K = (0.25, -1 / 3, 0.125)


def _cell(kb=True):
    lat, pos = inputs.diamond_cell(1, 10.26, 61)
    return lat, pos, (inputs.kb_strengths(len(pos), 62) if kb else None)


def _ctx(ecut, precision="fp64", kfrac=K, kb=True, nb=12, nocc=8):
    from paper_1702_04045_gb300 import paro
    lat, pos, d = _cell(kb)
    ctx = paro.Context(lat, pos, ecut, nb, nocc, precision, kpts=[kfrac])
    ctx.set_local_pp(**inputs.LOCAL_PP)
    if kb:
        ctx.set_kb(inputs.KB_RC, d)
    return ctx


def test_set_ecut_embeds_orbitals_and_rebuilds_the_problem():
    lat, pos, d = _cell()
    ctx = _ctx(4.0)
    c0 = inputs.start_vectors(12, ctx.npw(), 21)
    ctx.set_orbitals(c0)
    psi4, eps4 = ctx.get_orbitals(), ctx.eigenvalues()[0].copy()
    ctx.set_ecut(7.0)
    new = ladder.level_problem(lat, pos, 7.0, K, inputs.LOCAL_PP, inputs.KB_RC, d)
    old_basis = pw.Basis(lat, 4.0, pw.fft_grid(lat, 4.0, [K]), K)
    assert ctx.grid == new.basis.grid != old_basis.grid
    assert np.array_equal(ctx.miller(), new.basis.miller)
    assert np.array_equal(ctx.get_orbitals(), ladder.prolong(old_basis, new.basis, psi4))
    assert np.array_equal(ctx.eigenvalues()[0], eps4)
    assert np.abs(ctx.get_veff() - new.v_r).max() < 1e-11
    assert abs(ctx.sigma() - new.sigma) < 1e-10
    big = ladder.prolong(old_basis, new.basis, psi4)
    assert np.abs(ctx.residuals()[0] - opar.residuals(big, new.h(big), eps4)).max() < 1e-10
    from paper_1702_04045_gb300 import paro
    with pytest.raises(paro.ParoError):
        ctx.set_ecut(5.0)  # the ladder only goes up


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 2e-6)])
@pytest.mark.parametrize("alg", [1, 2])
def test_ladder_steps_match_oracle(alg, precision, tol):
    lat, pos, d = _cell()
    ctx = _ctx(4.0, precision)
    c0 = inputs.start_vectors(12, ctx.npw(), 22)
    _, _, _, hist = ladder.ladder_fixed_potential(lat, pos, [(4.0, 3), (7.0, 3)], c0, inputs.LOCAL_PP, K,
                                                  inputs.KB_RC, d, eta=0.0, max_inner=4, alg=alg)
    ctx.set_orbitals(c0)
    got = []
    for ecut in (4.0, 7.0):
        ctx.set_ecut(ecut)
        for _ in range(3):
            ctx.step(alg, 0.0, 4)
            got.append(ctx.eigenvalues()[0].copy())
    err = max(float(np.abs(g[:8] - h[:8]).max()) for g, h in zip(got, hist))
    print(f"{precision} Algorithm {alg} ladder 4 -> 7 Ha: max eigenvalue difference {err:.2e} Ha")
    assert err < tol


def test_ladder_fixed_point_matches_dense_at_the_final_cutoff():
    # the 8-atom local-pseudopotential cell: 6 Ha, then 10 Ha (32^3) to residual 1e-8
    from paper_1702_04045_gb300 import paro
    lat, pos, _, c = inputs.config_inputs("si8_local")
    ctx = paro.Context(lat, pos, 6.0, 20, 16, "fp64")
    ctx.set_local_pp(**inputs.LOCAL_PP)
    ctx.set_orbitals(inputs.start_vectors(20, ctx.npw(), 1002))
    for _ in range(30):
        ctx.step(2, 0.25, 8)
    ctx.set_ecut(10.0)
    assert ctx.grid == (32, 32, 32) and ctx.npw() == 1647
    for it in range(2000):
        r = ctx.step(2, 0.25, 8)
        if r < 1e-8:
            break
    assert r < 1e-8
    b = pw.Basis(lat, 10.0, ctx.grid)
    ev = np.linalg.eigvalsh(pw.dense_h(b, pw.vloc_real(lat, pos, ctx.grid, 10.0, **inputs.LOCAL_PP)))
    assert np.abs(ctx.eigenvalues()[0][:16] - ev[:16]).max() < 1e-10


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 8e-6)])
def test_scf_after_a_ladder_step_matches_oracle(precision, tol):
    # three SCF iterations at 4 Ha, the ladder step to 7 Ha (input density carried by Fourier
    # interpolation, Pulay history restarted), two more iterations; fixed inner iteration counts
    from paper_1702_04045_gb300 import paro
    lat, pos, d = _cell()
    sys4 = scf.ScfSystem(lat, pos, 4.0, 12, 8, inputs.LOCAL_PP, d, inputs.KB_RC, kpts=[K])
    sys7 = scf.ScfSystem(lat, pos, 7.0, 12, 8, inputs.LOCAL_PP, d, inputs.KB_RC, kpts=[K])
    ctx = _ctx(4.0, precision)
    c0 = inputs.start_vectors(12, ctx.npw(), 23)
    log = []
    with pytest.raises(RuntimeError):
        scf.paro_scf(sys4, [c0], tol=0.0, max_iter=3, eta=0.0, max_inner=3, log=log)
    eps, psi, _ = log[-1]["state"][0]
    rho = ladder.fourier_interpolate(log[-1]["rho_in"], sys7.grid)
    psi7 = ladder.prolong(sys4.bases[0], sys7.bases[0], psi)
    v, _, _ = sys7.veff(rho)
    p7 = opar.ParoProblem(sys7.bases[0], v, sys7.betas[0], d)
    state = [(eps, psi7, p7.h(psi7))]
    occs, _ = sys7.occupations([eps])
    mixer = scf.Pulay(8, 0.7)
    ref = []
    for _ in range(2):
        state, occs, rho, terms = scf.scf_step(sys7, state, occs, rho, mixer, 1, 0.0, 3)
        ref.append(terms["total"])
    ctx.set_orbitals(c0)
    opts = paro.ScfOptions(alg=1, tol_per_atom=0.0, inner_rel_tol=0.0, inner_max_it=3)
    for it in range(3):
        e, _ = ctx.scf_step(opts)
        assert abs(e["total"] - log[it]["energy"]) < tol
    ctx.set_ecut(7.0)
    for it in range(2):
        e, _ = ctx.scf_step(opts)
        print(f"{precision} SCF after the ladder step, iteration {it + 1}: |E_gpu - E_oracle| = "
              f"{abs(e['total'] - ref[it]):.2e} Ha")
        assert abs(e["total"] - ref[it]) < tol
