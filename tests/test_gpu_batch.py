"""GPU parity of the batched path (paro_batch_*): one persistent H psi launch over the orbitals of many
uneven problems, and one ParO step per CUDA graph, against the FP64 CPU oracle and against the
per-context calls on the same seeded inputs.

Tolerances as for the per-context path: FP64 H psi 1e-12 relative, eigenvalues 1e-10 Ha; FP32 (mixed)
H psi 2e-6 relative, eigenvalues 1e-6 Ha."""
import numpy as np
import pytest

from oracle import paro as opar
from oracle import pw
from paper_1702_04045_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _contexts(cells, precision, kb_seed=None, set_orbitals=True):
    from paper_1702_04045_gb300 import paro
    ctxs = []
    for i, c in enumerate(cells):
        ctx = paro.Context(c["lat"], c["pos"], c["ecut"], c["n_bands"], c["n_occ"], precision, kpts=c["kpts"],
                           kweights=c["kweights"])
        ctx.set_local_pp(**inputs.LOCAL_PP)
        if kb_seed is not None:
            ctx.set_kb(inputs.KB_RC, inputs.kb_strengths(len(c["pos"]), kb_seed + i))
        if set_orbitals:
            for ik in range(len(c["kpts"])):
                ctx.set_orbitals(inputs.start_vectors(c["n_bands"], ctx.npw(ik), c["seeds"][ik]), ik)
        ctxs.append(ctx)
    return ctxs


def _mixed_cells():
    # 3 k-points of the 8-atom cell at a lower cutoff and 3 of the random cells: uneven grids and N_pw
    m = inputs.batch_inputs("si8_mp27")[0]
    km = dict(m, ecut=6.0, kpts=m["kpts"][[0, 7, 19]], kweights=np.full(3, 1 / 3), seeds=m["seeds"][:3])
    return [km] + inputs.batch_inputs("cells64", limit=3)


@pytest.mark.parametrize("precision,dtype,tol", [("fp64", np.complex128, 1e-12), ("mixed", np.complex64, 2e-6)])
@pytest.mark.parametrize("kb", [False, True])
def test_batch_apply_h_matches_oracle(precision, dtype, tol, kb):
    from paper_1702_04045_gb300 import paro
    cells = _mixed_cells()
    ctxs = _contexts(cells, precision, kb_seed=900 if kb else None, set_orbitals=False)
    b = paro.Batch(ctxs)
    info = b.info()
    assert info["problems"] == 3 + 3 and info["items"] == 6 * 20
    psis, refs = [], []
    for ci, c in enumerate(cells):
        grid = ctxs[ci].grid
        v = pw.vloc_real(c["lat"], c["pos"], grid, c["ecut"], **inputs.LOCAL_PP)
        for ik, k in enumerate(c["kpts"]):
            basis = pw.Basis(c["lat"], c["ecut"], grid, k)
            beta = pw.kb_beta(c["lat"], c["pos"], basis.q, inputs.KB_RC) if kb else None
            dvec = pw.kb_dvec(inputs.kb_strengths(len(c["pos"]), 900 + ci)) if kb else None
            psi = inputs.start_vectors(c["n_bands"], basis.npw, 700 + 10 * ci + ik)
            psis.append(torch.from_numpy(psi.astype(dtype)).cuda())
            refs.append(pw.apply_h(basis, v, psi, beta, dvec))
    outs = b.apply_h(psis)
    for got, ref in zip(outs, refs):
        assert _rel(got.cpu().numpy(), ref) < tol
    b.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 2e-6)])
def test_batch_step_matches_per_context_step(precision, tol):
    # the same problems stepped by the per-context calls and by one batched, graph-captured step
    from paper_1702_04045_gb300 import paro
    cells = _mixed_cells() if precision == "mixed" else _mixed_cells()[:1]
    ref = _contexts(cells, precision)
    bat = _contexts(cells, precision)
    b = paro.Batch(bat)
    for _ in range(3):
        r_ref = max(c.step(1, 0.25, 8) for c in ref)
        r_bat = b.step(0.25, 8)
    for cr, cb in zip(ref, bat):
        assert np.abs(cr.eigenvalues() - cb.eigenvalues()).max() < tol
    assert r_bat == pytest.approx(r_ref, rel=1e-3)
    info = b.info()
    assert info["kernels_per_step"] > 0
    b.close()


def test_batch_step_matches_oracle_step():
    # one batched step of two k-points against the oracle's Algorithm 1 step from the same start
    from paper_1702_04045_gb300 import paro
    m = inputs.batch_inputs("si8_mp27")[0]
    cell = dict(m, ecut=5.0, kpts=m["kpts"][[3, 11]], kweights=np.full(2, 0.5), seeds=m["seeds"][:2])
    ctx = _contexts([cell], "fp64")[0]
    grid = ctx.grid
    start = [ctx.get_orbitals(ik) for ik in range(2)]
    eps0 = ctx.eigenvalues()
    b = paro.Batch([ctx])
    b.step(0.0, 4)
    v = pw.vloc_real(cell["lat"], cell["pos"], grid, cell["ecut"], **inputs.LOCAL_PP)
    for ik in range(2):
        basis = pw.Basis(cell["lat"], cell["ecut"], grid, cell["kpts"][ik])
        prob = opar.ParoProblem(basis, v, None, None)
        eps, psi, _, _ = opar.paro_step_alg1(prob, start[ik], eps0[ik], 0.0, 4)
        assert np.abs(ctx.eigenvalues()[ik] - eps).max() < 1e-10
        g = ctx.get_orbitals(ik)[:8]
        assert np.abs(g.T @ g.conj() - psi[:8].T @ psi[:8].conj()).max() < 1e-9
    b.close()


def test_batch_mp27_converges_to_dense_eigenvalues():
    # 8-atom cell on the 3x3x3 Monkhorst-Pack mesh (27 problems), FP64, to residual 1e-8
    from paper_1702_04045_gb300 import paro
    cell = inputs.batch_inputs("si8_mp27")[0]
    ctx = _contexts([cell], "fp64")[0]
    b = paro.Batch([ctx])
    assert b.info()["problems"] == 27
    for _ in range(3000):
        r = b.step(0.25, 8)
        if r < 1e-8:
            break
    assert r < 1e-8
    grid = ctx.grid
    v = pw.vloc_real(cell["lat"], cell["pos"], grid, cell["ecut"], **inputs.LOCAL_PP)
    for ik in [0, 13, 26]:
        basis = pw.Basis(cell["lat"], cell["ecut"], grid, cell["kpts"][ik])
        ev = np.linalg.eigvalsh(pw.dense_h(basis, v))
        assert np.abs(ctx.eigenvalues()[ik][:16] - ev[:16]).max() < 1e-10
    b.close()


def test_batch_cells64_mixed_matches_dense_eigenvalues():
    # 64 cells of uneven size, mixed precision: occupied eigenvalues of two cells within 1e-6 Ha of
    # the FP64 dense diagonalisation
    from paper_1702_04045_gb300 import paro
    cells = inputs.batch_inputs("cells64")
    ctxs = _contexts(cells, "mixed")
    b = paro.Batch(ctxs)
    info = b.info()
    assert info["problems"] == 64 and info["items"] == 64 * 20
    for _ in range(600):
        r = b.step(0.25, 8)
        if r < 1e-5:
            break
    for ci in [0, int(np.argmax([c["ecut"] for c in cells]))]:
        c = cells[ci]
        grid = ctxs[ci].grid
        basis = pw.Basis(c["lat"], c["ecut"], grid)
        v = pw.vloc_real(c["lat"], c["pos"], grid, c["ecut"], **inputs.LOCAL_PP)
        ev = np.linalg.eigvalsh(pw.dense_h(basis, v))
        assert np.abs(ctxs[ci].eigenvalues()[0][:16] - ev[:16]).max() < 1e-6
    b.close()


def test_batch_rejects_mismatched_contexts():
    from paper_1702_04045_gb300 import paro
    cells = _mixed_cells()[:2]
    a = _contexts(cells[:1], "fp64", set_orbitals=False)
    m = _contexts(cells[1:], "mixed", set_orbitals=False)
    with pytest.raises(paro.ParoError):
        paro.Batch(a + m)


def test_batch_autotuner_table_and_every_unit_shape():
    # the autotuner times unit shapes x launch forms x grids; the batch then runs the fastest. Each shape it
    # kept is checked against the oracle by the tests above; here the table is complete and its minimum is
    # the configuration in use
    from paper_1702_04045_gb300 import paro
    cells = _mixed_cells()
    ctxs = _contexts(cells, "mixed")
    b = paro.Batch(ctxs)
    tun = b.tuning()
    assert len(tun) >= 9
    assert set(tun[:, 2].astype(int)) <= {32, 64, 128} and set(tun[:, 3].astype(int)) <= {2048, 4096, 8192}
    best = tun[int(np.argmin(tun[:, 4]))]
    info = b.info()
    assert info["launches_per_apply"] == int(best[0]) and info["grid"] == int(best[1])
    print("batch autotuner: best", best.tolist(), "of", len(tun), "candidates")
