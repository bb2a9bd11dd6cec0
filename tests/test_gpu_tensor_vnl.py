"""Element-wise parity of the nonlocal term V_nl psi = sum_p beta_p D_p <beta_p|psi> (paro_apply_vnl) against
an FP64 product of the same inputs: the FP32 orbitals and the oracle's projectors.

The tensor-core form (3xTF32 with FP32 accumulation in tensor memory, the projectors split once into the
shared-memory image of every pipeline stage) is the product of the inexact inner solves; its relative error
was measured at about 7e-6 on the 64-atom cell and 1.4e-6 on the 8-atom cell, so the bound is 3e-5. The
accurate FP32 form (two-sum carried sums) is held to 2e-6 and the FP64 form to 1e-12. Shapes: odd band
counts and plane-wave counts (rows not 16-byte aligned), several N tiles of the update product, K slices
of the projections, a k-point off Gamma, and the full 64-atom cell (K = 23847, 256 projectors).
"""
import numpy as np
import pytest

from oracle import pw
from paper_1702_04045_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _vnl_ref(beta, dvec, psi):
    proj = np.conj(beta) @ psi.T                   # (nproj, nb)
    return (beta.T @ (dvec[:, None] * proj)).T     # (nb, npw)


def _small(ecut, kfrac, seed):
    from paper_1702_04045_gb300 import paro
    lat, pos = inputs.diamond_cell(1, 10.26, seed)
    d = inputs.kb_strengths(len(pos), seed + 1)
    ctx = paro.Context(lat, pos, ecut, 12, 8, "mixed", kpts=[kfrac])
    ctx.set_local_pp(**inputs.LOCAL_PP)
    ctx.set_kb(inputs.KB_RC, d)
    b = pw.Basis(lat, ecut, pw.fft_grid(lat, ecut, [kfrac]), kfrac)
    return ctx, pw.kb_beta(lat, pos, b.q, inputs.KB_RC), pw.kb_dvec(d), b.npw


@pytest.mark.parametrize("ecut,kfrac,nb", [(4.0, (0, 0, 0), 11), (10.0, (0, 0, 0), 37),
                                           (10.0, (1 / 3, -1 / 3, 0.25), 144), (10.0, (0, 0, 0), 1)])
def test_vnl_forms_match_fp64_product(ecut, kfrac, nb):
    from paper_1702_04045_gb300 import paro
    ctx, beta, dvec, npw = _small(ecut, kfrac, 71)
    assert ctx.npw() == npw
    psi = inputs.start_vectors(nb, npw, 72).astype(np.complex64)
    ref = _vnl_ref(beta, dvec, psi.astype(np.complex128))
    x32 = torch.from_numpy(psi).cuda()
    tc = ctx.apply_vnl(x32, paro.PARO_VNL_TENSOR).cpu().numpy()
    acc = ctx.apply_vnl(x32, paro.PARO_VNL_ACCURATE).cpu().numpy()
    f64 = ctx.apply_vnl(x32.to(torch.complex128), paro.PARO_VNL_ACCURATE).cpu().numpy()
    e_tc, e_acc, e_64 = _rel(tc, ref), _rel(acc, ref), _rel(f64, ref)
    print(f"npw {npw} nb {nb}: tensor cores {e_tc:.2e}, accurate FP32 {e_acc:.2e}, FP64 {e_64:.2e}")
    assert e_tc < 3e-5
    assert e_acc < 2e-6
    assert e_64 < 1e-12
    # the tensor-core call is repeatable (the projector images are formed once)
    tc2 = ctx.apply_vnl(x32, paro.PARO_VNL_TENSOR).cpu().numpy()
    assert np.array_equal(tc, tc2)


def test_vnl_tensor_full_size_64_atoms():
    from paper_1702_04045_gb300 import paro
    ctx = paro.context_from_config("si64_scf", "mixed")
    lat, pos, d, c = inputs.config_inputs("si64_scf")
    b = pw.Basis(lat, c["ecut"], ctx.grid)
    beta = pw.kb_beta(lat, pos, b.q, inputs.KB_RC)
    dvec = pw.kb_dvec(d)
    nb = c["n_bands"]
    psi = inputs.start_vectors(nb, b.npw, 73).astype(np.complex64)
    x32 = torch.from_numpy(psi).cuda()
    tc = ctx.apply_vnl(x32, paro.PARO_VNL_TENSOR).cpu().numpy()
    rows = [0, 1, nb // 2, nb - 1]
    ref = _vnl_ref(beta, dvec, psi[rows].astype(np.complex128))
    e = _rel(tc[rows], ref)
    print(f"64-atom cell, {nb} bands, K = {b.npw}: tensor-core V_nl relative error {e:.2e}")
    assert e < 3e-5


def test_vnl_rejects_tensor_form_in_fp64_and_bad_form():
    from paper_1702_04045_gb300 import paro
    ctx, beta, dvec, npw = _small(4.0, (0, 0, 0), 71)
    x = torch.zeros((3, npw), dtype=torch.complex128, device="cuda")
    with pytest.raises(paro.ParoError):
        ctx.apply_vnl(x, paro.PARO_VNL_TENSOR)
    with pytest.raises(paro.ParoError):
        ctx.apply_vnl(x.to(torch.complex64), 7)
