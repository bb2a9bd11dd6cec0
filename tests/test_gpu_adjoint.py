"""GPU parity of the adjoint of H psi (paro_apply_h_adjoint, paro_set_positions and the autograd
wrapper) against the FP64 CPU oracle (oracle/adjoint.py) on the same seeded inputs.

Tolerances: FP64 (complex128 inputs) to rounding, 1e-11 relative to the largest entry of each
output; FP32 (complex64 inputs) 2e-5 relative (FP32 FFTs and 3xTF32 tensor-core projections)."""
import numpy as np
import pytest

from oracle import adjoint, pw
from paper_1702_04045_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _case(ecut=10.0, kb=True, nb=6, seed=71, kfrac=(0.0, 0.0, 0.0)):
    from paper_1702_04045_gb300 import paro
    lat, pos = inputs.diamond_cell(1, 10.26, seed)
    d = inputs.kb_strengths(len(pos), seed + 1) if kb else None
    ctx = paro.Context(lat, pos, ecut, nb, nb, "fp64", kpts=[kfrac])
    ctx.set_local_pp(**inputs.LOCAL_PP)
    if kb:
        ctx.set_kb(inputs.KB_RC, d)
    grid = ctx.grid
    basis = pw.Basis(lat, ecut, grid, kfrac)
    rng = np.random.default_rng(seed + 2)
    v_rest = 0.2 * rng.standard_normal(grid)
    ctx.set_veff(ctx.get_vloc() + v_rest)
    psi = inputs.start_vectors(nb, basis.npw, seed + 3)
    w = inputs.start_vectors(nb, basis.npw, seed + 4)
    kbx = (inputs.KB_RC, d) if kb else None
    return ctx, basis, pos, psi, w, v_rest, kbx


@pytest.mark.parametrize("kb", [False, True])
@pytest.mark.parametrize("kfrac", [(0, 0, 0), (0.25, -1 / 3, 1 / 3)])
def test_adjoint_fp64_matches_oracle(kb, kfrac):
    ctx, basis, pos, psi, w, v_rest, kbx = _case(kb=kb, kfrac=kfrac)
    g_psi, g_v, g_pos = ctx.apply_h_adjoint(torch.from_numpy(psi).cuda(), torch.from_numpy(w).cuda())
    r_psi, r_v, r_pos = adjoint.hpsi_vjp(basis, v_rest, pos, inputs.LOCAL_PP, psi, w, kbx)
    assert _rel(g_psi.cpu().numpy(), r_psi) < 1e-11
    assert _rel(g_v.cpu().numpy(), r_v) < 1e-11
    assert _rel(g_pos.cpu().numpy(), r_pos) < 1e-10


def test_adjoint_fp32_matches_oracle():
    ctx, basis, pos, psi, w, v_rest, kbx = _case()
    g_psi, g_v, g_pos = ctx.apply_h_adjoint(torch.from_numpy(psi.astype(np.complex64)).cuda(),
                                            torch.from_numpy(w.astype(np.complex64)).cuda())
    r_psi, r_v, r_pos = adjoint.hpsi_vjp(basis, v_rest, pos, inputs.LOCAL_PP, psi, w, kbx)
    assert _rel(g_psi.cpu().numpy(), r_psi) < 2e-5
    assert _rel(g_v.cpu().numpy(), r_v) < 2e-5
    assert _rel(g_pos.cpu().numpy(), r_pos) < 2e-5


def test_adjoint_partial_outputs_and_no_pp():
    # outputs may be skipped; without a local pseudopotential the position gradient is the KB part only
    from paper_1702_04045_gb300 import paro
    lat, pos = inputs.diamond_cell(1, 10.26, 73)
    d = inputs.kb_strengths(len(pos), 74)
    ctx = paro.Context(lat, pos, 6.0, 3, 3, "fp64")
    ctx.set_kb(inputs.KB_RC, d)
    grid = ctx.grid
    v = 0.1 * np.random.default_rng(75).standard_normal(grid)
    ctx.set_veff(v)
    basis = pw.Basis(lat, 6.0, grid)
    psi = inputs.start_vectors(3, basis.npw, 76)
    w = inputs.start_vectors(3, basis.npw, 77)
    tp, tw = torch.from_numpy(psi).cuda(), torch.from_numpy(w).cuda()
    g_psi, g_v, g_pos = ctx.apply_h_adjoint(tp, tw, grads=("pos",))
    assert g_psi is None and g_v is None
    ref = adjoint.grad_pos_kb(basis, pos, (inputs.KB_RC, d), psi, w)
    assert _rel(g_pos.cpu().numpy(), ref) < 1e-10
    _, g_v2, _ = ctx.apply_h_adjoint(tp, tw, grads=("v",))
    assert _rel(g_v2.cpu().numpy(), adjoint.grad_v(basis, psi, w)) < 1e-11


def test_set_positions_rebuilds_h_keeping_v_rest():
    ctx, basis, pos, psi, w, v_rest, kbx = _case(nb=4)
    pos2 = pos + np.random.default_rng(81).uniform(-0.1, 0.1, pos.shape)
    ctx.set_positions(pos2)
    got = ctx.apply_h(torch.from_numpy(psi).cuda()).cpu().numpy()
    v_r, beta, dvec = adjoint.hamiltonian_parts(basis, v_rest, pos2, inputs.LOCAL_PP, kbx)
    assert _rel(got, pw.apply_h(basis, v_r, psi, beta, dvec)) < 1e-12
    assert np.abs(ctx.get_veff() - v_r).max() < 1e-12 * np.abs(v_r).max()


def test_autograd_wrapper_gradients():
    from paper_1702_04045_gb300 import paro
    ctx, basis, pos, psi, w, v_rest, kbx = _case(nb=3)
    tpsi = torch.from_numpy(psi).cuda().requires_grad_(True)
    tv = torch.from_numpy(v_rest).cuda().requires_grad_(True)
    tpos = torch.from_numpy(pos.copy()).cuda().requires_grad_(True)
    tw = torch.from_numpy(w).cuda()
    y = paro.hpsi(ctx, tpsi, tv, tpos)
    loss = torch.real(torch.sum(torch.conj(tw) * y))
    loss.backward()
    r_psi, r_v, r_pos = adjoint.hpsi_vjp(basis, v_rest, pos, inputs.LOCAL_PP, psi, w, kbx)
    assert _rel(tpsi.grad.cpu().numpy(), r_psi) < 1e-11
    assert _rel(tv.grad.cpu().numpy(), r_v) < 1e-11
    assert _rel(tpos.grad.cpu().numpy(), r_pos) < 1e-10
    # the forward pass alone against central differences of the GPU forward in one coordinate
    h = 1e-4

    def lval(p):
        with torch.no_grad():
            yy = paro.hpsi(ctx, tpsi.detach(), tv.detach(), torch.from_numpy(p).cuda())
            return float(torch.real(torch.sum(torch.conj(tw) * yy)))

    pp, pm = pos.copy(), pos.copy()
    pp[2, 1] += h
    pm[2, 1] -= h
    fd = (lval(pp) - lval(pm)) / (2 * h)
    assert abs(fd - r_pos[2, 1]) < 1e-6 * np.abs(r_pos).max()


@pytest.mark.parametrize("precision_dtype,tol", [(np.complex128, 1e-11), (np.complex64, 2e-5)])
def test_adjoint_full_size_64_atoms(precision_dtype, tol):
    # 64-atom cell, 23847 plane waves, KB projectors: dL/dV element-wise against the oracle, the V_loc
    # and KB position gradients of two atoms against the oracle, and the translation identity
    # sum_I dL/dR_Ia = Re sum conj(W) (-i q_a H Psi + i H (q_a Psi)) (V_eff = V_loc) through H psi.
    from paper_1702_04045_gb300 import paro
    name = "si64_scf"
    lat, pos, d, c = inputs.config_inputs(name)
    ctx = paro.context_from_config(name, "fp64")
    grid = ctx.grid
    basis = pw.Basis(lat, c["ecut"], grid)
    nb = 8
    psi = inputs.start_vectors(nb, basis.npw, 91)
    w = inputs.start_vectors(nb, basis.npw, 92)
    tp = torch.from_numpy(psi.astype(precision_dtype)).cuda()
    tw = torch.from_numpy(w.astype(precision_dtype)).cuda()
    g_psi, g_v, g_pos = ctx.apply_h_adjoint(tp, tw)
    g_v, g_pos = g_v.cpu().numpy(), g_pos.cpu().numpy()
    assert _rel(g_v, adjoint.grad_v(basis, psi, w)) < tol
    atoms = [5, 40]
    ref = adjoint.grad_pos_local(basis, pos, inputs.LOCAL_PP, adjoint.grad_v(basis, psi, w))
    ref = ref + adjoint.grad_pos_kb(basis, pos, (inputs.KB_RC, d), psi, w, atoms=atoms)
    assert _rel(g_pos[atoms], ref[atoms]) < max(tol, 1e-10) * np.abs(ref).max() / np.abs(ref[atoms]).max()
    # dL/dpsi = H W: bit for bit in FP64; in FP32 the adjoint's projector products run on the tensor cores
    assert _rel(g_psi.cpu().numpy(), ctx.apply_h(tw).cpu().numpy()) < (1e-13 if precision_dtype == np.complex128 else tol)
    q = torch.from_numpy(basis.q).cuda().to(tp.real.dtype)
    hp = ctx.apply_h(tp)
    for al in range(3):
        hq = ctx.apply_h(q[:, al][None, :] * tp)
        want = torch.real(torch.sum(torch.conj(tw) * (-1j * q[:, al][None, :] * hp + 1j * hq))).item()
        assert g_pos[:, al].sum() == pytest.approx(want, rel=max(tol, 1e-9), abs=tol * np.abs(g_pos).max())


def test_hellmann_feynman_density_8_atoms():
    # For orbitals of the 8-atom workload after ParO steps, W = 2 Psi_occ gives L = E_band and
    # dE_band/dV(r) = rho(r) Omega / N: the adjoint's dL/dV against the library's density pass.
    from paper_1702_04045_gb300 import paro
    name = "si8_local"
    lat, pos, _, c = inputs.config_inputs(name)
    ctx = paro.context_from_config(name, "fp64")
    ctx.set_orbitals(inputs.start_vectors(c["n_bands"], ctx.npw(), c["seed_psi"]))
    for _ in range(30):
        ctx.step(1, 0.25, 8)
    psi = ctx.get_orbitals(device=True)[: c["n_occ"]].contiguous()
    _, g_v, _ = ctx.apply_h_adjoint(psi, 2.0 * psi, grads=("v",))
    omega = abs(np.linalg.det(lat))
    n = int(np.prod(ctx.grid))
    rho = ctx.density().cpu().numpy()
    assert _rel(g_v.cpu().numpy() * n / omega, rho) < 1e-12


def test_adjoint_512_atoms_forces_central_differences():
    # 512-atom cell (137059 plane waves, 128^3 grid, 2048 KB projectors), FP32 adjoint: forces on 8 seeded
    # atoms against central differences (h = 1e-4 Bohr) of the FP64 oracle's L. Only the moved atom's
    # terms of L change: sum_r V_loc,I(r) dL/dV(r) with its single-atom local potential, and
    # Re sum_b sum_{p in I} D_p conj(A_pb) P_pb with its four projectors.
    from paper_1702_04045_gb300 import paro
    name = "si512"
    lat, pos, d, c = inputs.config_inputs(name)
    ctx = paro.context_from_config(name, "mixed")
    grid = ctx.grid
    basis = pw.Basis(lat, c["ecut"], grid)
    assert basis.npw == 137059 and grid == (128, 128, 128)
    nb = 16
    psi = inputs.start_vectors(nb, basis.npw, 5121)
    w = inputs.start_vectors(nb, basis.npw, 5122)
    _, g_v_gpu, g_pos = ctx.apply_h_adjoint(torch.from_numpy(psi.astype(np.complex64)).cuda(),
                                            torch.from_numpy(w.astype(np.complex64)).cuda(), grads=("v", "pos"))
    g_pos = g_pos.cpu().numpy()
    g_v = adjoint.grad_v(basis, psi, w)
    assert _rel(g_v_gpu.cpu().numpy(), g_v) < 2e-5
    dvec = pw.kb_dvec(d)
    rng = np.random.default_rng(5123)
    atoms = rng.choice(len(pos), 8, replace=False)
    axes = rng.integers(0, 3, 8)

    def l_atom(i_at, r):
        v_i = pw.vloc_real(lat, r[None], grid, c["ecut"], **inputs.LOCAL_PP)
        beta = pw.kb_beta(lat, r[None], basis.q, inputs.KB_RC)
        proj, aproj = np.conj(beta) @ psi.T, np.conj(beta) @ w.T
        dv = dvec[4 * i_at:4 * i_at + 4]
        return float(np.sum(v_i * g_v)) + float(np.real(np.sum(dv[:, None] * np.conj(aproj) * proj)))

    h = 1e-4
    scale = np.abs(g_pos).max()
    for i_at, al in zip(atoms, axes):
        rp, rm = pos[i_at].copy(), pos[i_at].copy()
        rp[al] += h
        rm[al] -= h
        fd = (l_atom(i_at, rp) - l_atom(i_at, rm)) / (2 * h)
        assert abs(fd - g_pos[i_at, al]) < 2e-5 * scale
