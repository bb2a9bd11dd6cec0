"""Pins of the oracle's basis, grid and Hamiltonian against closed forms and brute force."""
import math

import numpy as np
import pytest

from oracle import pw
from paper_1702_04045_gb300 import inputs


def _theta_count(radius2: int) -> int:
    """Integer points with n1^2+n2^2+n3^2 <= radius2, from the cube of the theta series
    theta(q) = sum_n q^{n^2} (a polynomial product, independent of sphere enumeration)."""
    m = int(math.isqrt(radius2))
    theta = np.zeros(radius2 + 1, dtype=np.int64)
    for n in range(-m, m + 1):
        theta[n * n] += 1
    t3 = np.convolve(np.convolve(theta, theta)[: radius2 + 1], theta)[: radius2 + 1]
    return int(t3.sum())


@pytest.mark.parametrize("a,ecut", [(10.26, 10.0), (20.52, 15.0), (41.04, 12.0)])
def test_npw_equals_theta_series_count(a, ecut):
    # Eq. e3 at Gamma in a cubic cell: |G|^2/2 = (2 pi/a)^2 |n|^2 / 2 <= ecut.
    lat = np.eye(3) * a
    n, _, kin = pw.gsphere(lat, ecut)
    r2 = int(math.floor(2.0 * ecut / (2 * math.pi / a) ** 2))
    assert len(n) == _theta_count(r2)
    assert np.all(kin <= ecut)


def test_workload_sizes():
    # 8/64/512-atom cells: N_pw 1647 / 23847 / 137059 on 32^3 / 72^3 / 128^3 grids.
    for name, npw, g in [("si8_local", 1647, 32), ("si64_scf", 23847, 72), ("si512", 137059, 128)]:
        lat, pos, _, c = inputs.config_inputs(name)
        assert len(pw.gsphere(lat, c["ecut"])[0]) == npw
        assert pw.fft_grid(lat, c["ecut"]) == (g, g, g)


def test_basis_lexicographic_and_sticks_contiguous():
    lat = np.eye(3) * 10.26
    n, _, _ = pw.gsphere(lat, 10.0, (0.1, -0.2, 0.3))
    key = (n[:, 0] * 1000 + n[:, 1]) * 1000 + n[:, 2]
    assert np.all(np.diff(key) > 0)
    cols = n[:, 0] * 1000 + n[:, 1]
    for c in np.unique(cols):
        z = n[cols == c, 2]
        assert np.all(np.diff(z) == 1)


def test_free_electron_eigenvalues_exact():
    # V = 0, no KB: eigenvalues are exactly |k+G|^2/2 (closed form); first shells at a = 10.26.
    lat = np.eye(3) * 10.26
    b = pw.Basis(lat, 4.0, (24, 24, 24))
    h = pw.dense_h(b, np.zeros(b.grid))
    ev = np.linalg.eigvalsh(h)
    g = (2 * math.pi / 10.26) ** 2 / 2
    assert np.allclose(ev, np.sort(b.kin), atol=1e-13)
    assert abs(ev[0]) < 1e-14
    assert np.allclose(ev[1:7], g, atol=1e-13) and np.allclose(ev[7:19], 2 * g, atol=1e-13)
    assert abs(g - 0.1875147) < 1e-6


def _small_cell(kfrac=(0, 0, 0), ecut=4.0, kb=True, seed=11):
    lat, pos = inputs.diamond_cell(1, 10.26, seed)
    grid = pw.fft_grid(lat, ecut, [kfrac])
    b = pw.Basis(lat, ecut, grid, kfrac)
    v = pw.vloc_real(lat, pos, grid, ecut, **inputs.LOCAL_PP)
    beta = pw.kb_beta(lat, pos, b.q, inputs.KB_RC) if kb else None
    d = inputs.kb_strengths(len(pos), seed + 1) if kb else None
    return lat, pos, b, v, beta, d


@pytest.mark.parametrize("kfrac", [(0, 0, 0), (1 / 3, -1 / 3, 0)])
def test_dense_h_hermitian_and_equals_fft_apply(kfrac):
    lat, pos, b, v, beta, d = _small_cell(kfrac)
    dvec = pw.kb_dvec(d)
    h = pw.dense_h(b, v, beta, dvec)
    assert np.abs(h - h.conj().T).max() < 1e-13
    rng = np.random.default_rng(0)
    psi = rng.standard_normal((3, b.npw)) + 1j * rng.standard_normal((3, b.npw))
    hp = pw.apply_h(b, v, psi, beta, dvec)
    assert np.abs(hp - psi @ h.T).max() < 1e-11 * np.abs(hp).max()
    # <phi, H psi> = conj <psi, H phi>
    a = np.vdot(psi[0], hp[1])
    c = np.vdot(psi[1], hp[0])
    assert abs(a - np.conj(c)) < 1e-11 * abs(a)


def test_grid_operator_equals_closed_form_galerkin():
    # For V_loc band limited to the density sphere the FFT grid operator (grid rule) is alias
    # free and equals the exact Galerkin matrix V_loc(G_m - G_n) built from the closed-form
    # Fourier transform, with no grid at all.
    lat, pos, b, v, _, _ = _small_cell(ecut=5.0, kb=False)
    h_grid = pw.dense_h(b, v)
    h_gal = pw.galerkin_h_local(b, pos, **inputs.LOCAL_PP)
    assert np.abs(h_grid - h_gal).max() < 1e-12


def test_vloc_gaussian_part_matches_real_space_image_sum():
    # Z = 0 leaves A exp(-r^2/a^2): the periodic image sum can be done directly in real space.
    lat, pos = inputs.diamond_cell(1, 10.26, 3)
    grid = (40, 40, 40)   # |n_i| <= 19: exp(-G^2 a^2/4) < 1e-14 beyond the grid's reach
    v = pw.vloc_real(lat, pos, grid, 40.0, Z=0.0, rc=0.8, A=2.0, a=1.0)
    j = np.stack(np.meshgrid(*[np.arange(n) / n for n in grid], indexing="ij"), -1).reshape(-1, 3) @ lat
    sel = np.arange(0, len(j), 37)
    j = j[sel]
    ref = np.zeros(len(j))
    shifts = np.array([[x, y, z] for x in (-1, 0, 1) for y in (-1, 0, 1) for z in (-1, 0, 1)]) @ lat
    for r in pos:
        for s in shifts:
            d = j - r - s
            ref += 2.0 * np.exp(-np.sum(d * d, axis=1))
    assert np.abs(v.reshape(-1)[sel] - ref).max() < 1e-10


def test_vloc_form_short_range_part_by_radial_quadrature():
    # -Z (erf(r/rc) - 1)/r is short ranged; its 3D transform is -4 pi Z (exp(-q^2 rc^2/4) - 1)/q^2.
    from scipy.integrate import quad
    from scipy.special import erf
    Z, rc = 4.0, 0.8
    for q in (0.5, 1.3, 3.0):
        f = lambda r: 4 * math.pi * r * r * (-Z * (erf(r / rc) - 1.0) / r) * math.sin(q * r) / (q * r)
        num = quad(f, 0, 30, limit=400)[0]
        closed = pw.vloc_form(np.array([q * q]), Z, rc, 0.0, 1.0)[0] + 4 * math.pi * Z / q ** 2
        assert abs(num - closed) < 1e-9


def _overlap_closed(pos, lat, i, j, rc):
    """<p_{I a}|p_{J b}> for a, b in (s, x, y, z), summed over periodic images (closed forms)."""
    out = np.zeros((4, 4))
    shifts = np.array([[x, y, z] for x in range(-2, 3) for y in range(-2, 3) for z in range(-2, 3)]) @ lat
    for s in shifts:
        d = pos[j] + s - pos[i]
        e = math.exp(-np.dot(d, d) / (2 * rc * rc))
        m = np.zeros((4, 4))
        m[0, 0] = e
        for a in range(3):
            m[0, 1 + a] = -d[a] / rc * e          # <s_I | a_J>
            m[1 + a, 0] = d[a] / rc * e           # <a_I | s_J>
            for c in range(3):
                m[1 + a, 1 + c] = ((1.0 if a == c else 0.0) - d[a] * d[c] / rc ** 2) * e
        out += m
    return out


def test_kb_projector_overlaps_closed_form():
    # sum_G beta_Ia(G)^* beta_Jb(G) -> int p_Ia p_Jb (Parseval) as E_cut grows: Gaussian products.
    lat, pos = inputs.diamond_cell(1, 10.26, 5)
    b = pw.Basis(lat, 30.0, pw.fft_grid(lat, 30.0))
    beta = pw.kb_beta(lat, pos, b.q, inputs.KB_RC)
    gram = np.conj(beta) @ beta.T
    for (i, j) in [(0, 0), (0, 4), (1, 5), (2, 7)]:
        ref = _overlap_closed(pos, lat, i, j, inputs.KB_RC)
        got = gram[4 * i: 4 * i + 4, 4 * j: 4 * j + 4]
        assert np.abs(got.imag).max() < 1e-10
        assert np.abs(got.real - ref).max() < 1e-8


def test_kb_single_s_channel_interlaces():
    # A rank-one perturbation D |beta><beta| (D > 0) moves every eigenvalue up by at most the next gap.
    lat, pos, b, v, beta, _ = _small_cell(kb=True)
    d = np.zeros(4 * len(pos))
    d[0] = 0.7
    h0 = np.linalg.eigvalsh(pw.dense_h(b, v))
    h1 = np.linalg.eigvalsh(pw.dense_h(b, v, beta, d))
    assert np.all(h1 >= h0 - 1e-12)
    assert np.all(h1[:-1] <= h0[1:] + 1e-12)
    assert abs((h1 - h0).sum() - 0.7 * np.vdot(beta[0], beta[0]).real) < 1e-10


def test_translation_invariance_of_spectrum():
    lat, pos, b, v, beta, d = _small_cell()
    t = np.array([0.37, -1.1, 2.3])
    v2 = pw.vloc_real(lat, pos + t, b.grid, b.ecut, **inputs.LOCAL_PP)
    beta2 = pw.kb_beta(lat, pos + t, b.q, inputs.KB_RC)
    dv = pw.kb_dvec(d)
    e1 = np.linalg.eigvalsh(pw.dense_h(b, v, beta, dv))
    e2 = np.linalg.eigvalsh(pw.dense_h(b, v2, beta2, dv))
    assert np.abs(e1 - e2).max() < 1e-11
