"""CPU FP64 oracle: plane-wave basis, pseudopotentials and the Kohn-Sham Hamiltonian.

TEST INFRASTRUCTURE ONLY. Only tests, the smoke check and the bench's CPU-baseline leg may import
this package; the product path (libparo.so and its binding) never does. Everything here is plain
NumPy in float64/complex128, written for a reader to check against the paper by eye.

Conventions (Hartree atomic units, Section 2 of the paper):
  * lattice rows a1, a2, a3 (Bohr); reciprocal rows b_i with a_i . b_j = 2 pi delta_ij;
  * G(n) = n1 b1 + n2 b2 + n3 b3 for integer Miller indices n; k given in reduced coordinates;
  * psi(r) = Omega^{-1/2} sum_G c_{k+G} exp(i (k+G).r)                               (Eq. e2);
  * basis = { G : |k+G|^2 / 2 <= E_cut }                                             (Eq. e3),
    stored in lexicographic (n1, n2, n3) order, so every z-column ("stick") is one contiguous run;
  * FFT grid index j = n mod N, C order (j1, j2, j3).

Readings of points the paper leaves open (all listed in the design notes):
  * the potential term of h_mn (Eq. e5) is printed with exp(-i(G_m + G_n).r); it is read as
    exp(-i(G_m - G_n).r), plus the nonlocal term the printed formula omits;
  * the FFT grid is the smallest 2^a 3^b with N_i > m_V,i + s_psi,i, where m_V,i is the largest
    |n_i| of the density sphere |G|^2/2 <= 4 E_cut and s_psi,i the span of n_i over the
    wavefunction sphere of every k: then V.psi computed on the grid is alias free;
  * the divergent -4 pi Z / G^2 part of the local pseudopotential at G = 0 is dropped
    (neutralising background), keeping v(0) = pi Z rc^2 + A pi^{3/2} a^3.
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


def reciprocal(lat: np.ndarray) -> np.ndarray:
    """Rows b_i with a_i . b_j = 2 pi delta_ij (Section 2.2, Bloch / plane-wave setting)."""
    return TWO_PI * np.linalg.inv(np.asarray(lat, dtype=np.float64)).T


def cell_volume(lat: np.ndarray) -> float:
    return abs(float(np.linalg.det(lat)))


def gsphere(lat, ecut, kfrac=(0.0, 0.0, 0.0)):
    """Plane-wave basis of Eq. e3: Miller indices n with |k+G(n)|^2/2 <= ecut.

    Returns (miller (npw,3) int64, q = k+G Cartesian (npw,3), kinetic |q|^2/2 (npw,)) in
    lexicographic (n1, n2, n3) order.
    """
    lat = np.asarray(lat, dtype=np.float64)
    bmat = reciprocal(lat)
    kfrac = np.asarray(kfrac, dtype=np.float64)
    kcart = kfrac @ bmat
    gmax = math.sqrt(2.0 * ecut)
    # |n_i + k_i| = |(k+G).a_i| / (2 pi) <= gmax |a_i| / (2 pi)
    lim = [int(math.floor(gmax * np.linalg.norm(lat[i]) / TWO_PI + abs(kfrac[i]))) + 1 for i in range(3)]
    r = [np.arange(-m, m + 1) for m in lim]
    n = np.stack(np.meshgrid(r[0], r[1], r[2], indexing="ij"), axis=-1).reshape(-1, 3)
    q = kcart[None, :] + n.astype(np.float64) @ bmat
    kin = 0.5 * np.sum(q * q, axis=1)
    keep = kin <= ecut
    n, q, kin = n[keep], q[keep], kin[keep]
    order = np.lexsort((n[:, 2], n[:, 1], n[:, 0]))
    return n[order].astype(np.int64), q[order], kin[order]


def _smooth_235(m: int) -> int:
    """Smallest integer > m whose only prime factors are 2 and 3."""
    x = m + 1
    while True:
        y = x
        for p in (2, 3):
            while y % p == 0:
                y //= p
        if y == 1:
            return x
        x += 1


def fft_grid(lat, ecut, kpts_frac=((0.0, 0.0, 0.0),)):
    """FFT grid (N1, N2, N3) by the alias-free rule stated in the module docstring."""
    dens, _, _ = gsphere(lat, 4.0 * ecut)
    m_v = np.max(np.abs(dens), axis=0)
    span = np.zeros(3, dtype=np.int64)
    for k in kpts_frac:
        n, _, _ = gsphere(lat, ecut, k)
        span = np.maximum(span, n.max(axis=0) - n.min(axis=0))
    return tuple(_smooth_235(int(m_v[i] + span[i])) for i in range(3))


def grid_index(miller: np.ndarray, grid) -> np.ndarray:
    """Flat C-order index of n mod N on the FFT grid."""
    n1, n2, n3 = grid
    j = np.mod(miller, np.array(grid))
    return (j[:, 0] * n2 + j[:, 1]) * n3 + j[:, 2]


def grid_miller(grid) -> np.ndarray:
    """Signed Miller index of every grid point: n = j if 2 j < N else j - N; shape (N1,N2,N3,3)."""
    axes = []
    for nn in grid:
        j = np.arange(nn)
        axes.append(np.where(2 * j < nn, j, j - nn))
    return np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1)


# ----------------------------------------------------------------------------------------------
# Local pseudopotential  v(r) = -Z erf(r/rc)/r + A exp(-(r/a)^2)      (Section 2.2, V_loc)
# ----------------------------------------------------------------------------------------------

def vloc_form(g2: np.ndarray, Z: float, rc: float, A: float, a: float) -> np.ndarray:
    """Fourier transform v(G) = int v(r) exp(-i G.r) d^3r of the local pseudopotential.

    -Z erf(r/rc)/r  ->  -4 pi Z exp(-G^2 rc^2 / 4) / G^2 ;  A exp(-r^2/a^2) -> A pi^{3/2} a^3 exp(-G^2 a^2/4).
    At G = 0 the divergent -4 pi Z / G^2 is dropped, leaving pi Z rc^2 + A pi^{3/2} a^3.
    """
    g2 = np.asarray(g2, dtype=np.float64)
    out = A * math.pi ** 1.5 * a ** 3 * np.exp(-g2 * a * a / 4.0)
    nz = g2 > 0
    coul = np.empty_like(g2)
    coul[nz] = -4.0 * math.pi * Z * np.exp(-g2[nz] * rc * rc / 4.0) / g2[nz]
    coul[~nz] = math.pi * Z * rc * rc
    return out + coul


def vloc_g_on_grid(lat, pos, grid, ecut, Z, rc, A, a):
    """V_loc(G) = Omega^{-1} sum_I exp(-i G.R_I) v(G) on the density sphere |G|^2/2 <= 4 ecut
    (and 2|n_i| < N_i), zero elsewhere; complex array of the grid's shape."""
    lat = np.asarray(lat, dtype=np.float64)
    omega = cell_volume(lat)
    nmil = grid_miller(grid).reshape(-1, 3)
    g = nmil.astype(np.float64) @ reciprocal(lat)
    g2 = np.sum(g * g, axis=1)
    keep = (0.5 * g2 <= 4.0 * ecut) & np.all(2 * np.abs(nmil) < np.array(grid), axis=1)
    sfac = np.exp(-1j * (g[keep] @ np.asarray(pos, dtype=np.float64).T)).sum(axis=1)
    vg = np.zeros(nmil.shape[0], dtype=np.complex128)
    vg[keep] = sfac * vloc_form(g2[keep], Z, rc, A, a) / omega
    return vg.reshape(grid)


def vloc_real(lat, pos, grid, ecut, Z, rc, A, a) -> np.ndarray:
    """V_loc(r_j) = sum_G V_loc(G) exp(i G.r_j) on the grid points r_j = sum_i (j_i/N_i) a_i."""
    vg = vloc_g_on_grid(lat, pos, grid, ecut, Z, rc, A, a)
    n = int(np.prod(grid))
    return np.real(np.fft.ifftn(vg) * n)


# ----------------------------------------------------------------------------------------------
# Kleinman-Bylander nonlocal part  V_nl = sum_{I,j} |beta_Ij> D_{I,l(j)} <beta_Ij|  (Section 2.2)
# ----------------------------------------------------------------------------------------------

def kb_norms(rc: float):
    """Normalisation of p_s = N0 exp(-r^2/rc^2) and p_x = N1 x exp(-r^2/rc^2) to int p^2 = 1."""
    n0 = ((math.pi / 2.0) ** 1.5 * rc ** 3) ** -0.5
    n1 = ((math.pi / 2.0) ** 1.5 * rc ** 5 / 4.0) ** -0.5
    return n0, n1


def kb_beta(lat, pos, q: np.ndarray, rc: float) -> np.ndarray:
    """beta_{Ij}(k+G) = Omega^{-1/2} exp(-i (k+G).R_I) p~_j(k+G), j = s, px, py, pz.

    p~_s(q) = N0 pi^{3/2} rc^3 exp(-q^2 rc^2/4);  p~_x(q) = -i N1 (pi^{3/2} rc^5 / 2) q_x exp(-q^2 rc^2/4).
    Returns (4 * n_atoms, npw) complex; projector index = 4 I + j.
    """
    omega = cell_volume(lat)
    n0, n1 = kb_norms(rc)
    q = np.asarray(q, dtype=np.float64)
    q2 = np.sum(q * q, axis=1)
    gauss = np.exp(-q2 * rc * rc / 4.0)
    ps = n0 * math.pi ** 1.5 * rc ** 3 * gauss
    pp = -1j * n1 * (math.pi ** 1.5 * rc ** 5 / 2.0) * q * gauss[:, None]
    forms = np.concatenate([ps[None, :].astype(np.complex128), pp.T], axis=0)  # (4, npw)
    pos = np.asarray(pos, dtype=np.float64)
    phase = np.exp(-1j * (pos @ q.T))  # (n_atoms, npw)
    beta = phase[:, None, :] * forms[None, :, :] / math.sqrt(omega)
    return beta.reshape(-1, q.shape[0])


def kb_dvec(dstr: np.ndarray) -> np.ndarray:
    """Strength per projector from one strength per (atom, l): (D_s, D_p, D_p, D_p) per atom."""
    dstr = np.asarray(dstr, dtype=np.float64)
    return np.stack([dstr[:, 0], dstr[:, 1], dstr[:, 1], dstr[:, 1]], axis=1).reshape(-1)


# ----------------------------------------------------------------------------------------------
# The Hamiltonian, Eq. e5: h_mn = |k+G_m|^2/2 delta_mn + V~(n_m - n_n) + sum_p beta_p(m) D_p beta_p(n)^*
# ----------------------------------------------------------------------------------------------

class Basis:
    """Basis of one k-point: Miller list, k+G, kinetic, grid indices, and KB table."""

    def __init__(self, lat, ecut, grid, kfrac=(0.0, 0.0, 0.0)):
        self.lat = np.asarray(lat, dtype=np.float64)
        self.ecut = float(ecut)
        self.grid = tuple(int(x) for x in grid)
        self.kfrac = np.asarray(kfrac, dtype=np.float64)
        self.miller, self.q, self.kin = gsphere(self.lat, ecut, kfrac)
        self.idx = grid_index(self.miller, self.grid)
        self.npw = len(self.kin)
        self.omega = cell_volume(self.lat)
        self.ngrid = int(np.prod(self.grid))


def to_real_space(basis: Basis, c: np.ndarray) -> np.ndarray:
    """psi(r_j) * Omega^{1/2} = sum_G c_G exp(2 pi i n.j/N): scatter on the grid, unnormalised inverse DFT.
    c: (nb, npw) -> (nb, N1, N2, N3)."""
    c = np.atleast_2d(c)
    f = np.zeros((c.shape[0], basis.ngrid), dtype=np.complex128)
    f[:, basis.idx] = c
    f = f.reshape((c.shape[0],) + basis.grid)
    return np.fft.ifftn(f, axes=(1, 2, 3)) * basis.ngrid


def from_real_space(basis: Basis, f: np.ndarray) -> np.ndarray:
    """Forward DFT sum_j f_j exp(-2 pi i n.j/N) / N_grid, gathered on the sphere: (nb, grid) -> (nb, npw)."""
    g = np.fft.fftn(f, axes=(1, 2, 3)).reshape(f.shape[0], -1) / basis.ngrid
    return g[:, basis.idx]


def apply_h(basis: Basis, v_r: np.ndarray, psi: np.ndarray, beta=None, dvec=None) -> np.ndarray:
    """H psi through the FFT (Eq. e5 applied as a cyclic convolution on the grid).

    psi: (nb, npw) complex, row = band. Returns (nb, npw).
    """
    psi = np.atleast_2d(np.asarray(psi, dtype=np.complex128))
    out = basis.kin[None, :] * psi
    out = out + from_real_space(basis, to_real_space(basis, psi) * v_r[None])
    if beta is not None:
        proj = np.conj(beta) @ psi.T              # P = beta^H Psi, (nproj, nb)
        out = out + (beta.T @ (dvec[:, None] * proj)).T
    return out


def dense_h(basis: Basis, v_r: np.ndarray, beta=None, dvec=None) -> np.ndarray:
    """The N_pw x N_pw matrix of the grid operator: V~(n) = N^{-1} sum_r V(r) exp(-2 pi i n.r/N)."""
    vt = np.fft.fftn(v_r) / basis.ngrid
    dn = np.mod(basis.miller[:, None, :] - basis.miller[None, :, :], np.array(basis.grid))
    h = vt[dn[..., 0], dn[..., 1], dn[..., 2]].astype(np.complex128)
    h[np.diag_indices(basis.npw)] += basis.kin
    if beta is not None:
        h = h + (beta.T * dvec[None, :]) @ np.conj(beta)
    return h


def galerkin_h_local(basis: Basis, pos, Z, rc, A, a) -> np.ndarray:
    """Exact Galerkin matrix of -Delta/2 + V_loc with V_loc(G_m - G_n) from the closed-form Fourier
    transform (no grid, no FFT). Equals dense_h for a potential band limited to the density sphere."""
    dq = basis.q[:, None, :] - basis.q[None, :, :]
    g2 = np.sum(dq * dq, axis=-1)
    sf = np.zeros(g2.shape, dtype=np.complex128)
    for r in np.asarray(pos, dtype=np.float64):
        sf += np.exp(-1j * (dq @ r))
    h = sf * vloc_form(g2, Z, rc, A, a) / basis.omega
    h[np.diag_indices(basis.npw)] += basis.kin
    return h
