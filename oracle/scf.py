"""CPU FP64 oracle: density, Hartree, LDA exchange-correlation, Pulay mixing, Ewald, energies, and
the ParO-merged SCF loop (Section 2.3 and Algorithm 1).

TEST INFRASTRUCTURE ONLY (see oracle/pw.py). Plain NumPy/SciPy in float64/complex128.

Readings of points the paper leaves open:
  * rho = sum_k w_k sum_i f_i |psi_ik|^2 with f = 2 for the lowest n_occ bands (spin unpolarised;
    the paper writes rho = sum |psi_i|^2) and w_k = 1/N_k (the paper's w_s = Omega_BZ/N_k belongs
    to the integral form);
  * exchange-correlation: LDA with the Perdew-Zunger (1981) fit of the Ceperley-Alder correlation
    energy, unpolarised (the paper only says E_xc is approximated);
  * mixing: Pulay/DIIS on R = rho_out - rho_in, depth 8, beta = 0.7 (the paper used modified
    Broyden; the workload definition fixes Pulay);
  * energy: E = sum f <psi|T + V_nl|psi> + int V_loc rho + E_H + E_xc + E_Ewald (the paper's
    functional lists neither the nonlocal nor the ion-ion term); the G = 0 terms of V_loc, V_H and
    the Ewald sum follow the neutralising-background convention;
  * one ParO iteration is one SCF iteration: V^n from rho_in^n drives the source solves; the
    density of the Cholesky-orthonormalised solutions is mixed into rho_in^{n+1/2}, whose potential
    drives the Rayleigh-Ritz step (Algorithm 1, step 4); rho_in^{n+1} := rho_in^{n+1/2};
  * convergence: |E^{n+1} - E^n| / N_atom below tol on two consecutive iterations;
  * initial density: uniform N_e / Omega;
  * occupations with smearing (kT > 0; the paper is silent, and a cell whose highest occupied and
    lowest empty levels cross has no fixed point at integer occupations): Fermi-Dirac
    f_ik = 2 / (1 + exp((eps_ik - mu)/kT)) over all n_bands, mu fixed by sum_k w_k sum_i f_ik = 2 n_occ,
    and the energy is the Mermin free energy E - T S, S = -sum_k w_k sum_i 2 [g ln g + (1-g) ln(1-g)],
    g = f/2. Within an iteration the source solutions x_i carry the occupations of the eps_i^n they
    were solved with; the Rayleigh-Ritz result carries those of its own Ritz values.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special as sps

from . import paro, pw


# ----------------------------------------------------------------------------------------------
# Density (Section 2.1: rho = sum |psi_i|^2; Section 2.2: k-point weights)
# ----------------------------------------------------------------------------------------------

def density(basis: pw.Basis, psi: np.ndarray, occ: np.ndarray, weight: float = 1.0) -> np.ndarray:
    """rho(r_j) = weight * sum_i occ_i |psi_i(r_j)|^2, psi_i(r) = Omega^{-1/2} sum_G c exp(i(k+G).r)."""
    fr = pw.to_real_space(basis, psi)
    return weight * np.einsum("i,ixyz->xyz", occ, np.abs(fr) ** 2) / basis.omega


def grid_g2(lat, grid) -> np.ndarray:
    """|G|^2 of every grid point with the signed index n = j if 2j < N else j - N."""
    g = pw.grid_miller(grid).reshape(-1, 3).astype(np.float64) @ pw.reciprocal(lat)
    return np.sum(g * g, axis=1).reshape(grid)


# ----------------------------------------------------------------------------------------------
# Hartree (Section 2.1, V_H and E_H): V_H(G) = 4 pi rho(G) / G^2, G != 0
# ----------------------------------------------------------------------------------------------

def hartree(lat, grid, rho: np.ndarray):
    """Returns (V_H(r), E_H) with E_H = (Omega/2) sum_{G != 0} 4 pi |rho(G)|^2 / G^2."""
    omega = pw.cell_volume(lat)
    n = int(np.prod(grid))
    rho_g = np.fft.fftn(rho) / n
    g2 = grid_g2(lat, grid)
    vh_g = np.zeros_like(rho_g)
    nz = g2 > 0
    vh_g[nz] = 4.0 * math.pi * rho_g[nz] / g2[nz]
    vh = np.real(np.fft.ifftn(vh_g) * n)
    eh = 0.5 * omega * float(np.sum(4.0 * math.pi * np.abs(rho_g[nz]) ** 2 / g2[nz]))
    return vh, eh


# ----------------------------------------------------------------------------------------------
# LDA exchange-correlation, Perdew-Zunger 1981 parametrisation (unpolarised)
# ----------------------------------------------------------------------------------------------

PZ_GAMMA, PZ_BETA1, PZ_BETA2 = -0.1423, 1.0529, 0.3334
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116
RHO_MIN = 1e-30


def lda_pz(rho: np.ndarray):
    """Energy per electron eps_xc(rho) and potential v_xc = d(rho eps_xc)/d rho; zero where rho < 1e-30.

    Exchange: eps_x = -(3/4)(3 rho/pi)^{1/3}, v_x = (4/3) eps_x.
    Correlation, r_s = (3/(4 pi rho))^{1/3}:
      r_s >= 1: eps_c = gamma / (1 + beta1 sqrt(r_s) + beta2 r_s),
                v_c = eps_c (1 + 7/6 beta1 sqrt(r_s) + 4/3 beta2 r_s) / (1 + beta1 sqrt(r_s) + beta2 r_s);
      r_s <  1: eps_c = A ln r_s + B + C r_s ln r_s + D r_s,
                v_c = A ln r_s + (B - A/3) + 2/3 C r_s ln r_s + (2D - C)/3 r_s.
    """
    rho = np.asarray(rho, dtype=np.float64)
    eps = np.zeros_like(rho)
    v = np.zeros_like(rho)
    m = rho >= RHO_MIN
    r = rho[m]
    ex = -0.75 * np.cbrt(3.0 * r / math.pi)
    vx = 4.0 / 3.0 * ex
    rs = np.cbrt(3.0 / (4.0 * math.pi * r))
    ec = np.empty_like(r)
    vc = np.empty_like(r)
    hi = rs >= 1.0
    s = np.sqrt(rs[hi])
    den = 1.0 + PZ_BETA1 * s + PZ_BETA2 * rs[hi]
    ec[hi] = PZ_GAMMA / den
    vc[hi] = ec[hi] * (1.0 + 7.0 / 6.0 * PZ_BETA1 * s + 4.0 / 3.0 * PZ_BETA2 * rs[hi]) / den
    lo = ~hi
    lr = np.log(rs[lo])
    ec[lo] = PZ_A * lr + PZ_B + PZ_C * rs[lo] * lr + PZ_D * rs[lo]
    vc[lo] = PZ_A * lr + (PZ_B - PZ_A / 3.0) + 2.0 / 3.0 * PZ_C * rs[lo] * lr + (2.0 * PZ_D - PZ_C) / 3.0 * rs[lo]
    eps[m] = ex + ec
    v[m] = vx + vc
    return eps, v


# ----------------------------------------------------------------------------------------------
# Ewald energy of point ions in a neutralising background (ion-ion term of the total energy)
# ----------------------------------------------------------------------------------------------

def ewald(lat, pos, charges, eta: float | None = None, tol: float = 1e-16) -> float:
    """E = 1/2 sum_{I,J,L}' Z_I Z_J erfc(eta d)/d + (2 pi/Omega) sum_{G != 0} |S(G)|^2 exp(-G^2/4eta^2)/G^2
           - eta/sqrt(pi) sum Z_I^2 - pi (sum Z_I)^2 / (2 Omega eta^2),   S(G) = sum_I Z_I exp(i G.R_I)."""
    lat = np.asarray(lat, dtype=np.float64)
    pos = np.asarray(pos, dtype=np.float64)
    z = np.asarray(charges, dtype=np.float64) * np.ones(len(pos))
    omega = pw.cell_volume(lat)
    if eta is None:
        eta = math.sqrt(math.pi) / omega ** (1.0 / 3.0)
    # real space: erfc(eta R)/R < tol
    rcut = 1.0
    while math.erfc(eta * rcut) / rcut > tol:
        rcut *= 1.2
    nmax = [int(math.ceil(rcut / (omega / np.linalg.norm(np.cross(lat[(i + 1) % 3], lat[(i + 2) % 3]))))) + 1
            for i in range(3)]
    e_real = 0.0
    rng = [np.arange(-m, m + 1) for m in nmax]
    lvec = np.stack(np.meshgrid(*rng, indexing="ij"), axis=-1).reshape(-1, 3).astype(np.float64) @ lat
    for i in range(len(pos)):
        d = pos[i][None, None, :] - pos[None, :, :] + lvec[:, None, :]   # (L, J, 3)
        dist = np.linalg.norm(d, axis=-1)
        ok = (dist > 1e-12) & (dist < rcut)
        e_real += 0.5 * z[i] * float(np.sum((z[None, :] * sps.erfc(eta * dist) / np.where(ok, dist, 1.0))[ok]))
    # reciprocal space: exp(-G^2/4eta^2)/G^2 < tol
    gcut = 2.0 * eta * math.sqrt(-math.log(tol))
    bmat = pw.reciprocal(lat)
    gm = [int(math.ceil(gcut * np.linalg.norm(lat[i]) / (2 * math.pi))) + 1 for i in range(3)]
    rng = [np.arange(-m, m + 1) for m in gm]
    g = np.stack(np.meshgrid(*rng, indexing="ij"), axis=-1).reshape(-1, 3).astype(np.float64) @ bmat
    g2 = np.sum(g * g, axis=1)
    ok = (g2 > 0) & (g2 < gcut * gcut)
    g, g2 = g[ok], g2[ok]
    sfac = np.exp(1j * (g @ pos.T)) @ z
    e_rec = 2.0 * math.pi / omega * float(np.sum(np.abs(sfac) ** 2 * np.exp(-g2 / (4 * eta * eta)) / g2))
    e_self = -eta / math.sqrt(math.pi) * float(np.sum(z * z))
    e_bg = -math.pi * float(np.sum(z)) ** 2 / (2.0 * omega * eta * eta)
    return e_real + e_rec + e_self + e_bg


# ----------------------------------------------------------------------------------------------
# Pulay (DIIS) density mixing (Section 2.3, step 5)
# ----------------------------------------------------------------------------------------------

class Pulay:
    """rho_new = sum_i a_i (rho_in^i + beta R^i), a minimising ||sum_i a_i R^i||_2 with sum a_i = 1,
    over the last `depth` pairs (rho_in^i, R^i = rho_out^i - rho_in^i)."""

    def __init__(self, depth: int = 8, beta: float = 0.7):
        self.depth, self.beta = depth, beta
        self.rin, self.res = [], []

    def mix(self, rho_in: np.ndarray, rho_out: np.ndarray) -> np.ndarray:
        self.rin.append(rho_in.copy())
        self.res.append(rho_out - rho_in)
        if len(self.rin) > self.depth:
            self.rin.pop(0)
            self.res.pop(0)
        m = len(self.res)
        bmat = np.zeros((m + 1, m + 1))
        for i in range(m):
            for j in range(m):
                bmat[i, j] = float(np.sum(self.res[i] * self.res[j]))
        bmat[:m, m] = 1.0
        bmat[m, :m] = 1.0
        rhs = np.zeros(m + 1)
        rhs[m] = 1.0
        coef = np.linalg.lstsq(bmat, rhs, rcond=None)[0][:m]
        return sum(coef[i] * (self.rin[i] + self.beta * self.res[i]) for i in range(m))


# ----------------------------------------------------------------------------------------------
# Fermi-Dirac occupations (fractional occupations for cells without a gap at the Fermi level)
# ----------------------------------------------------------------------------------------------

def fermi_occupations(eps_list, kw, n_el: float, kT: float):
    """f_ik = 2 g((eps_ik - mu)/kT), g(x) = 1/(1 + e^x), with mu found by bisection so that
    sum_k w_k sum_i f_ik = n_el. Returns (list of f arrays, mu, -T S) with the spin-summed entropy
    S = -sum_k w_k sum_i 2 [g ln g + (1 - g) ln(1 - g)]."""
    e_all = np.concatenate([np.asarray(e, dtype=np.float64) for e in eps_list])
    lo, hi = float(e_all.min()) - 40.0 * kT - 1.0, float(e_all.max()) + 40.0 * kT + 1.0

    def count(mu):
        return sum(w * float(np.sum(2.0 * sps.expit(-(np.asarray(e) - mu) / kT))) for e, w in zip(eps_list, kw))

    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if count(mid) < n_el:
            lo = mid
        else:
            hi = mid
    mu = 0.5 * (lo + hi)
    occ, ts = [], 0.0
    for e, w in zip(eps_list, kw):
        g = sps.expit(-(np.asarray(e, dtype=np.float64) - mu) / kT)
        occ.append(2.0 * g)
        ent = -(sps.xlogy(g, g) + sps.xlogy(1.0 - g, 1.0 - g))
        ts += w * 2.0 * kT * float(np.sum(ent))
    return occ, mu, -ts


# ----------------------------------------------------------------------------------------------
# The SCF system
# ----------------------------------------------------------------------------------------------

class ScfSystem:
    """Cell, pseudopotentials and bases of one SCF problem (one or more k-points)."""

    def __init__(self, lat, pos, ecut, n_bands, n_occ, pp, dstr=None, kb_rc=1.2, kpts=None, kw=None, kT=0.0):
        self.lat = np.asarray(lat, dtype=np.float64)
        self.pos = np.asarray(pos, dtype=np.float64)
        self.ecut, self.n_bands, self.n_occ = float(ecut), int(n_bands), int(n_occ)
        self.pp = dict(pp)
        self.kpts = np.zeros((1, 3)) if kpts is None else np.asarray(kpts, dtype=np.float64)
        self.kw = np.full(len(self.kpts), 1.0 / len(self.kpts)) if kw is None else np.asarray(kw)
        self.grid = pw.fft_grid(self.lat, ecut, self.kpts)
        self.bases = [pw.Basis(self.lat, ecut, self.grid, k) for k in self.kpts]
        self.omega = pw.cell_volume(self.lat)
        self.n_el = 2.0 * n_occ
        self.occ = np.zeros(n_bands)
        self.occ[:n_occ] = 2.0
        self.v_loc = pw.vloc_real(self.lat, self.pos, self.grid, ecut, **self.pp)
        self.dstr = dstr
        self.betas = [pw.kb_beta(self.lat, self.pos, b.q, kb_rc) if dstr is not None else None
                      for b in self.bases]
        self.e_ewald = ewald(self.lat, self.pos, self.pp["Z"])
        self.kT = float(kT)

    def occupations(self, eps_list):
        """(occupation array per k, -T S): the lowest n_occ bands doubly occupied when kT = 0, else
        Fermi-Dirac occupations of the eigenvalues eps_list (one array per k)."""
        if self.kT <= 0.0:
            return [self.occ.copy() for _ in self.kpts], 0.0
        occ, _, mts = fermi_occupations(eps_list, self.kw, self.n_el, self.kT)
        return occ, mts

    def veff(self, rho):
        vh, eh = hartree(self.lat, self.grid, rho)
        exc_d, vxc = lda_pz(rho)
        return self.v_loc + vh + vxc, eh, exc_d

    def density(self, psis, occs=None):
        """rho of the orbitals psis with occupations occs (one array per k; None: fixed occupations)."""
        rho = np.zeros(self.grid)
        if occs is None:
            occs = [self.occ] * len(psis)
        for b, w, psi, f in zip(self.bases, self.kw, psis, occs):
            n = int(np.count_nonzero(f))
            if n:
                rho += density(b, psi[:n], np.asarray(f)[:n], w)
        return rho

    def energy(self, psis, occs=None, minus_ts=0.0):
        """Total energy of the orbitals psis (one (n_bands, npw) array per k) with occupations occs
        (None: fixed) and their density; with smearing the Mermin free energy, its -T S term given."""
        if occs is None:
            occs = [self.occ] * len(psis)
        rho = self.density(psis, occs)
        e_kin = e_nl = 0.0
        for b, w, psi, beta, fo in zip(self.bases, self.kw, psis, self.betas, occs):
            n = int(np.count_nonzero(fo))
            po = psi[:n]
            f = np.asarray(fo)[:n]
            e_kin += w * float(np.sum(f[:, None] * b.kin[None, :] * np.abs(po) ** 2))
            if beta is not None:
                proj = np.conj(beta) @ po.T
                e_nl += w * float(np.sum(f[None, :] * pw.kb_dvec(self.dstr)[:, None] * np.abs(proj) ** 2))
        dv = self.omega / np.prod(self.grid)
        e_loc = dv * float(np.sum(self.v_loc * rho))
        _, e_h = hartree(self.lat, self.grid, rho)
        exc_d, _ = lda_pz(rho)
        e_xc = dv * float(np.sum(rho * exc_d))
        terms = {"kinetic": e_kin, "nonlocal": e_nl, "local": e_loc, "hartree": e_h, "xc": e_xc, "ewald": self.e_ewald}
        if self.kT > 0.0:
            terms["smearing"] = minus_ts
        terms["total"] = sum(terms.values())
        return terms, rho


def scf_step(sys: ScfSystem, state, occs, rho_in, mixer, alg=1, eta=paro.INNER_RTOL, max_inner=paro.INNER_MAX_IT,
             delta=0.5):
    """One ParO iteration merged with one SCF iteration (Algorithm 1, 2 or 3, Section 2.3) from the state
    (per k: eps, psi, H psi), its occupations and the input density rho_in. Returns the new state, its
    occupations, rho_in^{n+1} (= rho_in^{n+1/2}) and the energy terms of the new orbitals."""
    v, _, _ = sys.veff(rho_in)
    probs = [paro.ParoProblem(b, v, beta, sys.dstr, delta) for b, beta in zip(sys.bases, sys.betas)]
    # step 3: source problems with V(rho_in^n)
    xs = []
    for p, (eps, psi, hpsi) in zip(probs, state):
        if alg == 1:
            x, _ = paro.source_solve(p, psi, eps, eta, max_inner)
            xs.append(paro.cholesky_orthonormalize(x))
        else:
            if alg == 2:
                b = -(hpsi - eps[:, None] * psi)
                e, _ = paro.pcg(p.a, b, np.zeros_like(psi), p.precond, eta, max_inner)
            else:
                e, _ = paro.correction_alg3(p, psi, hpsi, eps, eta, max_inner)
            e = e - (e @ np.conj(psi).T) @ psi
            keep = np.linalg.norm(e, axis=1) > 1e-10
            xs.append(paro.cholesky_orthonormalize(np.concatenate([psi, e[keep]], axis=0)))
    # rho_in^{n+1/2} from the new orbitals and the history
    rho_out = sys.density(xs, occs) if alg == 1 else sys.density([s[1] for s in state], occs)
    rho_in = mixer.mix(rho_in, rho_out)
    v, _, _ = sys.veff(rho_in)
    probs = [paro.ParoProblem(b, v, beta, sys.dstr, delta) for b, beta in zip(sys.bases, sys.betas)]
    # step 4: Rayleigh-Ritz with V(rho_in^{n+1/2})
    state = []
    for p, y in zip(probs, xs):
        eps, psi, hpsi = paro.rayleigh_ritz(y, p.h(y))
        state.append((eps[: sys.n_bands], psi[: sys.n_bands], hpsi[: sys.n_bands]))
    occs, mts = sys.occupations([s[0] for s in state])
    terms, _ = sys.energy([s[1] for s in state], occs, mts)
    return state, occs, rho_in, terms


def paro_scf(sys: ScfSystem, c0s, tol=1e-8, max_iter=500, eta=paro.INNER_RTOL,
             max_inner=paro.INNER_MAX_IT, delta=0.5,
             pulay_depth=8, pulay_beta=0.7, alg=1, log=None):
    """ParO merged with SCF (Algorithm 1; Algorithms 2 and 3 with alg=2, 3). Returns (energy terms, eps, psis,
    n_iter)."""
    rho_in = np.full(sys.grid, sys.n_el / sys.omega)
    mixer = Pulay(pulay_depth, pulay_beta)
    v, _, _ = sys.veff(rho_in)
    probs = [paro.ParoProblem(b, v, beta, sys.dstr, delta) for b, beta in zip(sys.bases, sys.betas)]
    state = [paro.initial_state(p, c0) for p, c0 in zip(probs, c0s)]
    occs, _ = sys.occupations([s[0][: sys.n_bands] for s in state])
    e_old = None
    small = 0
    for it in range(1, max_iter + 1):
        state, occs, rho_in, terms = scf_step(sys, state, occs, rho_in, mixer, alg, eta, max_inner, delta)
        e = terms["total"]
        if log is not None:
            log.append(dict(it=it, energy=e, eta=eta, state=state, rho_in=rho_in))
        if e_old is not None and abs(e - e_old) / len(sys.pos) < tol:
            small += 1
            if small >= 2:
                return terms, [s[0] for s in state], [s[1] for s in state], it
        else:
            small = 0
        e_old = e
    raise RuntimeError("SCF did not converge")


def dense_scf(sys: ScfSystem, tol=1e-8, max_iter=200, pulay_depth=8, pulay_beta=0.7):
    """The same SCF fixed point with dense diagonalisation of H instead of ParO (small cells only)."""
    rho_in = np.full(sys.grid, sys.n_el / sys.omega)
    mixer = Pulay(pulay_depth, pulay_beta)
    e_old = None
    small = 0
    for it in range(1, max_iter + 1):
        v, _, _ = sys.veff(rho_in)
        psis, epss = [], []
        for b, beta in zip(sys.bases, sys.betas):
            h = pw.dense_h(b, v, beta, pw.kb_dvec(sys.dstr) if beta is not None else None)
            eps, vec = np.linalg.eigh(h)
            psis.append(vec[:, : sys.n_bands].T.copy())
            epss.append(eps[: sys.n_bands])
        occs, mts = sys.occupations(epss)
        terms, rho_out = sys.energy(psis, occs, mts)
        e = terms["total"]
        if e_old is not None and abs(e - e_old) / len(sys.pos) < tol:
            small += 1
            if small >= 2:
                return terms, epss, psis, it
        else:
            small = 0
        e_old = e
        rho_in = mixer.mix(rho_in, rho_out)
    raise RuntimeError("dense SCF did not converge")
