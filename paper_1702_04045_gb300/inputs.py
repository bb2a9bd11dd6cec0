"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds none of the method's arithmetic: it only draws random numbers and lays out
geometry, so that both sides of every parity test start from bit-identical inputs.

Stand-ins for the paper's workloads (Section 5 runs MgO, Al and Si through Quantum ESPRESSO with
norm-conserving pseudopotentials that are not available here): diamond-lattice cubic cells of
8, 64 and 512 atoms (a = 10.26, 20.52, 41.04 Bohr, the Si lattice constant family of the paper's
1000-atom Si run), each atom displaced by a seeded uniform +-0.05 Bohr, Gamma point (as in all of
the paper's runs), plus a 3x3x3 Monkhorst-Pack mesh and 64 random small cells for uneven batching.
"""
from __future__ import annotations

import numpy as np

# Fractional positions of the 8 atoms of the conventional diamond cell.
_FCC = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
DIAMOND_BASIS = np.concatenate([_FCC, _FCC + 0.25], axis=0)

# Local pseudopotential  v(r) = -Z erf(r/rc)/r + A exp(-(r/a)^2)  (Ha, Bohr).
LOCAL_PP = dict(Z=4.0, rc=0.8, A=2.0, a=1.0)
# Kleinman-Bylander s+p Gaussian projectors: radius and projectors per atom.
KB_RC = 1.2
KB_PER_ATOM = 4


def diamond_cell(n_rep: int, a_cubic: float, seed: int | None, disp: float = 0.05):
    """Lattice (rows a1,a2,a3, Bohr) and Cartesian positions of an n_rep^3 diamond supercell.

    Each Cartesian coordinate gets an independent U[-disp, disp] shift drawn from PCG64(seed);
    seed=None gives the perfect lattice.
    """
    lat = np.eye(3) * (a_cubic * n_rep)
    cells = np.array([[i, j, k] for i in range(n_rep) for j in range(n_rep) for k in range(n_rep)],
                     dtype=np.float64)
    frac = (cells[:, None, :] + DIAMOND_BASIS[None, :, :]).reshape(-1, 3) / n_rep
    pos = frac @ lat
    if seed is not None:
        rng = np.random.default_rng(seed)
        pos = pos + rng.uniform(-disp, disp, size=pos.shape)
    return lat, np.ascontiguousarray(pos)


def kb_strengths(n_atoms: int, seed: int) -> np.ndarray:
    """One KB strength per (atom, l), l = s, p, drawn U[-1, 1] Ha; shape (n_atoms, 2)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(n_atoms, 2))


def start_vectors(nb: int, npw: int, seed: int) -> np.ndarray:
    """Complex standard-normal start coefficients, shape (nb, npw), row = band (not orthonormal)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((nb, npw))
    im = rng.standard_normal((nb, npw))
    return re + 1j * im


def monkhorst_pack(q: int):
    """Monkhorst-Pack q x q x q mesh: reduced coordinates (2r-q-1)/(2q), equal weights 1/q^3."""
    r = (2.0 * np.arange(1, q + 1) - q - 1) / (2.0 * q)
    k = np.array([[x, y, z] for x in r for y in r for z in r])
    return k, np.full(len(k), 1.0 / len(k))


def random_cells(n_cells: int, seed: int):
    """Lattice constants U[9.8, 10.8] Bohr and cutoffs U[8, 14] Ha for n_cells 8-atom cells."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(9.8, 10.8, size=n_cells)
    ecut = rng.uniform(8.0, 14.0, size=n_cells)
    return a, ecut


# The synthetic workloads (a = conventional cubic constant; the supercell edge is n_rep * a).
# Seeds: displacements, start vectors, KB strengths.
CONFIGS = {
    # 8-atom cell, local pseudopotential only, fixed potential, FP64.
    "si8_local": dict(n_rep=1, a=10.26, ecut=10.0, n_bands=20, n_occ=16, kb=False,
                      seed_pos=1001, seed_psi=1002, seed_kb=None),
    # 64-atom cell, local + KB, SCF (LDA, Pulay 8). Its bands 128 and 129 are degenerate to ~1e-5 Ha, so
    # the SCF uses Fermi-Dirac occupations of width kT (Ha) over the 144 bands (256 electrons).
    "si64_scf": dict(n_rep=2, a=10.26, ecut=15.0, n_bands=144, n_occ=128, kb=True,
                     seed_pos=2001, seed_psi=2002, seed_kb=2003, kT=0.002),
    # 512-atom cell, local + KB, 1088 orbitals.
    "si512": dict(n_rep=4, a=10.26, ecut=12.0, n_bands=1088, n_occ=1024, kb=True,
                  seed_pos=5001, seed_psi=5002, seed_kb=5003),
}


def config_inputs(name: str):
    """Geometry, KB strengths (or None) and config dict for a named workload."""
    c = CONFIGS[name]
    lat, pos = diamond_cell(c["n_rep"], c["a"], c["seed_pos"])
    d = kb_strengths(len(pos), c["seed_kb"]) if c["kb"] else None
    return lat, pos, d, c


# Batched workloads of uneven problems: the 8-atom cell on a 3x3x3 Monkhorst-Pack mesh (27 k-points,
# plane-wave counts differing per k) and 64 independent 8-atom cells with seeded lattice constants and
# cutoffs (uneven plane-wave counts and FFT grids). 20 orbitals (16 occupied) per problem, local
# pseudopotential as in the 8-atom fixed-potential workload.
BATCHES = {
    "si8_mp27": dict(kind="kmesh", a=10.26, ecut=10.0, q=3, n_bands=20, n_occ=16, seed_pos=1001, seed_psi=4002),
    "cells64": dict(kind="cells", n_cells=64, seed_cells=4101, seed_pos=4102, seed_psi=4103, n_bands=20,
                    n_occ=16),
}


def batch_inputs(name: str, limit: int | None = None):
    """Problems of a batched workload: one dict per cell with lattice, positions, cutoff, k-points
    (reduced), k-weights, bands, occupied bands and the start-vector seed of each k-point."""
    c = BATCHES[name]
    out = []
    if c["kind"] == "kmesh":
        lat, pos = diamond_cell(1, c["a"], c["seed_pos"])
        k, w = monkhorst_pack(c["q"])
        out.append(dict(lat=lat, pos=pos, ecut=c["ecut"], kpts=k, kweights=w, n_bands=c["n_bands"],
                        n_occ=c["n_occ"], seeds=[c["seed_psi"] + i for i in range(len(k))]))
    else:
        a, ecut = random_cells(c["n_cells"], c["seed_cells"])
        for i in range(c["n_cells"]):
            lat, pos = diamond_cell(1, float(a[i]), c["seed_pos"] + i)
            out.append(dict(lat=lat, pos=pos, ecut=float(ecut[i]), kpts=np.zeros((1, 3)), kweights=np.ones(1),
                            n_bands=c["n_bands"], n_occ=c["n_occ"], seeds=[c["seed_psi"] + i]))
    return out[:limit] if limit else out

