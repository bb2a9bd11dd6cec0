"""Writes the expected values of the SCF fixed-point tests from the CPU oracle only.

The 8-atom diamond cell (a = 10.26 Bohr, seeded displacements, seed 41), local + Kleinman-Bylander
pseudopotential (strengths seed 42), E_cut 10 Ha (1647 plane waves, 32^3 grid):
  scf_si8kb_ecut10.json        12 bands, 8 occupied (a gap of 9 mHa above band 8), integer occupations;
  scf_si8kb_ecut10_smear.json  20 bands, 16 occupied (bands 16 and 17 cross), Fermi-Dirac kT = 0.002 Ha.
SCF fixed point by dense diagonalisation of the grid Hamiltonian (the loop of oracle.scf.dense_scf:
Pulay mixing, Section 2.3 with the readings of the oracle's docstrings), run until the density itself
has converged, max |rho_out - rho_in| < 1e-11, so that the eigenvalues of H[rho_in] are those of the
fixed point to ~1e-11 Ha.

  python tests/golden/make_scf_golden.py      (a few minutes on 8 cores)
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import pw, scf  # noqa: E402
from paper_1702_04045_gb300 import inputs  # noqa: E402


def fixed_point(n_bands, n_occ, kT):
    lat, pos = inputs.diamond_cell(1, 10.26, 41)
    d = inputs.kb_strengths(len(pos), 42)
    sys_ = scf.ScfSystem(lat, pos, 10.0, n_bands, n_occ, inputs.LOCAL_PP, d, inputs.KB_RC, kT=kT)
    rho_in = np.full(sys_.grid, sys_.n_el / sys_.omega)
    mixer = scf.Pulay(8, 0.7)
    for n_iter in range(1, 201):
        v, _, _ = sys_.veff(rho_in)
        h = pw.dense_h(sys_.bases[0], v, sys_.betas[0], pw.kb_dvec(sys_.dstr))
        eps, vec = np.linalg.eigh(h)
        eps = eps[: sys_.n_bands]
        psi = vec[:, : sys_.n_bands].T.copy()
        occ, mts = sys_.occupations([eps])
        rho_out = sys_.density([psi], occ)
        if np.abs(rho_out - rho_in).max() < 1e-11:
            break
        rho_in = mixer.mix(rho_in, rho_out)
    else:
        raise RuntimeError("dense SCF did not converge")
    terms, _ = sys_.energy([psi], occ, mts)
    return {"cell": f"8-atom diamond a=10.26 seed 41, KB seed 42, ecut 10 Ha, {n_bands} bands, {n_occ} occupied"
                    + (f", Fermi-Dirac kT={kT} Ha" if kT > 0 else ""),
            "source": "dense-diagonalisation SCF of the oracle, density converged to 1e-11",
            "grid": list(sys_.grid), "npw": sys_.bases[0].npw, "dense_scf_iterations": n_iter,
            "energy": terms, "eigenvalues": [float(x) for x in eps], "occupations": [float(x) for x in occ[0]]}


def main():
    for name, args in (("scf_si8kb_ecut10.json", (12, 8, 0.0)), ("scf_si8kb_ecut10_smear.json", (20, 16, 0.002))):
        with open(os.path.join(HERE, name), "w") as f:
            json.dump(fixed_point(*args), f, indent=1)


if __name__ == "__main__":
    main()
