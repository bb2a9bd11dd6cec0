"""Writes the expected values of the SCF fixed point tests from the CPU oracle only.

The 8-atom diamond cell (a = 10.26 Bohr, seeded displacements, seed 41), local + Kleinman-Bylander
pseudopotential (strengths seed 42), E_cut 10 Ha (1647 plane waves, 32^3 grid), 12 bands of which 8
occupied: SCF fixed point by dense diagonalisation of the grid Hamiltonian (the loop of
oracle.scf.dense_scf: Pulay mixing, Section 2.3 with the readings of the oracle's docstrings), run until
the density itself has converged, max |rho_out - rho_in| < 1e-11, so that the eigenvalues of H[rho_in]
are those of the fixed point to ~1e-11 Ha.

  python tests/golden/make_scf_golden.py      (about 30 s on 8 cores)
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import pw, scf  # noqa: E402
from paper_1702_04045_gb300 import inputs  # noqa: E402


def main():
    lat, pos = inputs.diamond_cell(1, 10.26, 41)
    d = inputs.kb_strengths(len(pos), 42)
    sys_ = scf.ScfSystem(lat, pos, 10.0, 12, 8, inputs.LOCAL_PP, d, inputs.KB_RC)
    rho_in = np.full(sys_.grid, sys_.n_el / sys_.omega)
    mixer = scf.Pulay(8, 0.7)
    for n_iter in range(1, 201):
        v, _, _ = sys_.veff(rho_in)
        h = pw.dense_h(sys_.bases[0], v, sys_.betas[0], pw.kb_dvec(sys_.dstr))
        eps, vec = np.linalg.eigh(h)
        psi = vec[:, : sys_.n_bands].T.copy()
        rho_out = sys_.density([psi])
        if np.abs(rho_out - rho_in).max() < 1e-11:
            break
        rho_in = mixer.mix(rho_in, rho_out)
    else:
        raise RuntimeError("dense SCF did not converge")
    terms, _ = sys_.energy([psi])
    out = {"cell": "8-atom diamond a=10.26 seed 41, KB seed 42, ecut 10 Ha, 12 bands, 8 occupied",
           "source": "dense-diagonalisation SCF of the oracle, density converged to 1e-11",
           "grid": list(sys_.grid), "npw": sys_.bases[0].npw, "dense_scf_iterations": n_iter,
           "energy": terms, "eigenvalues": [float(x) for x in eps[: sys_.n_bands]]}
    with open(os.path.join(HERE, "scf_si8kb_ecut10.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
