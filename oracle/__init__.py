"""Plain, slow, FP64 CPU oracle of the ParO plane-wave method (arXiv:1702.04045).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check in __graft_entry__ and by the
CPU-baseline leg of bench.py, never by the product (libparo.so and its Python binding), with
which it shares no code. Modules:
  pw     basis (Eq. e3), grid, local and KB pseudopotentials, FFT and dense Hamiltonian (Eq. e5)
  paro   PCG source problems and the ParO projection step (Algorithms 1 and 2)
  scf    density, Hartree, LDA-PZ, Pulay, Ewald, energies and the ParO-merged SCF (Section 2.3)

Parity unpinned (no independent check exists): the ParO iteration counts. The PZ-LDA constants are
pinned by the exact high-density coefficient and by an independent fit of the same Monte Carlo data;
the energy assembly by its variational derivative and the double-counting identity.
"""
