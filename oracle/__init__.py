"""Oracle: a plain, slow CPU FP64 restricted Hartree-Fock energy and gradient.

TEST INFRASTRUCTURE ONLY. Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import this
package. It shares no code with the CUDA library (`paper_1601_02713_gb300`):
its integrals are McMurchie-Davidson (integrals.c), the library's are
Obara-Saika / Head-Gordon-Pople; its linear algebra is numpy/LAPACK.

The paper (Sec. 2) defines the computation as the Born-Oppenheimer energy and
forces of every replica; Sec. 3.1 fixes the integral cutoff (1e-12) and an SCF
density threshold. It gives no electronic-structure algorithm, so the oracle
follows the standard closed-shell Roothaan-Hall SCF with Pulay DIIS and the
standard analytic RHF gradient (see `rhf.py`). `dft.py` (imported as
`oracle.dft`) is the paper's own level of theory, B3LYP, as a plain
grid-based Kohn-Sham energy; the CUDA library has no counterpart yet.
"""
from .rhf import (OracleBasis, boys, build, core_guess, eri_block, eri_full,  # noqa: F401
                  jk, nuclear_repulsion, one_electron, rhf_energy_gradient,
                  run_scf, schwarz, num_threads, grad_1e, grad_2e, normalise_shell,
                  eri_list, deriv_list, canonical_quartets, g_block,
                  sad_atomic_density, orthogonaliser)
