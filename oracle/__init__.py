"""FP64 CPU oracle for the statically condensed HHO Stokes system and its
p-multilevel V-cycle / FGMRES solve (arXiv 2009.13840, Secs. 2-4).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, step-by-step
restatement of the paper used to check the CUDA library.  Only the tests, the
smoke check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may
import it.  The CUDA path never imports it, and it never imports the CUDA path:
the two share only the seeded input generators in ``synthetic/``.

Every function cites the section, equation or algorithm of the paper it
follows.  Where the paper is silent or garbled the reading taken is stated in
the docstring.  Parity status: every part is pinned by the tests in
``tests/test_oracle_*.py`` (closed forms, exact polynomial reproduction,
convergence rates, the paper's DOF/MNZ tables, brute-force dense V-cycle).
"""
