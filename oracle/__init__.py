"""Plain FP64 CPU oracle for the LOBPCG-F Dirac-Kohn-Sham eigensolver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls, links or
executes this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It
shares no code with the CUDA path: the only common module is ``workloads``,
which produces seeded inputs and holds none of the method's arithmetic.

What it computes (Lin, Shao, E, "Efficient iterative method for solving the
Dirac-Kohn-Sham density functional theory"):

* ``basis``     -- the planewave sphere |k+G|^2/2 <= Ecut (Sec. 2.3) in the
                   canonical order (Miller triples sorted lexicographically).
* ``operator``  -- the shifted valence DKS operator H' = H - c^2 of Eq. (vDKS)
                   with the free Dirac term of Eq. (2) per planewave, the local
                   potential on the FFT grid and the spin-orbit projectors of
                   Eq. (HGH); both as a dense matrix and matrix-free (numpy FFT);
                   the filter of Eq. (filter); the Teter-Payne-Allan
                   preconditioner (Sec. 4).
* ``lobpcgf``   -- Algorithm 1 (LOBPCG-F; without the filter lines it is
                   standard LOBPCG) and the plain definition of the result: the
                   lowest nev eigenpairs of the dense matrix above the gap.
* ``davidson``  -- block Davidson with the filter step of Algorithm 1 (the
                   paper's remark that the filter carries over to Davidson-type
                   solvers, Sec. 3).
* ``scf``       -- the self-consistent field loop around the eigenproblem: the
                   density of Eq. (density), the Hartree and LDA potential of
                   Sec. 2.1, Anderson mixing with the Kerker preconditioner
                   (Sec. 4.1), on the dense operator.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants, library routines or brute force (see each test's docstring).
"""
from . import basis, operator, lobpcgf, davidson, scf  # noqa: F401
