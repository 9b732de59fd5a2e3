"""Plain FP64 CPU oracle for the matrix-free elastic Lippmann-Schwinger method.

TEST INFRASTRUCTURE ONLY.  This package is a slow, obviously correct NumPy
restatement of what the paper's method computes, used to check the CUDA path.
Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference legs may import it.  The product path (the C-ABI
library and its Python binding) never calls it, and it shares no code with
that path: the only common module is ``synthetic`` (seeded inputs).

Contents, each following the paper's passage cited in its module:

* ``green``    - background Green's tensor G and its derivative (Eq. 7,
                 Appendix A Eqs. A.4-A.11), the sampled kernel table with its
                 self-cell value;
* ``operator`` - Voigt strain by finite differences (Eq. 18), contrast stress
                 (Eq. 11), the discrete LS operator A u = u - G (D sigma +
                 w^2 drho u) both as an explicit dense matrix (direct sums)
                 and matrix-free by FFT (Eq. 21), and its adjoint;
* ``source``   - the moment-tensor background field u0 (Eqs. 13-16);
* ``solver``   - BiCGSTAB (Van der Vorst 1992) with the relative residual of
                 Eq. 22, and a dense direct solve.

Every function is pinned by a test in ``tests/test_oracle_*.py`` against
closed forms, invariants, special cases or brute force.  The one function
whose result the paper itself never prints (none is: its figures are
stripped) is still pinned mathematically; "parity unpinned" applies only to
agreement with the paper's own figures.
"""
from . import green, operator, source, solver  # noqa: F401
