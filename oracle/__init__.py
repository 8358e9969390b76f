"""Plain, slow FP64 CPU oracle for the recursively preconditioned hierarchical
interpolative factorization (PHIF) of Feliu-Faba, Ho and Ying.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
package: only the test-suite, the smoke check and the CPU-baseline leg of the
benchmark use it.  It shares no code with the CUDA path; both read their inputs
from :mod:`workloads`, which holds no arithmetic of the method.

The oracle follows the paper's own formulation: it keeps the *global* active
matrix ``A_l`` as one sparse matrix and applies the paper's operators to it in
the paper's order (cell elimination, block Jacobi preconditioning,
skeletonization, root Cholesky), without any blocking, fusion or reordering
beyond what the paper states.  Library primitives used as single steps:
``numpy.linalg.cholesky`` (dense Cholesky), ``scipy.linalg.solve_triangular``
(triangular solve) and scipy.sparse products/sums.

Modules:

* :mod:`oracle.fd`    -- finite-difference matrix, Eqs. (1.1)-(1.2), Sec. 3.1/3.2.
* :mod:`oracle.tree`  -- quadtree/octree DOF grouping, Sec. 3.1 (Fig. 3), Sec. 3.2.
* :mod:`oracle.dense` -- column-pivoted QR interpolative decomposition, Sec. 2.2.
* :mod:`oracle.phif`  -- factorization (Sec. 3), apply of F^{-1} and F (Eqs. 3.1-3.3),
  PCG (Sec. 1, Sec. 4), error estimators (Sec. 4), adjoint gradient.

Parity status of each function is stated in its docstring; the pins live in
``tests/test_oracle_*.py``.
"""
