"""FP64 CPU oracle of the HDG method of Fu, Gatica and Sayas, "Matlab tools for HDG in
three dimensions" (arXiv 1305.1489).

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg
of `bench.py` may import or run anything in this package.  The product path (the CUDA
library under `paper_1305_1489_gb300/`) never calls it, and this package never calls the
product path: the two share no code.  Both take their inputs from `workloads/`.

The oracle follows the paper's steps literally, in plain numpy/scipy FP64:
  quadrature.py   eq. 3.1, Section 4 "Integrals on faces" (conical Gauss-Jacobi rules)
  basis.py        eq. 3.3, Section 4 "Bases, faces, and boundaries" (Dubiner bases)
  geometry.py     Section 2 (expanded mesh: faces, facebyele, perm, normals, eq. 2.0-2.5)
  hdg.py          Sections 3-6 and 9 (local blocks, eq. 5.1-5.7 with full LU of A_1,
                  CSR assembly eq. 6.5, Dirichlet/Neumann data eq. 6.3-6.4, recovery eq. 5.3,
                  postprocess eq. 9.11, errors eq. 10.1), and the monolithic solve of eq. 1.2.

Every function cites the passage it follows.  Pins (tests/test_oracle_*.py) tie it to
closed forms, invariants and exact solutions rather than to itself.
"""
