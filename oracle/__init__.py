"""FP64 CPU oracle of the deflated MG-FGMRES solve (arXiv:1912.02868).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA library; the two
meet only in the seeded inputs of ``synth``.

The oracle is plain numpy in complex128, written to be checked against the paper
by eye rather than to be fast:

* ``dirac``     - the 2D Wilson-Dirac operator D and the coarse block stencil
                  (Section 2; the operator is the standard Schwinger-model one)
* ``hierarchy`` - near-null vectors, global orthonormalisation, chiral doubling,
                  local 4^2 blocking and orthonormalisation, Galerkin D^ = P^+ D P
                  (Section 2, first paragraph)
* ``krylov``    - GMRES(2) smoother, FGMRES(m), GMRES-DR(m,k), GMRES-Proj(m,k),
                  CGNE (Section 2, second paragraph)
* ``mg``        - the three-level V-cycle and the full deflated MG-FGMRES solve
                  with the fine-equivalent Mvps count (Section 3, Eq. 1)

Parity pins (tests/test_oracle_*.py) tie each function to facts fixed by the
paper and the mathematics: free-field spectrum, sigma3-hermiticity, P^+P = I,
Galerkin against the dense product, Krylov results against dense LU and dense
eigendecompositions.
"""
