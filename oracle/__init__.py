"""FP64 CPU oracle for the fundamental-scheme implicit FDTD methods.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow reference that the
CUDA path is checked against.  Only the test suite, the package's smoke check
and the benchmark's CPU-baseline leg may import it; the product library never
does, and the oracle imports nothing from the product library.

It follows E. L. Tan, "Fundamental Schemes for Efficient Unconditionally
Stable Implicit Finite-Difference Time-Domain Methods" (arXiv 2011.14043):

* ``grid``      Yee grid, materials, the splitting operators A and B (Eqs. 33-34),
                b and d (Eq. 36), PEC walls.
* ``tridiag``   textbook Thomas elimination (the line solver of Sec. IV).
* ``schemes``   the original splitting formulae (ADI Eq. 1, LOD1 Eq. 11,
                SS2 Eq. 16, LOD2 Eqs. 18-20) and the fundamental ones (FADI
                Eqs. 7-10 in the component form of Eqs. 37-44, FLOD Eq. 15,
                FSS Eq. 17, FLOD2 Eqs. 21-23 in the component form of
                Eqs. 45-52).
* ``invariants`` field energy, the discrete-dispersion closed form, mode
                projections.
* ``dense``     brute-force dense assembly of A and B for tiny grids.

Every function is FP64, round-to-nearest, and favours being checkable against
the paper by eye over speed.
"""
