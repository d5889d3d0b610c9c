"""CPU FP64 oracle for the PQ / PH amplitude equations.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package; only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path or with the schedule generator of the package.

Contents
--------
fci      determinant-string machinery and brute-force FCI (the exactness pins).
detcc    O-det: coupled cluster on the pair-truncated manifold M_K, evaluated
         exactly in the full determinant space (Theory section, Eq. decompose,
         Tables I-II; the truncated-integral reading K_H of the Implementation
         section), plus the Jacobi/DIIS solver.
loccc    O-loc: the same residual assembled by inclusion-exclusion over pair
         label subsets of local determinant-space CC problems, for sizes the
         full determinant space cannot reach.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(FCI exactness of PQ at 4e/4o and PH at 6e/6o, K >= N equals FCI, fragment
additivity, pair-permutation and orbital-sign invariance, O-loc == O-det).
The paper's printed energies (Tables VI, VII) need ab-initio inputs that are
not available, so no function is pinned to a printed number: that part of
parity is unpinned.
"""
