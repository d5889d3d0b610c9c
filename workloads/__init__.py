"""Seeded synthetic inputs for the PQ/PH solver and its oracle.

This package builds Hamiltonians only: model geometries, site/AO integrals, a
closed-shell RHF, the MO transform and the occupied/virtual pairing of Fig. 1
(hole indices reversed).  It holds none of the PQ/PH arithmetic, so the CUDA
path, the oracle, the tests and the benchmark can all draw their inputs from
it without sharing any of the method's code.
"""
from .ppp import polyene_geometry, acene_geometry, ppp_site_hamiltonian
from .hchain import hchain_ao_integrals
from .scf import (rhf, mo_integrals, pair_orbitals, Hamiltonian, build_ppp, build_hchain, ppp_eri_device,
                  ppp_cholesky_vectors, cholesky_vectors)
from .rng import random_pair_amplitude_seed

__all__ = [
    "polyene_geometry", "acene_geometry", "ppp_site_hamiltonian",
    "hchain_ao_integrals", "rhf", "mo_integrals", "pair_orbitals",
    "Hamiltonian", "build_ppp", "build_hchain", "random_pair_amplitude_seed", "ppp_cholesky_vectors",
    "cholesky_vectors",
]
