"""Input generators: the torch H-chain builder reproduces the NumPy one, and
the H2 / STO-3G RHF energy matches the textbook value."""
import numpy as np
import pytest

from workloads import build_hchain, build_ppp


def test_h2_sto3g_rhf_textbook():
    H = build_hchain(2, 0.7414)
    assert abs(H.e_rhf - (-1.1167)) < 2e-4   # minimal-basis H2 near equilibrium


def test_torch_hchain_matches_numpy():
    torch = pytest.importorskip("torch")
    from workloads.hchain_torch import build_hchain_torch
    A = build_hchain(10, 1.7)
    B = build_hchain_torch(10, 1.7, device="cpu")
    assert abs(A.e_rhf - B.e_rhf) < 1e-9
    assert np.abs(A.mo_energy - B.mo_energy).max() < 1e-8
    # MO integrals agree up to orbital phases: compare phase-invariant pieces
    ha, hb = A.h, B.h.numpy()
    assert np.abs(np.abs(ha) - np.abs(hb)).max() < 1e-8
    assert np.abs(np.einsum('ppqq->pq', A.eri) - np.einsum('ppqq->pq', B.eri.numpy())).max() < 1e-8


def test_localised_pairing_preserves_reference_energy():
    A = build_ppp('polyene', 12)
    B = build_ppp('polyene', 12, orbitals="local")
    occ = B.occ_of_pair
    f = B.h + 2 * B.eri[:, :, occ, occ].sum(-1) - B.eri[:, occ, occ, :].sum(1)
    e_ref = np.sum(B.h[occ, occ]) + np.sum(f[occ, occ]) + B.e_const
    assert abs(e_ref - A.e_rhf) < 1e-10


def test_acene_geometry_hueckel_spectra():
    """The acene builder (the PH workloads: fused hexagons, C-C 1.40 A): 4n+2
    sites, 5n+1 bonds of 1.40 A, and the bond graph's spectrum equals the
    textbook Hueckel values -- benzene 2, 1, 1, -1, -1, -2 and naphthalene
    +-(1+sqrt(13))/2, +-(1+sqrt(5))/2, +-(-1+sqrt(13))/2, +-1, +-(sqrt(5)-1)/2
    (in units of |beta|)."""
    from workloads import acene_geometry
    for n in range(1, 8):
        xyz, bonds = acene_geometry(n)
        assert len(xyz) == 4 * n + 2 and len(bonds) == 5 * n + 1
        d = [np.linalg.norm(xyz[i] - xyz[j]) for i, j in bonds]
        assert np.allclose(d, 1.40, atol=1e-5)
    for n, want in ((1, [2, 1, 1, -1, -1, -2]),
                    (2, [(1 + 13 ** .5) / 2, (1 + 5 ** .5) / 2, (-1 + 13 ** .5) / 2, 1, (5 ** .5 - 1) / 2])):
        xyz, bonds = acene_geometry(n)
        A = np.zeros((len(xyz), len(xyz)))
        for i, j in bonds:
            A[i, j] = A[j, i] = 1.0
        ev = np.sort(np.linalg.eigvalsh(A))
        if n == 2:
            want = want + [-w for w in want]
        assert np.allclose(ev, np.sort(want), atol=1e-12)


def test_cholesky_factors_reproduce_integrals():
    # the three-index inputs of pq_solve_cd: exact for PPP (one vector per
    # site), within the pivot threshold for the Gaussian H-chain integrals
    from workloads import ppp_cholesky_vectors, cholesky_vectors
    H = build_ppp('polyene', 8)
    B = ppp_cholesky_vectors(H)
    assert B.shape == (8, 8, 8)
    assert np.abs(np.einsum('qab,qcd->abcd', B, B) - H.eri).max() < 1e-14
    Hh = build_hchain(8, 1.5)
    B2 = cholesky_vectors(Hh.eri, 1e-12)
    assert B2.shape[0] < Hh.n_orb ** 2
    assert np.abs(np.einsum('qab,qcd->abcd', B2, B2) - Hh.eri).max() < 1e-10
