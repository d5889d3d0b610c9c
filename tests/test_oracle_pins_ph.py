"""Pins of the oracle's three-pair (PH) path, independent of its formulas.

* Residual and energy at random amplitudes for K = 3 (every excitation of
  three pairs, up to hextuples) against a Jordan-Wigner construction of
  exp(-T) H exp(T) with scipy's expm, in the 400-state sector of three
  alpha and three beta electrons in twelve spin orbitals, with the integrals truncated to three labels (all kept at
  N = 3) and to two labels (Table I, Implementation section).
* The truncated bare Hamiltonian against the Slater-Condon rules: its
  normal-ordered one-body part is the full Fock matrix and its two-body part
  keeps an integral exactly when its orbitals carry at most K_H labels.
* Size consistency of PH (Theory section): a direct sum of a three-pair and a
  one-pair fragment, pairs interleaved, has the sum of the fragment FCI
  energies (PH is exact for each fragment).
* The excitation-rank mask (Conclusions: higher excitations disabled; PH
  with singles and doubles is a local CCSD): with ranks <= 2 kept, three
  non-interacting H2 molecules (one pair each) still get the sum of their FCI
  energies (CCSD is exact for two electrons, and the connected higher
  excitations of a product of two-electron fragments vanish), while
  hexatriene does not get its FCI energy; with every rank kept (6) it does.
"""
import numpy as np
import pytest
from scipy.linalg import expm

from workloads import build_ppp, build_hchain
from oracle.detcc import Problem
from oracle.fci import fci_energy
from tests.test_oracle_pins import _direct_sum
from tests.jw import JW


def _labels(H):
    lab = np.empty(H.n_orb, dtype=np.int64)
    lab[H.occ_of_pair] = np.arange(H.n_pairs)
    lab[H.vir_of_pair] = np.arange(H.n_pairs)
    return lab


@pytest.mark.parametrize("K_H", [3, 2])
def test_ph_residual_random_t_against_jordan_wigner_expm(K_H):
    """N = 3 (hexatriene PPP, 12 spin orbitals, 400 states of 3 + 3 electrons):
    every tau_D of the 399 three-pair amplitudes and H as sparse Jordan-Wigner
    products, exp(+-T) by scipy expm; linked residual and energy compared."""
    H = build_ppp('polyene', 6)
    n = H.n_orb
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=3, K_H=K_H)
    assert P.cc.n_amp == 3 * 3 + 29 * 3 + 303
    t = np.random.default_rng(4242).uniform(-0.1, 0.1, P.cc.n_amp)
    R, e = P.residual(t)

    jw = JW(n, n // 2, n // 2)
    occ = sorted(int(i) for i in H.occ_of_pair)
    ref = jw.det(occ, occ)
    T = 0.0
    dets = []
    for tk, (ah, ap, bh, bp) in zip(t, P.cc.manifold):
        tau, D = jw.excitation(ah, ap, bh, bp, occ)
        T = T + tk * tau
        dets.append(D)
    Hm = jw.hamiltonian(P.hp, P.vt).toarray()
    Tm = T.toarray()
    Hbar = expm(-Tm) @ Hm @ expm(Tm)
    R_jw = np.array([d @ Hbar @ ref for d in dets])
    e_jw = ref @ Hbar @ ref - ref @ Hm @ ref
    assert np.abs(R - R_jw).max() < 1e-12
    assert abs(e - e_jw) < 1e-12


@pytest.mark.parametrize("K_H", [3, 2])
def test_truncated_hamiltonian_slater_condon(K_H):
    """N = 3: the oracle's bare (h', v') as a Jordan-Wigner operator.  Its
    reference expectation is the full E_ref, its singles-reference elements
    are the full Fock matrix, and its doubles-reference and opposite-spin
    singles-singles elements are the integrals (ai|bj) and (ai|jb) when
    a, i, b, j carry at most K_H labels and zero otherwise."""
    H = build_ppp('polyene', 6)
    n = H.n_orb
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=3, K_H=K_H)
    jw = JW(n, n // 2, n // 2)
    a, ad = jw.a, jw.ad
    Hm = jw.hamiltonian(P.hp, P.vt)
    occ = sorted(int(i) for i in H.occ_of_pair)
    vir = sorted(int(x) for x in H.vir_of_pair)
    ref = jw.det(occ, occ)
    Href = Hm @ ref
    eri, h = H.eri, H.h
    f = h + 2.0 * np.einsum('pqii->pq', eri[:, :, occ][:, :, :, occ]) \
        - np.einsum('piiq->pq', eri[:, occ][:, :, occ])
    assert abs(ref @ Href - sum(h[i, i] + f[i, i] for i in occ)) < 1e-12

    lab = _labels(H)

    def kept(*orbs):
        return len({lab[o] for o in orbs}) <= K_H

    al = lambda p: p
    be = lambda p: p + n
    n_masked = 0
    for i in occ:
        for x in vir:
            for s in (al, be):
                v = jw.product([ad[s(x)], a[s(i)]]) @ ref
                assert abs(v @ Href - f[x, i]) < 1e-12
            for j in occ:
                for y in vir:
                    d = jw.product([ad[al(x)], ad[be(y)], a[be(j)], a[al(i)]]) @ ref
                    want = eri[x, i, y, j] if kept(x, i, y, j) else 0.0
                    assert abs(d @ Href - want) < 1e-12
                    n_masked += not kept(x, i, y, j)
                    s1 = jw.product([ad[al(x)], a[al(i)]]) @ ref
                    s2 = jw.product([ad[be(y)], a[be(j)]]) @ ref
                    want = eri[x, i, j, y] if kept(x, i, j, y) else 0.0
                    assert abs(s1 @ (Hm @ s2) - want) < 1e-12
                    if i < j and x < y:
                        d = jw.product([ad[al(x)], ad[al(y)], a[al(j)], a[al(i)]]) @ ref
                        want = ((eri[x, i, y, j] if kept(x, i, y, j) else 0.0)
                                - (eri[x, j, y, i] if kept(x, j, y, i) else 0.0))
                        assert abs(d @ Href - want) < 1e-12
    # the two-label truncation really removes three-label integrals here
    assert (n_masked > 0) == (K_H == 2)
    assert np.abs(eri[np.ix_(vir, occ, vir, occ)]).max() > 1e-3


def test_ph_size_consistency_three_plus_one_pairs():
    """Hexatriene PPP (3 pairs) and H2 (1 pair) as one non-interacting system,
    pairs interleaved: E_PH(A+B) = E_FCI(A) + E_FCI(B)."""
    A = build_ppp('polyene', 6)
    B = build_hchain(2, 1.4)
    AB = _direct_sum(A, B)
    P = Problem(AB.h, AB.eri, AB.occ_of_pair, AB.vir_of_pair, K=3, e_const=AB.e_const)
    r = P.solve(r_tol=1e-11, e_tol=1e-13, max_iter=400)
    assert r['converged']
    fa = fci_energy(A.h, A.eri, 3, A.e_const)
    fb = fci_energy(B.h, B.eri, 1, B.e_const)
    assert abs(r['e_corr'] + P.e_ref - (fa + fb)) < 1e-9


def test_excitation_rank_mask():
    A, B, C = build_hchain(2, 1.4), build_hchain(2, 1.5), build_hchain(2, 1.3)
    ABC = _direct_sum(_direct_sum(A, B), C)
    P = Problem(ABC.h, ABC.eri, ABC.occ_of_pair, ABC.vir_of_pair, K=3, e_const=ABC.e_const, max_rank=2)
    assert P.cc.n_amp < Problem(ABC.h, ABC.eri, ABC.occ_of_pair, ABC.vir_of_pair, K=3).cc.n_amp
    r = P.solve(r_tol=1e-11, e_tol=1e-13, max_iter=400)
    assert r['converged']
    fsum = sum(fci_energy(X.h, X.eri, 1, X.e_const) for X in (A, B, C))
    assert abs(r['e_corr'] + P.e_ref - fsum) < 1e-9
    H = build_ppp('polyene', 6)
    fci = fci_energy(H.h, H.eri, 3, H.e_const)
    es = {}
    for mr in (2, 4, 6):
        P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=3, e_const=H.e_const, max_rank=mr)
        r = P.solve(r_tol=1e-11, e_tol=1e-13, max_iter=400)
        assert r['converged']
        es[mr] = r['e_corr'] + P.e_ref
    assert abs(es[6] - fci) < 1e-9
    assert abs(es[2] - fci) > 1e-4 and abs(es[4] - fci) < abs(es[2] - fci)
