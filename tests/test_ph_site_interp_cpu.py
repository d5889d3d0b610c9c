"""The three-pair residual in the site formulation (tests/ph_site_interp.py)
against the oracle's full-space residual, through the C-ABI K = 3 layout.

N = 3 and 4, random amplitudes (uniform +-0.1), integrals truncated to three
and to two labels: every residual element and the energy agree to FP64
rounding.  This pins, without a GPU, the site-basis ingredients of the PH
path: the three-site Hamiltonian built from the 576 three-label integral keys,
the graded signs of operators embedded among other sites, the 303 three-pair
channels and the layout's sign conventions.  Control: dropping the sign picked
up from the sites before an operator breaks the agreement.
"""
import numpy as np
import pytest

import paper_1609_00077_gb300 as ppq
from workloads import build_ppp, build_hchain
from oracle.detcc import Problem
from tests.layout import LayoutMap
import tests.ph_site_interp as psi

SYSTEMS = {"C6H8": lambda: build_ppp('polyene', 6), "C8H10": lambda: build_ppp('polyene', 8),
           "H8": lambda: build_hchain(8, 1.5)}


def _desc3():
    try:
        return ppq.amp_layout(3)
    except ppq.PPQError:
        pytest.skip("libppq.so not built")


def _run(name, K_H):
    desc3 = _desc3()
    H = SYSTEMS[name]()
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=3, K_H=K_H)
    t = np.random.default_rng(3).uniform(-0.1, 0.1, P.cc.n_amp)
    R, e = P.residual(t)
    lm = LayoutMap(P.cc.manifold, H.occ_of_pair, H.vir_of_pair, H.n_orb, desc3)
    r, e2 = psi.SiteInterp(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K_H, desc3).residual(lm.to_layout(t))
    return R, e, lm.from_layout(r), e2


@pytest.mark.parametrize("name,K_H", [("C6H8", 3), ("C6H8", 2), ("C8H10", 3), ("H8", 2)])
def test_site_formulation_matches_oracle(name, K_H):
    R, e, R2, e2 = _run(name, K_H)
    assert np.abs(R).max() > 0.05
    assert np.abs(R2 - R).max() < 1e-12
    assert abs(e2 - e) < 1e-12


def test_embedding_sign_control(monkeypatch):
    monkeypatch.setattr(psi, "_SECTORS", {})
    monkeypatch.setattr(psi, "_CLUSTER", {})
    monkeypatch.setattr(psi, "_PIECE", {})
    monkeypatch.setattr(psi.Sector, "_before", staticmethod(lambda st, j: np.zeros(len(st), dtype=np.int64)))
    R, e, R2, e2 = _run("C6H8", 3)
    assert np.abs(R2 - R).max() > 1e-3


def test_disjoint_class_as_closure_row_times_links():
    """Every (M, S) with no common label at N = 4 (all interleavings of the
    labels, |M| + |S| <= 4): the generic term equals the closure row
    G_S[s'] = <ref| H_S exp(I_S) |s'> times the link coefficients
    <mu s'| exp(L) |ref> with the interleaving sign -- the form the six-label
    PH class takes on the tensor cores.  G_S vanishes beyond two holes."""
    import itertools
    desc3 = _desc3()
    H = SYSTEMS["C8H10"]()
    N = H.n_pairs
    si = psi.SiteInterp(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, 3, desc3)
    amp = si.amplitudes(np.random.default_rng(4).uniform(-0.1, 0.1, ppq.amp_count(N, 3)))
    mats = {}
    n = 0
    for km in (1, 2, 3):
        for M in itertools.combinations(range(N), km):
            rest = [X for X in range(N) if X not in M]
            for ks in range(1, len(rest) + 1):
                for S in itertools.combinations(rest, ks):
                    U, w, _ = si.term(M, S, amp, mats)
                    want = si._read(M, U, w)
                    got = si.disjoint_term(M, S, amp, mats)
                    assert np.abs(got - want).max() < 1e-14 * max(1.0, np.abs(want).max())
                    n += 1
    assert n == 50
    # the closure row of a three-label piece has no entry beyond two holes
    S = (0, 1, 3)
    I_S = si._ops(amp, S, lambda L: True, mats)
    row = psi._expv(I_S.T.tocsr(), si.piece(3, (0, 1, 2), S).T @ si._ref(3))
    holes = (si.sector(3).states & 1).astype(bool).sum(1) + (si.sector(3).states & 2).astype(bool).sum(1)
    assert np.abs(row).max() > 1e-3 and np.all(row[holes > 2] == 0.0)


def test_site_formulation_ph_solve_is_fci_at_6e6o():
    """Jacobi/DIIS on the K = 3 layout with the site-formulation residual and
    the layout's orbital-energy denominators: for hexatriene (6 electrons in
    6 orbitals) PH converges to the FCI energy (Abstract: PH is exact there)."""
    from oracle.fci import fci_energy
    desc3 = _desc3()
    H = SYSTEMS["C6H8"]()
    si = psi.SiteInterp(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, 3, desc3)
    t, e, rn, it, ok = psi.solve(si, si.f, r_tol=1e-11, e_tol=1e-13)
    assert ok
    e_ref = sum(H.h[i, i] + si.f[i, i] for i in H.occ_of_pair) + H.e_const
    assert abs(e + e_ref - fci_energy(H.h, H.eri, 3, H.e_const)) < 1e-9


@pytest.mark.slow
@pytest.mark.skipif(__import__("os").environ.get("PPQ_LONG_CHECKS") != "1",
                    reason="about 2 min; set PPQ_LONG_CHECKS=1")
def test_site_formulation_ph_solve_matches_oracle_n4():
    """Octatetraene (N = 4, where PH is not exact): the site-formulation PH
    solve reaches the oracle's PH energy."""
    from oracle.detcc import Problem
    desc3 = _desc3()
    H = SYSTEMS["C8H10"]()
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=3, e_const=H.e_const)
    r = P.solve(r_tol=1e-11, e_tol=1e-13, max_iter=400)
    si = psi.SiteInterp(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, 3, desc3)
    t, e, rn, it, ok = psi.solve(si, si.f, r_tol=1e-11, e_tol=1e-13)
    assert r['converged'] and ok
    assert abs(e - r['e_corr']) < 1e-9


def _disjoint_pairs(N, max_sites):
    import itertools
    for km in (1, 2, 3):
        for M in itertools.combinations(range(N), km):
            rest = [X for X in range(N) if X not in M]
            for ks in range(1, len(rest) + 1):
                for S in itertools.combinations(rest, ks):
                    if km + ks <= max_sites:
                        yield M, S


@pytest.mark.parametrize("max_sites", [3, pytest.param(4, marks=[pytest.mark.slow, pytest.mark.skipif(
    __import__("os").environ.get("PPQ_LONG_CHECKS") != "1", reason="about 3 min; set PPQ_LONG_CHECKS=1")])])
def test_disjoint_class_from_configuration_tables(max_sites):
    """The link coefficients expanded into configurations generated per
    interleaving pattern (tests/ph_disjoint_tables.py) reproduce the
    disjoint-class term: every disjoint (M, S) of at most three labels at
    N = 4 (all 50, four labels included, with PPQ_LONG_CHECKS=1)."""
    from tests.ph_disjoint_tables import disjoint_term_from_tables
    desc3 = _desc3()
    H = SYSTEMS["C8H10"]()
    N = H.n_pairs
    si = psi.SiteInterp(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, 3, desc3)
    amp = si.amplitudes(np.random.default_rng(4).uniform(-0.1, 0.1, ppq.amp_count(N, 3)))
    mats, cache = {}, {}
    n = 0
    for M, S in _disjoint_pairs(N, max_sites):
        want = si.disjoint_term(M, S, amp, mats)
        got = disjoint_term_from_tables(si, M, S, amp, mats, cache)
        assert np.abs(got - want).max() < 1e-14 * max(1.0, np.abs(want).max())
        n += 1
    assert n == (36 if max_sites == 3 else 50)


@pytest.mark.parametrize("max_sites", [3, pytest.param(4, marks=[pytest.mark.slow, pytest.mark.skipif(
    __import__("os").environ.get("PPQ_LONG_CHECKS") != "1", reason="about 30 s; set PPQ_LONG_CHECKS=1")])])
def test_link_factors_per_label_merge_to_exp_L(max_sites):
    """exp(L)|ref> of the clusters joining S to M, built as the graded product
    of one factor per label of S and one per pair of labels of S (each
    shareable across pieces), equals exp(L)|ref> on the sector of U."""
    from tests.ph_disjoint_tables import link_factors, merge
    desc3 = _desc3()
    H = SYSTEMS["C8H10"]()
    N = H.n_pairs
    si = psi.SiteInterp(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, 3, desc3)
    amp = si.amplitudes(np.random.default_rng(4).uniform(-0.1, 0.1, ppq.amp_count(N, 3)))
    mats = {}
    n = 0
    for M, S in _disjoint_pairs(N, max_sites):
        U, fs = link_factors(si, M, S, amp, mats)
        prod = fs[0]
        for f in fs[1:]:
            prod = merge(prod, f)
        L = si._ops(amp, U, lambda L: bool(L & set(S)) and bool(L & set(M)), mats)
        w = psi._expv(L, si._ref(len(U)))
        Sec = si.sector(len(U))
        v = np.zeros(Sec.dim)
        for st, c in prod.items():
            v[Sec.index(np.array([st]))[0]] += c
        assert np.abs(v - w).max() < 1e-14
        n += 1
    assert n == (36 if max_sites == 3 else 50)
