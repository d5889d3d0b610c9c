"""The structure tables of the label-subset expansion (generated natively by
the library, read through ph_tables_copy) interpreted on the CPU
(tests/ph_subset_interp.py) against the oracle.

What this pins, without a GPU:
  * the sector sizes: the zero-charge, zero-S_z states of k sites number
    C(2k, k)^2 (k alpha and k beta electrons in 2k orbitals of each spin);
  * the recursion of exp(T)|ref>, the Hamiltonian rows and the
    back-substitution: every residual element and the energy of the three-pair
    model equal the determinant-space oracle (O-det) at random amplitudes for
    N = 2, 3, 4 with integrals truncated to three and to two labels, to FP64
    rounding;
  * the inclusion-exclusion over label subsets with nonzero coefficients for
    several sizes: two-pair amplitudes at N = 5 and 6 (K + K_H = 4 < N) and
    three-pair amplitudes with two-label integrals at N = 6 (K + K_H = 5 < N),
    against the oracle's own local assembly (O-loc), which restricts the
    normal-ordered Hamiltonian instead of the bare one;
  * a control: ignoring the signs of the recursion breaks the agreement.
"""
import os
from math import comb

import numpy as np
import pytest

import paper_1609_00077_gb300 as ppq
from workloads import build_ppp, build_hchain
from oracle.detcc import Problem, enumerate_manifold
from oracle.loccc import LocalAssembly
from tests.layout import LayoutMap
from tests.ph_subset_interp import SubsetInterp, tables


def _lib():
    try:
        ppq.lib()
    except ppq.PPQError:
        pytest.skip("libppq.so not built")


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_sector_sizes_and_table_shapes(k):
    _lib()
    T = tables(k, 3, 3)
    assert len(T["code"]) == comb(2 * k, k) ** 2
    # levels: sub-states of a state lie on lower levels
    lvl = np.repeat(np.arange(len(T["lvl_ptr"]) - 1), np.diff(T["lvl_ptr"]))
    owner = np.repeat(np.arange(len(T["code"])), np.diff(T["ent_ptr"]))
    assert np.all(lvl[T["ent_sub"]] < lvl[owner])
    # outputs: the reference and every channel on at most three of the k sites
    assert len(T["out_state"]) == 1 + 3 * k + 29 * comb(k, 2) + 303 * comb(k, 3)
    # every state but the reference is reached by the recursion
    assert np.all(np.diff(T["ent_ptr"])[1:] > 0)


def _oracle_case(H, K, K_H, seed=3):
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=K, K_H=K_H)
    t = np.random.default_rng(seed).uniform(-0.1, 0.1, P.cc.n_amp)
    R, e = P.residual(t)
    lm = LayoutMap(P.cc.manifold, H.occ_of_pair, H.vir_of_pair, H.n_orb, ppq.amp_layout(K))
    return t, R, e, lm


def _interp(H, K, K_H, t, lm, **kw):
    si = SubsetInterp(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K, K_H)
    r, e = si.residual(lm.to_layout(t), **kw)
    return lm.from_layout(si.fill_copies(r, lm)), e


@pytest.mark.parametrize("name,K_H", [("C4H6", 3), ("C6H8", 3), ("C6H8", 2), ("C8H10", 3), ("H8", 2)])
def test_tables_match_oracle_three_pair(name, K_H):
    _lib()
    H = {"C4H6": lambda: build_ppp('polyene', 4), "C6H8": lambda: build_ppp('polyene', 6),
         "C8H10": lambda: build_ppp('polyene', 8), "H8": lambda: build_hchain(8, 1.5)}[name]()
    t, R, e, lm = _oracle_case(H, 3, K_H)
    R2, e2 = _interp(H, 3, K_H, t, lm)
    assert np.abs(R).max() > 0.05
    assert np.abs(R2 - R).max() < 1e-12
    assert abs(e2 - e) < 1e-12


@pytest.mark.parametrize("K,K_H,sites", [(2, 2, 10), (2, 2, 12), (3, 2, 12)])
def test_inclusion_exclusion_against_local_assembly(K, K_H, sites):
    _lib()
    H = build_ppp('polyene', sites)
    LA = LocalAssembly(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=K, K_H=K_H)
    t = np.random.default_rng(5).uniform(-0.1, 0.1, len(LA.manifold))
    R, e = LA.residual(t)
    lm = LayoutMap(LA.manifold, H.occ_of_pair, H.vir_of_pair, H.n_orb, ppq.amp_layout(K))
    R2, e2 = _interp(H, K, K_H, t, lm)
    assert np.abs(R2 - R).max() < 1e-12
    assert abs(e2 - e) < 1e-12


@pytest.mark.parametrize("name", ["C8H10", "H8"])
def test_untruncated_integrals_two_pair(name):
    # K_H = FULL: integrals over four labels enter (384 keys per quadruple),
    # terms reach K + 4 = 6 labels; against O-det with the untruncated Hamiltonian
    _lib()
    H = {"C8H10": lambda: build_ppp('polyene', 8), "H8": lambda: build_hchain(8, 1.5)}[name]()
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=2, K_H=-1)
    t = np.random.default_rng(9).uniform(-0.1, 0.1, P.cc.n_amp)
    R, e = P.residual(t)
    lm = LayoutMap(P.cc.manifold, H.occ_of_pair, H.vir_of_pair, H.n_orb, ppq.amp_layout(2))
    R2, e2 = _interp(H, 2, 4, t, lm)
    assert np.abs(R2 - R).max() < 1e-12
    assert abs(e2 - e) < 1e-12
    # the four-label integrals matter here
    P2 = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=2, K_H=2)
    assert np.abs(P2.residual(t)[0] - R).max() > 1e-4


def _full_golden():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "pq_full_c14h16.npz")
    if not os.path.exists(path):
        pytest.skip("golden file not generated")
    return np.load(path)


def test_untruncated_integrals_inclusion_exclusion_n7():
    # N = 7 > K + 4: every subset size enters; against the stored O-det values
    _lib()
    g = _full_golden()
    occ, vir = g["occ"], g["vir"]
    man = enumerate_manifold(occ, vir, 2)
    lm = LayoutMap(man, occ, vir, g["h"].shape[0], ppq.amp_layout(2))
    si = SubsetInterp(g["h"], g["eri"], occ, vir, 2, 4)
    r, e2 = si.residual(lm.to_layout(g["t"]))
    R2 = lm.from_layout(si.fill_copies(r, lm))
    assert np.abs(g["R"]).max() > 0.05
    assert np.abs(R2 - g["R"]).max() < 1e-12
    assert abs(e2 - float(g["e_corr"])) < 1e-12


@pytest.mark.skipif(not os.environ.get("PPQ_LONG_CHECKS"), reason="PPQ_LONG_CHECKS=1 (about 10 min)")
def test_local_assembly_untruncated_against_stored_odet_n7():
    # pins the oracle's local assembly with untruncated integrals (subset bound
    # K + 4) against O-det at 7 pairs
    g = _full_golden()
    LA = LocalAssembly(g["h"], g["eri"], g["occ"], g["vir"], K=2, K_H=-1)
    R, e = LA.residual(g["t"])
    assert np.abs(R - g["R"]).max() < 1e-12
    assert abs(e - float(g["e_corr"])) < 1e-12


def test_recursion_sign_control():
    _lib()
    H = build_ppp('polyene', 6)
    t, R, e, lm = _oracle_case(H, 3, 3)
    R2, _ = _interp(H, 3, 3, t, lm, sign_flip_control=True)
    assert np.abs(R2 - R).max() > 1e-3
