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
  * a control: ignoring the signs of the recursion breaks the agreement;
  * the transposed (adjoint) tables: grad_t L of the Lagrangian E_c +
    lambda . R equals the oracle's complex-step Jacobian product at N = 2, 3,
    and the integral adjoints equal central differences of the Lagrangian.
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


@pytest.mark.parametrize("name,K_H", [("C4H6", 3), ("C4H6", 2), ("C6H8", 3)])
def test_adjoint_tables_match_oracle_lagrangian_gradient(name, K_H):
    # the transposed tables (reverse pass of the local problems, weighted by
    # c_k lambda and c^E_k) give grad_t L = dE_c/dt + J^T lambda of the oracle,
    # whose Jacobian is taken by the complex step through O-det
    _lib()
    from oracle.gradient import grad_t_lagrangian
    from tests.ph_subset_interp import SubsetAdjoint
    H = {"C4H6": lambda: build_ppp('polyene', 4), "C6H8": lambda: build_ppp('polyene', 6)}[name]()
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=3, K_H=K_H)
    rng = np.random.default_rng(21)
    t = rng.uniform(-0.1, 0.1, P.cc.n_amp)
    lam = rng.uniform(-0.1, 0.1, P.cc.n_amp)
    g_ref = grad_t_lagrangian(P, t, lam)
    lm = LayoutMap(P.cc.manifold, H.occ_of_pair, H.vir_of_pair, H.n_orb, ppq.amp_layout(3))
    sa = SubsetAdjoint(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, 3, K_H)
    g, _ = sa.lagrangian_gradient(lm.to_layout(t), lm.to_layout(lam))
    g2 = lm.from_layout(sa.fill_copies(g, lm))
    assert np.abs(g_ref).max() > 0.05
    assert np.abs(g2 - g_ref).max() < 1e-12


@pytest.mark.parametrize("K,K_H,sites", [(3, 3, 8), (3, 2, 10)])
def test_adjoint_tables_integral_keys_by_central_differences(K, K_H, sites):
    # dL/d(integral key) of the reverse pass against central differences of
    # the Lagrangian in the bare truncated integrals, for the ten keys of
    # largest gradient (one dense element may feed several keys: the keys of
    # an element are summed)
    _lib()
    from tests.ph_subset_interp import SubsetAdjoint
    H = build_ppp('polyene', sites)
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=K, K_H=K_H)
    rng = np.random.default_rng(22)
    lm = LayoutMap(P.cc.manifold, H.occ_of_pair, H.vir_of_pair, H.n_orb, ppq.amp_layout(K))
    t = lm.to_layout(rng.uniform(-0.1, 0.1, P.cc.n_amp))
    lam = lm.to_layout(rng.uniform(-0.1, 0.1, P.cc.n_amp))
    sa = SubsetAdjoint(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K, K_H)
    uniq = lm.to_layout(np.arange(1, P.cc.n_amp + 1)) != 0
    _, gv = sa.lagrangian_gradient(t, lam)
    dense = {}
    for (labels, j), val in gv.items():
        kind = sa.keys[len(labels)][j]
        orbs = [o for X in labels for o in (sa.occ[X], sa.vir[X])]
        el = (kind[0],) + tuple(orbs[i] for i in kind[1:(3 if kind[0] == 'h' else 5)])
        dense[el] = dense.get(el, 0.0) + val
    top = sorted(dense.items(), key=lambda kv: -abs(kv[1]))[:10]
    assert abs(top[0][1]) > 0.05

    def lag(el, delta):
        arr = sa.hp if el[0] == 'h' else sa.v
        arr[el[1:]] += delta
        r, e = sa.residual(t)
        arr[el[1:]] -= delta
        return e + np.sum(lam[uniq] * r[uniq])

    eps = 1e-5
    for el, val in top:
        fd = (lag(el, eps) - lag(el, -eps)) / (2 * eps)
        assert abs(fd - val) < 1e-8, (el, fd, val)
