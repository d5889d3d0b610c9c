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
