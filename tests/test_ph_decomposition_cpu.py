"""The residual by Hamiltonian pieces (tests/ph_decomposition.py) against the
oracle's full-space residual.

At N = 4 (octatetraene PPP, 16 spin orbitals) and random amplitudes
(uniform +-0.1), summing <mu| exp(-B) H_S exp(B) exp(A) |Phi> over the pieces
H_S reproduces every residual element and the energy to FP64 rounding, for
PH with three- and two-label integrals and for PQ.  Controls: without the
exp(-B) transform, or with A cut down to the clusters inside S, the sum is
wrong; with A widened to clusters that leave U, it is unchanged (those
clusters leave a label excited).  With PPQ_LONG_CHECKS=1 the same holds at
N = 5 (H10), where terms reach five labels (about 4 min per case; both cases
agreed to 4e-15 when last run).
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from workloads import build_ppp, build_hchain
from oracle.detcc import Problem
from tests.ph_decomposition import Decomposed, _expv


@pytest.fixture(scope="module")
def system():
    return build_ppp('polyene', 8)


def _case(H, K, K_H):
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=K, K_H=K_H)
    t = np.random.default_rng(1609 + 10 * K + K_H).uniform(-0.1, 0.1, P.cc.n_amp)
    R, e = P.residual(t)
    return P, t, R, e


_BUILT = {}


def _built(H, K, K_H):
    if (K, K_H) not in _BUILT:
        P, t, R, e = _case(H, K, K_H)
        D = Decomposed(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K_H, P.cc.manifold)
        _BUILT[(K, K_H)] = (D, t, R, e)
    return _BUILT[(K, K_H)]


@pytest.mark.parametrize("K,K_H", [(3, 3), (3, 2), (2, 2)])
def test_pieces_sum_to_the_residual(system, K, K_H):
    D, t, R, e = _built(system, K, K_H)
    R2, e2 = D.residual(t)
    assert np.abs(R).max() > 0.05
    assert np.abs(R2 - R).max() < 1e-12
    assert abs(e2 - e) < 1e-12


class _Variant(Decomposed):
    mode = None

    def piece_term(self, C, M, S):
        H_S = dict(self.pieces)[S]
        E = S - M
        U = M | E
        zero = sp.csr_matrix((self.jw.dim, self.jw.dim))
        if self.mode == "wide":
            A = sum((C[L] for L in self.cluster_sets if L & E), zero)
        elif self.mode == "internal":
            A = sum((C[L] for L in self.cluster_sets if L <= S), zero)
        else:
            A = sum((C[L] for L in self.cluster_sets if L <= U and L & E), zero)
        B = sum((C[L] for L in self.cluster_sets if L <= M and L & S), zero)
        if self.mode == "no_transform":
            B = zero
        w = _expv(A, self.ref)
        w = _expv(B, w)
        return _expv(B, H_S @ w, -1.0)


@pytest.mark.parametrize("mode,exact", [("wide", True), ("no_transform", False), ("internal", False)])
def test_decomposition_controls(system, mode, exact):
    D, t, R, _ = _built(system, 3, 3)
    V = _Variant.__new__(_Variant)
    V.__dict__.update(D.__dict__)
    V.mode = mode
    err = np.abs(V.residual(t)[0] - R).max()
    if exact:
        assert err < 1e-12
    else:
        assert err > 1e-3


@pytest.mark.slow
@pytest.mark.skipif(os.environ.get("PPQ_LONG_CHECKS") != "1",
                    reason="about 4 min per case; set PPQ_LONG_CHECKS=1")
@pytest.mark.parametrize("K_H", [3, 2])
def test_pieces_sum_to_the_residual_n5(K_H):
    """N = 5 (H10): terms of up to five labels (|M| = 3 with two extra labels)."""
    H = build_hchain(10, 1.6)
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=3, K_H=K_H)
    t = np.random.default_rng(9).uniform(-0.1, 0.1, P.cc.n_amp)
    R, e = P.residual(t)
    R2, e2 = Decomposed(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K_H, P.cc.manifold).residual(t)
    assert np.abs(R2 - R).max() < 1e-12 and abs(e2 - e) < 1e-12
