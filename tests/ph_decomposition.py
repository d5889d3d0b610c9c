"""The residual as a sum over Hamiltonian pieces, each with only the clusters
that reach it (test infrastructure; a check of the three-pair formulation).

Write the Hamiltonian as H = sum_S H_S, H_S the part whose orbitals carry
exactly the label set S (|S| <= K_H), and the cluster operator as
T = sum_L T_L, T_L the amplitudes whose orbitals carry exactly the labels L
(|L| <= K; Eq. decompose).  For an output mu with label set M, and E = S \\ M,
U = M + E,

    <mu| exp(-T) H_S exp(T) |Phi> = <mu| exp(-B) H_S exp(B) exp(A) |Phi>,

    A = sum of T_L with L inside U and L meeting E,
    B = sum of T_L with L inside M and L meeting S.

Why: a cluster with a label outside U leaves that label excited (neither H_S
nor <mu| touches it); clusters inside M that miss S commute with H_S and
cancel between exp(-T) and exp(T); every cluster of A excites a label of E,
where <mu| holds the reference, so exp(-A) acting to the left on <mu| is the
identity.  Summing over S gives R_mu exactly, with at most |M| + K_H labels
per term: for PH (K = K_H = 3) a six-label term per (M, S) pair, O(N^6) per
residual -- the cost of the exact model.

This module evaluates that sum with sparse Jordan-Wigner operators in the
determinant space, independently of the oracle, so that a test can hold it
against the oracle's full-space residual.  It is a statement of the
formulation the three-pair kernels are to follow, not a fast evaluator.
"""
import itertools

import numpy as np
import scipy.sparse as sp

from tests.jw import JW


def bare_truncated_hamiltonian(h, eri, occ, vir, K_H):
    """(h', v'): v' keeps (pq|rs) when p, q, r, s carry at most K_H labels;
    h' = f - sum_i [2 v'(pq|ii) - v'(pi|iq)] with f the full Fock matrix, so
    that normal ordering gives back f and the truncated two-body part."""
    n = h.shape[0]
    lab = np.empty(n, dtype=np.int64)
    lab[occ] = np.arange(len(occ))
    lab[vir] = np.arange(len(vir))
    v = eri.copy()
    for p, q, r, s in itertools.product(range(n), repeat=4):
        if len({lab[p], lab[q], lab[r], lab[s]}) > K_H:
            v[p, q, r, s] = 0.0
    f = h + 2.0 * np.einsum('pqii->pq', eri[:, :, occ][:, :, :, occ]) \
        - np.einsum('piiq->pq', eri[:, occ][:, :, occ])
    hp = f - 2.0 * np.einsum('pqii->pq', v[:, :, occ][:, :, :, occ]) \
        + np.einsum('piiq->pq', v[:, occ][:, :, occ])
    return hp, v, lab


def _expv(X, v, sign=1.0):
    """exp(sign X) v for a nilpotent X (the series ends on its own)."""
    out = v.copy()
    term = v
    for k in range(1, 64):
        term = (sign / k) * (X @ term)
        if not np.any(term):
            return out
        out = out + term
    raise RuntimeError("series did not terminate")


class Decomposed:
    """Residual by Hamiltonian pieces.  manifold: list of excitations
    (alpha holes, alpha particles, beta holes, beta particles) of spatial
    orbitals; tau_D maps the reference to +|D>."""

    def __init__(self, h, eri, occ, vir, K_H, manifold):
        occ = [int(i) for i in occ]
        vir = [int(a) for a in vir]
        n = h.shape[0]
        assert 2 * len(occ) == n
        self.jw = JW(n, len(occ), len(occ))
        hp, v, lab = bare_truncated_hamiltonian(h, eri, np.array(occ), np.array(vir), K_H)
        occ_s = sorted(occ)
        self.ref = self.jw.det(occ_s, occ_s)
        self.taus, self.dets, self.labels = [], [], []
        for ah, ap, bh, bp in manifold:
            tau, D = self.jw.excitation(ah, ap, bh, bp, occ_s)
            self.taus.append(tau)
            self.dets.append(D)
            self.labels.append(frozenset(int(lab[x]) for x in (*ah, *ap, *bh, *bp)))
        self.cluster_sets = sorted(set(self.labels), key=lambda L: (len(L), sorted(L)))
        # Hamiltonian pieces by exact label set
        N = len(occ)
        self.pieces = []
        for k in range(1, min(K_H, N) + 1):
            for S in itertools.combinations(range(N), k):
                S = frozenset(S)
                m1 = np.array([[{lab[p], lab[q]} == S for q in range(n)] for p in range(n)])
                h1 = np.where(m1, hp, 0.0)
                m2 = np.zeros(v.shape, dtype=bool)
                for p, q, r, s in itertools.product(range(n), repeat=4):
                    m2[p, q, r, s] = {lab[p], lab[q], lab[r], lab[s]} == S
                v2 = np.where(m2, v, 0.0)
                if np.any(h1) or np.any(v2):
                    self.pieces.append((S, self.jw.hamiltonian(h1, v2)))

    def _clusters(self, t):
        C = {L: sp.csr_matrix((self.jw.dim, self.jw.dim)) for L in self.cluster_sets}
        for tk, tau, L in zip(t, self.taus, self.labels):
            C[L] = C[L] + tk * tau
        return C

    def piece_term(self, C, M, S):
        """exp(-B) H_S exp(B) exp(A) |Phi> for outputs on M (a vector; its
        component on <mu| is the contribution of H_S to R_mu)."""
        H_S = dict(self.pieces)[S]
        E = S - M
        U = M | E
        zero = sp.csr_matrix((self.jw.dim, self.jw.dim))
        A = sum((C[L] for L in self.cluster_sets if L <= U and L & E), zero)
        B = sum((C[L] for L in self.cluster_sets if L <= M and L & S), zero)
        w = _expv(A, self.ref)
        w = _expv(B, w)
        w = H_S @ w
        return _expv(B, w, -1.0)

    def residual(self, t):
        """(R over the manifold, correlation energy)."""
        C = self._clusters(t)
        R = np.zeros(len(self.taus))
        by_M = {}
        for k, L in enumerate(self.labels):
            by_M.setdefault(L, []).append(k)
        for M, ks in by_M.items():
            y = sum(self.piece_term(C, M, S) for S, _ in self.pieces)
            for k in ks:
                R[k] = self.dets[k] @ y
        e = 0.0
        for S, H_S in self.pieces:
            e += self.ref @ self.piece_term(C, frozenset(), S) - self.ref @ (H_S @ self.ref)
        return R, e
