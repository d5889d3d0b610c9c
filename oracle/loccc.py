"""O-loc: the PQ / PH residual assembled from local determinant-space problems
(test infrastructure only; see the package header).

Why it is exact.  With H_N = F_N + W_N^(K_H), every connected term of
<mu| exp(-T) H_N exp(T) |Phi> contains one Hamiltonian element (at most K_H
labels) and amplitudes that are each contracted with it, so its labels lie in
labels(mu) + labels(H element): at most K + K_H labels (Theory section: all
tensors are block-decomposed over pairing labels).  Write r_mu[L] for the sum of
the terms whose label set is exactly L, and R^(L')_mu for the residual of the
problem restricted to the orbitals of the labels in L' (amplitudes and
integrals restricted to L', Fock operator still the full one).  Then
R^(L') = sum_{L subset of L'} r[L]; Moebius inversion gives r[L], and summing
over L containing labels(mu) with |L| <= K + K_H gives

    R_mu = sum_{L' containing labels(mu), |L'| <= K+K_H} c_|L'| R^(L')_mu,
    c_k  = sum_{j=0}^{K+K_H-k} (-1)^j binom(N-k, j).

The same holds for the energy with labels(mu) empty and K + K_H replaced by K_H.
With untruncated integrals (K_H = -1) an element (pq|rs) carries at most four
labels, so the bounds read K + 4 and 4.
Each local problem is solved with ``detcc.DetCC`` in its own determinant space
(orbital order preserved); amplitudes and residuals are mapped between the
global and local excitation operators with the sign relating the two
determinant conventions.
"""
from itertools import combinations
from math import comb
import numpy as np

from .fci import Strings
from .detcc import DetCC, truncated_hamiltonian, enumerate_manifold, _side_ops


def _moebius_coeff(N, k, kmax):
    return sum((-1) ** j * comb(N - k, j) for j in range(0, kmax - k + 1))


class LocalAssembly:
    """Residual and energy of a PQ/PH problem by local inclusion-exclusion."""

    def __init__(self, h, eri, occ_of_pair, vir_of_pair, K, K_H=0, subsets=None, truncated=None):
        """subsets: optional list of label subsets; when given, only those local
        problems are built and residual() returns their partial sum (used to
        time a bounded sample of a large problem, and to split one residual
        over processes).  truncated: optional result of truncated_hamiltonian
        for these integrals, pairing and K_H, computed once by the caller (h
        and eri are then not read)."""
        self.K = K
        self.K_H = K if K_H == 0 else K_H
        # labels one Hamiltonian element can carry (four for untruncated integrals)
        self.span_H = 4 if self.K_H < 0 else self.K_H
        self.occ = np.asarray(occ_of_pair); self.vir = np.asarray(vir_of_pair)
        self.N = len(self.occ)
        if truncated is None:
            truncated = truncated_hamiltonian(h, eri, self.occ, self.vir, self.K_H)
        self.hp, self.vt, self.f, self.e_ref = truncated
        self.manifold = enumerate_manifold(self.occ, self.vir, K)
        self.index = {d: k for k, d in enumerate(self.manifold)}
        self.global_ref = sum(1 << int(i) for i in self.occ)
        kmax = K + self.span_H
        self.kmax = kmax
        self.locals = []
        if subsets is not None:
            for Lset in subsets:
                self.locals.append(self._local(tuple(sorted(Lset))))
            return
        for m in range(1, min(kmax, self.N) + 1):
            for Lset in combinations(range(self.N), m):
                self.locals.append(self._local(Lset))

    def _labels(self, d):
        if not hasattr(self, "_lab"):
            self._lab = {}
            for k, (i, a) in enumerate(zip(self.occ, self.vir)):
                self._lab[int(i)] = k; self._lab[int(a)] = k
        return {self._lab[x] for x in d[0] + d[1] + d[2] + d[3]}

    def _local(self, Lset):
        orbs = sorted([int(self.occ[k]) for k in Lset] + [int(self.vir[k]) for k in Lset])
        pos = {p: i for i, p in enumerate(orbs)}
        locc = [pos[int(self.occ[k])] for k in Lset]
        lvir = [pos[int(self.vir[k])] for k in Lset]
        # local bare Hamiltonian: full Fock restricted, minus the mean field of
        # the local occupied orbitals only
        o = np.array(orbs)
        occL = np.array([int(self.occ[k]) for k in Lset])
        vt = self.vt
        h_loc = (self.f[np.ix_(o, o)]
                 - 2.0 * vt[np.ix_(o, o, occL, occL)].diagonal(axis1=2, axis2=3).sum(-1)
                 + vt[np.ix_(o, occL, occL, o)].diagonal(axis1=1, axis2=2).sum(-1))
        v_loc = vt[np.ix_(o, o, o, o)]
        # local manifold = global excitations whose labels lie in Lset
        if not hasattr(self, "_by_labels"):
            self._by_labels = {}
            for d in self.manifold:
                self._by_labels.setdefault(frozenset(self._labels(d)), []).append(d)
        glob, locm = [], []
        for m in range(1, len(Lset) + 1):
            for sub in combinations(Lset, m):
                for d in self._by_labels.get(frozenset(sub), []):
                    glob.append(self.index[d])
                    locm.append(tuple(tuple(pos[x] for x in part) for part in d))
        order = np.argsort(glob, kind="stable")
        glob = [glob[i] for i in order]
        locm = [locm[i] for i in order]
        cc = DetCC(len(orbs), locc, lvir, self.K, manifold=locm)
        # sign between the global and local operator conventions
        lref = sum(1 << i for i in locc)
        sgn = np.empty(len(locm))
        for k, (d, dl) in enumerate(zip((self.manifold[g] for g in glob), locm)):
            s = 1
            for (hh, pp), (hl, pl) in (((d[0], d[1]), (dl[0], dl[1])), ((d[2], d[3]), (dl[2], dl[3]))):
                _, sg = Strings.apply(self.global_ref, _side_ops(hh, pp))
                _, sl = Strings.apply(lref, _side_ops(hl, pl))
                s *= sg * sl
            sgn[k] = s
        e0 = cc.reference_energy(h_loc, v_loc)
        return dict(L=Lset, cc=cc, h=h_loc, v=v_loc, glob=np.array(glob, dtype=np.int64),
                    sgn=sgn, e0=e0)

    def residual(self, t):
        """(R over the global manifold, E_c) at global amplitudes t."""
        t = np.asarray(t, dtype=float)
        R = np.zeros(len(self.manifold))
        e = 0.0
        for loc in self.locals:
            m = len(loc['L'])
            tl = loc['sgn'] * t[loc['glob']]
            Rl, el = loc['cc'].residual(tl, loc['h'], loc['v'])
            R[loc['glob']] += _moebius_coeff(self.N, m, self.kmax) * loc['sgn'] * Rl
            if m <= self.span_H:
                e += _moebius_coeff(self.N, m, self.span_H) * (el - loc['e0'])
        # every amplitude's own label set must be counted from |labels(mu)| up
        return R, e
