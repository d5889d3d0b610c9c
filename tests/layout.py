"""Map between the oracle's amplitudes (one per excitation, operator tau_D with
tau_D|Phi> = +|D> in the determinant basis) and the C-ABI layout of
include/ppq.h (t1[P][k], t2[P][Q][k], t3[P][Q][R][k]; operators E_P^m,
E_P^a E_Q^b and E_P^a E_Q^b E_R^c).

Written from the layout documentation (ppq_amp_layout descriptors), with its
own Jordan-Wigner sign evaluation; it shares nothing with the CUDA path or the
oracle."""
import numpy as np


def _apply(state, ops):
    sign = 1
    for p, dag in reversed(ops):
        occ = (state >> p) & 1
        if dag == occ:
            return None, 0
        if bin(state & ((1 << p) - 1)).count("1") & 1:
            sign = -sign
        state ^= 1 << p
    return state, sign


def _mono_ops(m, occ_orb, vir_orb, n):
    # E^m = (a+_{v,a})^{b2} (a+_{v,b})^{b3} (a_{o,b})^{b1} (a_{o,a})^{b0};
    # determinant spin orbitals: alpha p -> p, beta p -> n + p
    ops = []
    if m & 4: ops.append((vir_orb, 1))
    if m & 8: ops.append((n + vir_orb, 1))
    if m & 2: ops.append((n + occ_orb, 0))
    if m & 1: ops.append((occ_orb, 0))
    return ops


def _par(m):
    return bin(m).count("1") & 1


def order_sign(monos, perm):
    """Sign of E^{monos[perm[0]]} E^{monos[perm[1]]} ... against
    E^{monos[0]} E^{monos[1]} ... (operators on different pairs): -1 for every
    inverted pair of odd monomials."""
    s = 1
    for i in range(len(perm)):
        for j in range(i + 1, len(perm)):
            if perm[i] > perm[j] and _par(monos[perm[i]]) and _par(monos[perm[j]]):
                s = -s
    return s


class LayoutMap:
    """K = 2 descriptors (3 columns) give the PQ layout; K = 3 descriptors
    (4 columns) add t3[P][Q][R][k], with all six orders of each triple."""

    def __init__(self, manifold, occ, vir, n_orb, desc):
        occ = [int(x) for x in occ]; vir = [int(x) for x in vir]
        self.N = N = len(occ)
        lab = {}
        for k in range(N):
            lab[occ[k]] = k; lab[vir[k]] = k
        ref = sum(1 << i for i in occ) | sum(1 << (n_orb + i) for i in occ)
        ch1 = {int(d[1]): c for c, d in enumerate(desc) if d[0] == 1}
        ch2 = {(int(d[1]), int(d[2])): c - 3 for c, d in enumerate(desc) if d[0] == 2}
        self.A3 = [tuple(int(x) for x in d[1:4]) for d in desc if d[0] == 3]
        ch3 = {m: c for c, m in enumerate(self.A3)}
        self.entries3 = []
        self.swap = {}
        for (a, b), k in ch2.items():
            self.swap[k] = (ch2[(b, a)], (-1) ** (_par(a) * _par(b)))
        self.entries = []
        for d, (ah, ap, bh, bp) in enumerate(manifold):
            mono = {}
            for x in ah: mono[lab[x]] = mono.get(lab[x], 0) | 1
            for x in bh: mono[lab[x]] = mono.get(lab[x], 0) | 2
            for x in ap: mono[lab[x]] = mono.get(lab[x], 0) | 4
            for x in bp: mono[lab[x]] = mono.get(lab[x], 0) | 8
            sites = sorted(mono)
            ops = []
            for X in sites:
                ops += _mono_ops(mono[X], occ[X], vir[X], n_orb)
            st, s = _apply(ref, ops)
            assert st is not None
            if len(sites) == 1:
                self.entries.append((d, sites[0], -1, ch1[mono[sites[0]]], s))
            elif len(sites) == 2:
                X, Y = sites
                self.entries.append((d, X, Y, ch2[(mono[X], mono[Y])], s))
            else:
                self.entries3.append((d, tuple(sites), ch3[tuple(mono[X] for X in sites)], s))
        self.n_amp = 3 * N + 29 * N * N + len(self.A3) * N ** 3
        self.n_unique = len(self.entries) + len(self.entries3)

    def _t3(self, v):
        N = self.N
        return v[3 * N + 29 * N * N:].reshape(N, N, N, len(self.A3))

    def _copies3(self, sites, ch):
        """(ordered labels, channel, sign) of the six stored copies."""
        monos = self.A3[ch]
        out = []
        for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
            m = tuple(monos[i] for i in perm)
            out.append((tuple(sites[i] for i in perm), self.A3.index(m), order_sign(monos, perm)))
        return out

    def to_layout(self, t):
        N = self.N
        out = np.zeros(self.n_amp)
        t1 = out[:3 * N].reshape(N, 3)
        t2 = out[3 * N:3 * N + 29 * N * N].reshape(N, N, 29)
        for d, X, Y, ch, s in self.entries:
            if Y < 0:
                t1[X, ch] = s * t[d]
            else:
                t2[X, Y, ch] = s * t[d]
                k2, sg = self.swap[ch]
                t2[Y, X, k2] = sg * s * t[d]
        if self.entries3:
            t3 = self._t3(out)
            for d, sites, ch, s in self.entries3:
                for lbl, c, sg in self._copies3(sites, ch):
                    t3[lbl + (c,)] = sg * s * t[d]
        return out

    def from_layout(self, v):
        N = self.N
        t1 = v[:3 * N].reshape(N, 3)
        t2 = v[3 * N:3 * N + 29 * N * N].reshape(N, N, 29)
        R = np.zeros(self.n_unique)
        for d, X, Y, ch, s in self.entries:
            R[d] = s * (t1[X, ch] if Y < 0 else t2[X, Y, ch])
        if self.entries3:
            t3 = self._t3(v)
            for d, sites, ch, s in self.entries3:
                R[d] = s * t3[sites + (ch,)]
        return R

    def mirror_error(self, v):
        """max |t2[P,Q,k] - sign t2[Q,P,swap k]| (consistency of the two copies)."""
        N = self.N
        t2 = v[3 * N:3 * N + 29 * N * N].reshape(N, N, 29)
        err = 0.0
        for P in range(N):
            for Q in range(N):
                if P == Q:
                    err = max(err, np.abs(t2[P, Q]).max())
                    continue
                for k in range(29):
                    k2, sg = self.swap[k]
                    err = max(err, abs(t2[P, Q, k] - sg * t2[Q, P, k2]))
        if self.A3:
            t3 = self._t3(v)
            for P in range(N):
                for Q in range(N):
                    for R in range(N):
                        if len({P, Q, R}) < 3:
                            err = max(err, np.abs(t3[P, Q, R]).max())
                        elif P < Q < R:
                            for k in range(len(self.A3)):
                                for lbl, c, sg in self._copies3((P, Q, R), k):
                                    err = max(err, abs(t3[lbl + (c,)] - sg * t3[P, Q, R, k]))
        return err
