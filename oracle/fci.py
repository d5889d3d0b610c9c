"""Determinant strings and brute-force FCI (textbook; used to pin the statement
that PQ is exact for four electrons in four orbitals and PH for six in six,
Abstract and Theory section).

A determinant is |I_alpha I_beta> = a+(alpha string, ascending) a+(beta string,
ascending) |vac>, spin orbitals ordered all-alpha then all-beta.  Because every
operator used here conserves the alpha and the beta electron counts
separately, alpha and beta parts act independently without cross signs.
"""
from itertools import combinations
import numpy as np
import scipy.sparse as sp


class Strings:
    """All bit strings of n_elec electrons in n_orb spatial orbitals."""

    def __init__(self, n_orb, n_elec):
        self.n_orb, self.n_elec = n_orb, n_elec
        self.list = [sum(1 << p for p in c) for c in combinations(range(n_orb), n_elec)]
        self.index = {s: i for i, s in enumerate(self.list)}
        self.n = len(self.list)
        self._E = None

    @staticmethod
    def apply(s, ops):
        """Apply elementary operators right to left.  ops: list of (p, dagger).
        Returns (new string, sign) or (None, 0)."""
        sign = 1
        for p, dag in reversed(ops):
            occ = (s >> p) & 1
            if dag == occ:
                return None, 0
            if bin(s & ((1 << p) - 1)).count("1") & 1:
                sign = -sign
            s ^= 1 << p
        return s, sign

    def op_map(self, ops):
        """(src, dst, sign) arrays of the string operator given by ops."""
        src, dst, sg = [], [], []
        for i, s in enumerate(self.list):
            t, g = self.apply(s, ops)
            if t is not None:
                src.append(i); dst.append(self.index[t]); sg.append(g)
        return (np.array(src, dtype=np.int64), np.array(dst, dtype=np.int64),
                np.array(sg, dtype=float))

    def E(self):
        """Sparse matrices of the one-body operators a+_p a_q, indexed [p][q]."""
        if self._E is None:
            n = self.n_orb
            self._E = [[None] * n for _ in range(n)]
            for p in range(n):
                for q in range(n):
                    src, dst, sg = self.op_map([(p, 1), (q, 0)])
                    self._E[p][q] = sp.csr_matrix((sg, (dst, src)), shape=(self.n, self.n))
        return self._E


def sigma(strings, h1, eri, C):
    """H C for the spin-free Hamiltonian sum h1_pq E_pq + 1/2 sum (pq|rs)(E_pq E_rs
    - delta_qr E_ps), with C[I_alpha, I_beta] (equal alpha and beta electron
    counts, so both spins share one string space)."""
    n = h1.shape[0]
    E = strings.E()
    k = h1 - 0.5 * np.einsum('prrq->pq', eri)
    D = np.empty((n, n) + C.shape, dtype=np.result_type(C, eri))
    for r in range(n):
        for s in range(n):
            D[r, s] = E[r][s] @ C + (E[r][s] @ C.T).T
    G = np.tensordot(eri, D, axes=([2, 3], [0, 1]))
    out = np.tensordot(k, D, axes=([0, 1], [0, 1]))
    for p in range(n):
        for q in range(n):
            X = 0.5 * G[p, q]
            out += E[p][q] @ X + (E[p][q] @ X.T).T
    return out


def fci_energy(h, eri, n_alpha, e_const=0.0):
    """Lowest FCI energy in the M_s = 0 sector with n_alpha = n_beta electrons.
    Dense diagonalisation for small spaces, Lanczos (scipy eigsh) otherwise."""
    n = h.shape[0]
    S = Strings(n, n_alpha)
    dim = S.n * S.n
    if dim <= 800:
        Hm = np.empty((dim, dim))
        for j in range(dim):
            c = np.zeros(dim); c[j] = 1.0
            Hm[:, j] = sigma(S, h, eri, c.reshape(S.n, S.n)).ravel()
        return float(np.linalg.eigvalsh(0.5 * (Hm + Hm.T))[0]) + e_const
    from scipy.sparse.linalg import LinearOperator, eigsh
    op = LinearOperator((dim, dim), dtype=float,
                        matvec=lambda x: sigma(S, h, eri, x.reshape(S.n, S.n)).ravel())
    # start from the closed-shell determinant of the lowest orbitals
    v0 = np.zeros((S.n, S.n)); v0[0, 0] = 1.0
    w = eigsh(op, k=1, which='SA', v0=v0.ravel() + 1e-3, tol=1e-13, maxiter=5000)[0]
    return float(w[0]) + e_const
