"""Jordan-Wigner fermion operators for small checks (test infrastructure).

Spin orbital p + n*s (s = 0 alpha, 1 beta) of n spatial orbitals is the
(p + n*s)-th Kronecker factor; basis state 0 of a factor is empty.  Operators
are scipy sparse matrices, either on the whole Fock space or restricted to the
sector of fixed alpha and beta electron numbers, where products are formed by
applying the factors to the sector's basis vectors (cheap) rather than by
multiplying full matrices.
"""
import numpy as np
import scipy.sparse as sp


def annihilators(nso):
    """a_k for k < nso on the 2^nso-dimensional Fock space."""
    I = sp.identity(2, format="csr")
    Z = sp.csr_matrix(np.diag([1.0, -1.0]))
    a = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]]))
    ops = []
    for k in range(nso):
        m = sp.csr_matrix(np.array([[1.0]]))
        for j in range(nso):
            m = sp.kron(m, Z if j < k else (a if j == k else I), format="csr")
        ops.append(m)
    return ops


class JW:
    """Operators of n spatial orbitals in the sector (n_alpha, n_beta)."""

    def __init__(self, n, n_alpha, n_beta):
        self.n = n
        nso = 2 * n
        self.a = annihilators(nso)
        self.ad = [x.T.tocsr() for x in self.a]
        idx = np.arange(2 ** nso)
        bits = (idx[:, None] >> (nso - 1 - np.arange(nso))[None, :]) & 1
        self.sector = np.flatnonzero((bits[:, :n].sum(1) == n_alpha) & (bits[:, n:].sum(1) == n_beta))
        self.dim = len(self.sector)
        self._inject = sp.csr_matrix((np.ones(self.dim), (self.sector, np.arange(self.dim))),
                                     shape=(2 ** nso, self.dim))
        self._E = {}

    def product(self, seq):
        """prod(seq) (leftmost factor applied last) restricted to the sector;
        seq must conserve both electron numbers."""
        X = self._inject
        for m in reversed(seq):
            X = m @ X
        return X.tocsr()[self.sector].tocsr()

    def E(self, p, q, s):
        """a+_{p s} a_{q s} on the sector."""
        key = (p, q, s)
        if key not in self._E:
            n = self.n
            self._E[key] = self.product([self.ad[p + n * s], self.a[q + n * s]])
        return self._E[key]

    def det(self, alpha, beta):
        """a+ (alpha ascending) a+ (beta ascending) |vac>, as a sector vector.
        Creators applied in descending spin-orbital order never pass an
        occupied orbital, so the state is +1 on its basis vector."""
        nso = 2 * self.n
        idx = 0
        for x in list(alpha) + [b + self.n for b in beta]:
            idx |= 1 << (nso - 1 - x)
        v = np.zeros(self.dim)
        pos = np.searchsorted(self.sector, idx)
        if pos == self.dim or self.sector[pos] != idx:
            raise ValueError("determinant outside the sector")
        v[pos] = 1.0
        return v

    def _lincomb(self, terms):
        """sum of coef * matrix over (coef, matrix) pairs, in one pass."""
        rows, cols, vals = [], [], []
        for c, m in terms:
            m = m.tocoo()
            rows.append(m.row); cols.append(m.col); vals.append(c * m.data)
        if not rows:
            return sp.csr_matrix((self.dim, self.dim))
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.dim, self.dim))

    def hamiltonian(self, h1, v2):
        """sum h1[p,q] E_pq + 1/2 sum v2[p,q,r,s] (E_pq E_rs - delta_qr E_ps),
        spin-summed; v2 in chemists' notation."""
        n = self.n
        terms = [(h1[p, q], self.E(p, q, s)) for s in range(2) for p in range(n)
                 for q in range(n) if h1[p, q] != 0.0]
        for s1 in range(2):
            for p in range(n):
                for q in range(n):
                    blk = v2[p, q]
                    if not np.any(blk):
                        continue
                    inner = self._lincomb([(blk[r, u], self.E(r, u, s2)) for s2 in range(2)
                                           for r in range(n) for u in range(n) if blk[r, u] != 0.0])
                    terms.append((0.5, self.E(p, q, s1) @ inner))
                    # the delta_qr E_ps term (same spin only)
                    terms += [(-0.5 * blk[q, u], self.E(p, u, s1)) for u in range(n) if blk[q, u] != 0.0]
        return self._lincomb(terms)

    def excitation(self, holes_a, parts_a, holes_b, parts_b, occ):
        """tau with tau|Phi> = +|D>: the particle creators then the hole
        annihilators (alpha, then beta), normalised by the sign of <D|tau|Phi>.
        Returns (tau on the sector, |D>)."""
        n = self.n
        seq = ([self.ad[x] for x in parts_a] + [self.a[x] for x in reversed(holes_a)]
               + [self.ad[x + n] for x in parts_b] + [self.a[x + n] for x in reversed(holes_b)])
        op = self.product(seq)
        ref = self.det(sorted(occ), sorted(occ))
        D = self.det(sorted(set(occ) - set(holes_a) | set(parts_a)),
                     sorted(set(occ) - set(holes_b) | set(parts_b)))
        sgn = float(D @ (op @ ref))
        assert abs(abs(sgn) - 1.0) < 1e-12
        return sgn * op, D
