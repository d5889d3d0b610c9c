"""The three-pair (PH) residual in the site formulation, on the CPU (test
infrastructure; the site-basis statement the three-pair kernels are to follow).

Each pairing label is a site with 16 local states |m> = E^m|ref> (m a 4-bit
monomial mask, as in ``tables``).  A residual element mu with label set M is
the sum over Hamiltonian pieces H_S (integrals whose orbitals carry exactly
the labels S) of

    <mu (x) ref_E| exp(-B) H_S exp(B) exp(A) |ref_U>,   E = S \\ M, U = M + E,

with A the clusters inside U that meet E and B the clusters inside M that
meet S (the decomposition checked in ``tests/ph_decomposition.py``).  Every
quantity here lives in the zero-charge, zero-S_z sector of the sites U (at
most 4900 states for four sites) in the monomial basis:

* cluster operators E_P^a E_Q^b E_R^c of the layout (t1, t2, t3 channels of
  ``ppq_amp_layout(3)``), applied with the graded rule: E^a on site j of
  |m_0 m_1 ...> gives prod[a, m_j] (-1)^{|a| (|m_0| + ... + |m_{j-1}|)};
* H_S from the generated integral keys (20 per site, 232 per pair, 576 per
  triple) as second-quantised terms, each fermion operator acting on its site
  by the one-site Jordan-Wigner table and picking up (-1)^{|m_0| + ... +
  |m_{j-1}|} from the sites before it.

The result is written in the C-ABI layout (sorted label order), so a test can
compare it with the oracle through the layout map.
"""
import itertools

import numpy as np
import scipy.sparse as sp

from paper_1609_00077_gb300 import tables as T
from tests.ph_decomposition import bare_truncated_hamiltonian

PAR = np.array([bin(m).count("1") & 1 for m in range(16)])
PROD = T.local_product_table()
QN = np.array([T.qn(m) for m in range(16)])


def _local_fermion_tables():
    """new[x, dag, m], sign[x, dag, m]: a_x or a+_x (x = 0 o_up, 1 o_dn,
    2 v_up, 3 v_dn) on the one-site state E^m|ref>; sign 0 if it vanishes."""
    S1 = T.Space(1)
    new = np.zeros((4, 2, 16), dtype=np.int64)
    sgn = np.zeros((4, 2, 16), dtype=np.int64)
    for x in range(4):
        for dag in (0, 1):
            for m in range(16):
                st, s = S1.jw[(m,)]
                st2, s2 = T._apply(st, [(x, dag)])
                if st2 is None:
                    continue
                (m2,), s3 = S1.inv[st2]
                new[x, dag, m] = m2
                sgn[x, dag, m] = s * s2 * s3
    return new, sgn


FNEW, FSGN = _local_fermion_tables()

# operator structures depend only on the sector size, the positions and the
# channel / key lists, not on the system: shared by every instance
_SECTORS = {}
_CLUSTER = {}
_PIECE = {}


class Sector:
    """Zero-charge, zero-S_z states of k sites, as rows of monomials."""

    def __init__(self, k):
        self.k = k
        allst = np.array(list(itertools.product(range(16), repeat=k)), dtype=np.int64).reshape(-1, k)
        q = QN[allst].sum(1)
        self.states = allst[(q[:, 0] == 0) & (q[:, 1] == 0)]
        self.dim = len(self.states)
        self.lookup = -np.ones(16 ** k, dtype=np.int64)
        self.lookup[self._code(self.states)] = np.arange(self.dim)

    def _code(self, st):
        c = np.zeros(len(st), dtype=np.int64)
        for j in range(self.k):
            c = c * 16 + st[:, j]
        return c

    def index(self, st):
        return self.lookup[self._code(st)]

    @staticmethod
    def _before(st, j):
        """Parity of the monomials on the sites before j."""
        p = np.zeros(len(st), dtype=np.int64)
        for i in range(j):
            p ^= PAR[st[:, i]]
        return p

    def monomial(self, st, j, a):
        """E^a on site j: (new states, sign); sign 0 where it vanishes."""
        m = st[:, j]
        ok = (m & a) == 0
        s = np.where(ok, PROD[a, m] * np.where(PAR[a] & self._before(st, j), -1, 1), 0)
        out = st.copy()
        out[:, j] = m | a
        return out, s

    def fermion(self, st, j, x, dag):
        m = st[:, j]
        s = FSGN[x, dag, m] * np.where(self._before(st, j), -1, 1)
        out = st.copy()
        out[:, j] = FNEW[x, dag, m]
        return out, s

    def matrix(self, rows, cols, vals):
        keep = vals != 0
        return sp.csr_matrix((vals[keep], (rows[keep], cols[keep])), shape=(self.dim, self.dim))


class SiteInterp:
    def __init__(self, h, eri, occ, vir, K_H, desc3):
        self.occ = [int(i) for i in occ]
        self.vir = [int(a) for a in vir]
        self.N = len(self.occ)
        self.K_H = K_H
        self.hp, self.v, _ = bare_truncated_hamiltonian(h, eri, np.array(self.occ), np.array(self.vir), K_H)
        o = self.occ
        self.f = h + 2.0 * np.einsum('pqii->pq', eri[:, :, o][:, :, :, o]) \
            - np.einsum('piiq->pq', eri[:, o][:, :, o])
        self.A1 = [int(d[1]) for d in desc3 if d[0] == 1]
        self.A2 = [(int(d[1]), int(d[2])) for d in desc3 if d[0] == 2]
        self.A3 = [tuple(int(x) for x in d[1:4]) for d in desc3 if d[0] == 3]
        self.keys = {1: T.site_integral_keys(), 2: T.pair_integral_keys(), 3: T.triple_integral_keys()}
        self.terms = {k: T._hamiltonian_terms(self.keys[k]) for k in (1, 2, 3)}

    def sector(self, k):
        if k not in _SECTORS:
            _SECTORS[k] = Sector(k)
        return _SECTORS[k]

    # ------------------------------------------------------------ operators
    def _cluster_structure(self, k, pos):
        """COO of every channel of the cluster on positions pos of a k-site
        sector: (rows, cols, channel, sign)."""
        chans = {1: [(m,) for m in self.A1], 2: self.A2, 3: self.A3}[len(pos)]
        key = (k, pos, tuple(chans))
        if key not in _CLUSTER:
            S = self.sector(k)
            R, C, CH, SG = [], [], [], []
            for c, mons in enumerate(chans):
                st = S.states
                s = np.ones(S.dim, dtype=np.int64)
                for j, a in reversed(list(zip(pos, mons))):
                    st, s2 = S.monomial(st, j, a)
                    s = s * s2
                idx = np.where(s != 0, S.index(np.where((s != 0)[:, None], st, 0)), -1)
                ok = (s != 0) & (idx >= 0)
                R.append(idx[ok]); C.append(np.flatnonzero(ok)); CH.append(np.full(ok.sum(), c)); SG.append(s[ok])
            _CLUSTER[key] = tuple(np.concatenate(a) for a in (R, C, CH, SG))
        return _CLUSTER[key]

    def cluster(self, k, pos, amps):
        R, C, CH, SG = self._cluster_structure(k, pos)
        return self.sector(k).matrix(R, C, SG * amps[CH])

    def _piece_structure(self, k, pos):
        """COO of H_S on positions pos of a k-site sector: (rows, cols, key, coef)."""
        key = (k, pos)
        if key not in _PIECE:
            S = self.sector(k)
            R, C, J, V = [], [], [], []
            for j, coef, ops in self.terms[len(pos)]:
                st = S.states
                s = np.ones(S.dim, dtype=np.int64)
                for so, dag in reversed(ops):
                    st, s2 = S.fermion(st, pos[so // 4], so % 4, dag)
                    s = s * s2
                q = QN[st].sum(1)
                ok = (s != 0) & (q[:, 0] == 0) & (q[:, 1] == 0)
                idx = np.where(ok, S.index(np.where(ok[:, None], st, 0)), -1)
                ok &= idx >= 0
                R.append(idx[ok]); C.append(np.flatnonzero(ok)); J.append(np.full(ok.sum(), j))
                V.append(coef * s[ok])
            _PIECE[key] = tuple(np.concatenate(a) for a in (R, C, J, V))
        return _PIECE[key]

    def piece(self, k, pos, labels):
        """H_S for the labels (sorted) at positions pos of a k-site sector."""
        orbs = []
        for X in labels:
            orbs += [self.occ[X], self.vir[X]]
        vals = []
        for key in self.keys[len(labels)]:
            if key[0] == "h":
                vals.append(self.hp[orbs[key[1]], orbs[key[2]]])
            else:
                vals.append(self.v[orbs[key[1]], orbs[key[2]], orbs[key[3]], orbs[key[4]]])
        vals = np.array(vals)
        R, C, J, V = self._piece_structure(k, pos)
        return self.sector(k).matrix(R, C, V * vals[J])

    # ------------------------------------------------------------ residual
    def amplitudes(self, v):
        """Cluster amplitudes by sorted label tuple from the layout vector."""
        N = self.N
        t1 = v[:3 * N].reshape(N, 3)
        t2 = v[3 * N:3 * N + 29 * N * N].reshape(N, N, 29)
        t3 = v[3 * N + 29 * N * N:].reshape(N, N, N, len(self.A3))
        amp = {}
        for X in range(N):
            amp[(X,)] = t1[X]
        for X, Y in itertools.combinations(range(N), 2):
            amp[(X, Y)] = t2[X, Y]
        for L in itertools.combinations(range(N), 3):
            amp[L] = t3[L]
        return amp

    def _ops(self, amp, U, select, mats):
        """Sum of the clusters L inside U with select(L), on U's sector."""
        k = len(U)
        at = {X: i for i, X in enumerate(U)}
        Sec = self.sector(k)
        out = sp.csr_matrix((Sec.dim, Sec.dim))
        for L, tl in amp.items():
            if set(L) <= set(U) and select(set(L)):
                pos = tuple(at[X] for X in L)
                if (k, pos, L) not in mats:
                    mats[(k, pos, L)] = self.cluster(k, pos, tl)
                out = out + mats[(k, pos, L)]
        return out

    def _ref(self, k):
        Sec = self.sector(k)
        ref = np.zeros(Sec.dim)
        ref[Sec.index(np.zeros((1, k), dtype=np.int64))[0]] = 1.0
        return ref

    def _read(self, M, U, w):
        """Components of a U-vector on the channels of M, reference elsewhere."""
        at = {X: i for i, X in enumerate(U)}
        chans = {1: [(m,) for m in self.A1], 2: self.A2, 3: self.A3}[len(M)]
        st = np.zeros((len(chans), len(U)), dtype=np.int64)
        for j, X in enumerate(M):
            st[:, at[X]] = [c[j] for c in chans]
        return w[self.sector(len(U)).index(st)]

    def term(self, M, S, amp, mats):
        """exp(-B) H_S exp(B) exp(A) |ref_U> on the sector of U = M + S."""
        U = tuple(sorted(set(M) | set(S)))
        at = {X: i for i, X in enumerate(U)}
        E = set(S) - set(M)
        A = self._ops(amp, U, lambda L: bool(L & E), mats)
        B = self._ops(amp, U, lambda L: not (L & E) and L <= set(M) and bool(L & set(S)), mats)
        H_S = self.piece(len(U), tuple(at[X] for X in S), S)
        w = _expv(A, self._ref(len(U)))
        w = _expv(B, w)
        return U, _expv(B, H_S @ w, -1.0), H_S

    def residual(self, v):
        """R (same layout, sorted-order slots filled) and E_c at layout amplitudes v."""
        N = self.N
        amp = self.amplitudes(v)
        out = np.zeros_like(v)
        o1 = out[:3 * N].reshape(N, 3)
        o2 = out[3 * N:3 * N + 29 * N * N].reshape(N, N, 29)
        o3 = out[3 * N + 29 * N * N:].reshape(N, N, N, len(self.A3))
        pieces = [S for k in range(1, min(self.K_H, N) + 1) for S in itertools.combinations(range(N), k)]
        outputs = [M for k in range(1, min(3, N) + 1) for M in itertools.combinations(range(N), k)]
        mats = {}
        e = 0.0
        for S in pieces:
            U, w, H_S = self.term((), S, amp, mats)
            ref = self._ref(len(U))
            e += w @ ref - ref @ (H_S @ ref)
        for M in outputs:
            y = sum(self._read(M, *self.term(M, S, amp, mats)[:2]) for S in pieces)
            (o1 if len(M) == 1 else o2 if len(M) == 2 else o3)[M] = y
        return out, e

    # ------------------------------------------------------------ disjoint class
    def disjoint_term(self, M, S, amp, mats):
        """The contribution of H_S to the outputs on M when S and M share no
        label, as a closure row times link coefficients:

            sum_{s'} G_S[s'] (-1)^{sum_{s in S} |s'_s| #odd(mu before s)} Lambda(mu, s'),
            G_S[s'] = <ref_S| H_S exp(I_S) |s'>,   Lambda(mu, s') = <mu s'| exp(L) |ref_U>,

        I_S the clusters inside S, L the clusters inside U = M + S meeting both,
        s' over the zero-charge sector of S (mu has zero charge on M).  The
        sign moves the per-site factors of H_S exp(I_S) past the odd monomials
        of mu on the labels of M that precede them."""
        assert not set(M) & set(S)
        kS = len(S)
        I_S = self._ops(amp, tuple(S), lambda L: True, mats)
        H_S = self.piece(kS, tuple(range(kS)), S)
        row = _expv(I_S.T.tocsr(), H_S.T @ self._ref(kS))         # G_S as a row on S's sector
        U = tuple(sorted(set(M) | set(S)))
        at = {X: i for i, X in enumerate(U)}
        L = self._ops(amp, U, lambda L: bool(L & set(S)) and bool(L & set(M)), mats)
        w = _expv(L, self._ref(len(U)))
        SecS = self.sector(kS)
        chans = {1: [(m,) for m in self.A1], 2: self.A2, 3: self.A3}[len(M)]
        out = np.zeros(len(chans))
        nz = np.flatnonzero(row)
        for c, mu in enumerate(chans):
            st = np.zeros((len(nz), len(U)), dtype=np.int64)
            for j, X in enumerate(M):
                st[:, at[X]] = mu[j]
            sgn = np.ones(len(nz))
            for j, X in enumerate(S):
                st[:, at[X]] = SecS.states[nz, j]
                odd_before = sum(PAR[mu[i]] for i, Y in enumerate(M) if Y < X) & 1
                sgn *= np.where(PAR[SecS.states[nz, j]] & odd_before, -1.0, 1.0)
            out[c] = np.sum(row[nz] * sgn * w[self.sector(len(U)).index(st)])
        return out


def _expv(X, v, sign=1.0):
    out = v.copy()
    term = v
    for k in range(1, 64):
        term = (sign / k) * (X @ term)
        if not np.any(term):
            return out
        out = out + term
    raise RuntimeError("series did not terminate")


# ---------------------------------------------------------------- solver
def layout_denominators(si, f):
    """D for every sorted slot of the K = 3 layout: sum over the labels of
    (holes x f_ii - particles x f_aa), diagonal Fock (Jacobi update of the
    Implementation section); 1 on the unused copies."""
    N = si.N
    nh = np.array([bin(m & 3).count("1") for m in range(16)])
    npart = np.array([bin(m & 12).count("1") for m in range(16)])
    fo = np.array([f[i, i] for i in si.occ])
    fv = np.array([f[a, a] for a in si.vir])

    def d(labels, monos):
        return sum(nh[m] * fo[X] - npart[m] * fv[X] for X, m in zip(labels, monos))

    D = np.ones(3 * N + 29 * N * N + len(si.A3) * N ** 3)
    D1 = D[:3 * N].reshape(N, 3)
    D2 = D[3 * N:3 * N + 29 * N * N].reshape(N, N, 29)
    D3 = D[3 * N + 29 * N * N:].reshape(N, N, N, len(si.A3))
    mask = np.zeros(D.shape, dtype=bool)
    m1 = mask[:3 * N].reshape(N, 3)
    m2 = mask[3 * N:3 * N + 29 * N * N].reshape(N, N, 29)
    m3 = mask[3 * N + 29 * N * N:].reshape(N, N, N, len(si.A3))
    for X in range(N):
        D1[X] = [d((X,), (m,)) for m in si.A1]
        m1[X] = True
    for L in itertools.combinations(range(N), 2):
        D2[L] = [d(L, ab) for ab in si.A2]
        m2[L] = True
    for L in itertools.combinations(range(N), 3):
        D3[L] = [d(L, abc) for abc in si.A3]
        m3[L] = True
    return D, mask


def solve(si, f, r_tol=1e-10, e_tol=1e-12, max_iter=200, diis_dim=8, diis_start=3):
    """Jacobi steps t <- t + R/D on the sorted slots with Pulay DIIS on the
    steps.  Returns (t layout, E_c, ||R||, iterations, converged)."""
    D, mask = layout_denominators(si, f)
    t = np.zeros(D.shape)
    ts, es, e_old = [], [], None
    for it in range(1, max_iter + 1):
        R, e = si.residual(t)
        rn = float(np.linalg.norm(R[mask]))
        if e_old is not None and rn <= r_tol and abs(e - e_old) <= e_tol:
            return t, e, rn, it, True
        e_old = e
        step = np.where(mask, R / D, 0.0)
        ts.append(t + step); es.append(step[mask])
        ts, es = ts[-diis_dim:], es[-diis_dim:]
        t = ts[-1]
        if it >= diis_start and len(ts) > 1:
            m = len(ts)
            B = -np.ones((m + 1, m + 1))
            B[m, m] = 0.0
            G = np.array([[a @ b for b in es] for a in es])
            B[:m, :m] = G / np.abs(np.diag(G)).max()
            rhs = np.zeros(m + 1)
            rhs[m] = -1.0
            c = np.linalg.lstsq(B, rhs, rcond=None)[0][:m]
            t = sum(ci * ti for ci, ti in zip(c, ts))
    return t, e, rn, max_iter, False
