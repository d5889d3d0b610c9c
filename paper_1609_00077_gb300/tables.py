"""Build-time generator of the site-algebra tables used by the CUDA kernels.

Each pairing label P (a quartet: alpha/beta occupied orbital, alpha/beta
virtual orbital -- Theory section) is treated as a site with a 16-state local
Fock space.  Local spin orbitals: 0 = o_up, 1 = o_dn, 2 = v_up, 3 = v_dn.

Every excitation is a product of per-site *monomials* E^m: m is a 4-bit mask,
bits 0/1 annihilate the occupied up/down orbital and bits 2/3 create the
virtual up/down orbital, E^m = a+_{v_up}^{b2} a+_{v_dn}^{b3} a_{o_dn}^{b1} a_{o_up}^{b0}.
Applied to the site reference (both occupied orbitals filled) the 16 monomials
give the 16 local states, so local states are labelled by monomials:
|m> := E^m |ref>.  Multi-site states are |m0, m1, ...> := E_0^{m0} E_1^{m1} ... |ref>
(a graded tensor product; odd monomials on different sites anticommute).

The amplitude manifold of PQ is, in this language (Eq. decompose and Table II):
  A1 = the 3 non-identity single-site monomials that conserve charge and S_z,
  A2 = the 29 pairs (a, b) of non-identity monomials on two sites whose charge
       and S_z changes cancel.
So T = sum_P sum_{m in A1} t1[P,m] E_P^m
     + 1/2 sum_{P != Q} sum_{(a,b) in A2} t2[P,Q,(a,b)] E_P^a E_Q^b,
with t2[Q,P,(b,a)] = (-1)^{|a||b|} t2[P,Q,(a,b)] and zero diagonal (the
paper's vanishing-diagonal convention).

The Hamiltonian (two-electron integrals truncated to two labels, full Fock
matrix -- Table I and the Implementation section) is written as one-site
pieces H_P and two-site pieces H_{PQ} whose matrices are linear maps of
integrals gathered per site (20 numbers) and per ordered pair (232 numbers).

Signs are computed here by explicit Jordan-Wigner evaluation (sites in order,
four spin orbitals per site), never by hand.
"""
import itertools
import numpy as np

REF = 0b0011
NS = 16


# ---------------------------------------------------------------- JW helpers
def _apply(state, ops):
    """ops: list of (spin orbital, dagger) applied right to left."""
    sign = 1
    for p, dag in reversed(ops):
        occ = (state >> p) & 1
        if dag == occ:
            return None, 0
        if bin(state & ((1 << p) - 1)).count("1") & 1:
            sign = -sign
        state ^= 1 << p
    return state, sign


def mono_ops(m, site=0):
    o = 4 * site
    ops = []
    if m & 4: ops.append((o + 2, 1))
    if m & 8: ops.append((o + 3, 1))
    if m & 2: ops.append((o + 1, 0))
    if m & 1: ops.append((o + 0, 0))
    return ops


def parity(m):
    return bin(m).count("1") & 1


def qn(m):
    """(charge change, 2*S_z change) of monomial m."""
    dn = bin(m & 12).count("1") - bin(m & 3).count("1")
    ds = ((m >> 2) & 1) - ((m >> 3) & 1) - ((m & 1) - ((m >> 1) & 1))
    return dn, ds


class Space:
    """k-site space in the monomial basis, with its map to JW determinants."""

    def __init__(self, k):
        self.k = k
        self.ref = sum(REF << (4 * j) for j in range(k))
        self.tuples = list(itertools.product(range(NS), repeat=k))
        self.jw = {}
        self.inv = {}
        for tup in self.tuples:
            ops = []
            for j, m in enumerate(tup):
                ops += mono_ops(m, j)
            st, sg = _apply(self.ref, ops)
            assert st is not None
            self.jw[tup] = (st, sg)
            self.inv[st] = (tup, sg)

    def index(self, tup):
        idx = 0
        for m in tup:
            idx = idx * NS + m
        return idx

    def op_matrix_terms(self, terms):
        """terms: list of (key, coef, ops).  Returns dict (row, col) -> {key: coef}
        for the operator sum coef*ops in the monomial basis."""
        out = {}
        for tup in self.tuples:
            st, sg = self.jw[tup]
            for key, coef, ops in terms:
                st2, sg2 = _apply(st, ops)
                if st2 is None or st2 not in self.inv:
                    continue
                tup2, sg3 = self.inv[st2]
                r, c = self.index(tup2), self.index(tup)
                d = out.setdefault((r, c), {})
                d[key] = d.get(key, 0.0) + coef * sg * sg2 * sg3
        return out

    def apply_monomials(self, tup_ops, tup):
        """Apply the product prod_j E_{site_j}^{m_j} (left to right as given in
        tup_ops = [(site, m), ...]) to the basis state tup: (tup', sign) or None."""
        st, sg = self.jw[tup]
        ops = []
        for site, m in tup_ops:
            ops += mono_ops(m, site)
        st2, sg2 = _apply(st, ops)
        if st2 is None:
            return None
        tup2, sg3 = self.inv[st2]
        return tup2, sg * sg2 * sg3


# ---------------------------------------------------------------- tables
def local_product_table():
    """prod_sign[a, m] = s with E^a E^m = s E^{a|m} (0 if a & m != 0)."""
    S1 = Space(1)
    tab = np.zeros((NS, NS), dtype=np.int64)
    for a in range(NS):
        for m in range(NS):
            r = S1.apply_monomials([(0, a)], (m,))
            if r is None:
                continue
            (m2,), s = r
            assert m2 == a | m and (a & m) == 0
            tab[a, m] = s
    return tab


def amplitude_channels():
    A1 = [m for m in range(1, NS) if qn(m) == (0, 0)]
    A2 = [(a, b) for a in range(1, NS) for b in range(1, NS)
          if qn(a)[0] + qn(b)[0] == 0 and qn(a)[1] + qn(b)[1] == 0]
    return A1, A2


def amplitude_channels3():
    """Three-pair (PH) amplitude channels: triples of nonzero per-site
    monomials with zero total charge and S_z (Eq. decompose with K = 3,
    Table II); 303 of them per unordered triple of pairing labels."""
    return [(a, b, c) for a in range(1, NS) for b in range(1, NS) for c in range(1, NS)
            if qn(a)[0] + qn(b)[0] + qn(c)[0] == 0 and qn(a)[1] + qn(b)[1] + qn(c)[1] == 0]


def triple_integral_keys():
    """Three-label integrals of PH (K_H = 3, Table I: rank-3 subtensors of v):
    (pq|rs) over the 6 spatial orbitals 0 = X_o, 1 = X_v, 2 = W_o, 3 = W_v,
    4 = V_o, 5 = V_v whose orbitals touch all three sites; 6^4 - 3 4^4 + 3 2^4
    = 576 of them per ordered triple.  (No one-body element touches three.)"""
    keys = [("v", p, q, r, s) for p in range(6) for q in range(6) for r in range(6)
            for s in range(6) if len({p // 2, q // 2, r // 2, s // 2}) == 3]
    assert len(keys) == 576
    return keys


def quad_integral_keys():
    """Four-label integrals, kept only when the two-electron part is not
    truncated (the paper's integral truncation controlled separately from the
    amplitudes, Implementation section): (pq|rs) over the 8 spatial orbitals
    2 X + x of four sites whose orbitals touch all four; 8 * 6 * 4 * 2 = 384
    of them per ordered quadruple."""
    keys = [("v", p, q, r, s) for p in range(8) for q in range(8) for r in range(8)
            for s in range(8) if len({p // 2, q // 2, r // 2, s // 2}) == 4]
    assert len(keys) == 384
    return keys


def _spin_orbital(site, x, sigma):
    return 4 * site + 2 * x + sigma


def site_integral_keys():
    """20 per-site integrals: 4 one-body h'[x,x'] then 16 (x x'|x'' x''')."""
    keys = [("h", x, y) for x in range(2) for y in range(2)]
    keys += [("v", p, q, r, s) for p in range(2) for q in range(2)
             for r in range(2) for s in range(2)]
    return keys


def pair_integral_keys():
    """232 per-ordered-pair integrals over the 4 spatial orbitals
    0 = X_o, 1 = X_v, 2 = W_o, 3 = W_v: 8 cross one-body h'[p,q] and the 224
    (pq|rs) whose orbitals touch both sites."""
    keys = [("h", p, q) for p in range(4) for q in range(4) if (p // 2) != (q // 2)]
    keys += [("v", p, q, r, s) for p in range(4) for q in range(4) for r in range(4)
             for s in range(4) if len({p // 2, q // 2, r // 2, s // 2}) == 2]
    assert len(keys) == 232
    return keys


def _hamiltonian_terms(keys):
    """Second-quantised terms of sum h[p,q] a+_{p s} a_{q s}
    + 1/2 sum (pq|rs) a+_{p s} a+_{r t} a_{s t} a_{q s} for the given keys;
    spatial orbital p lives on site p // 2 with local spatial index p % 2."""
    terms = []
    for j, key in enumerate(keys):
        if key[0] == "h":
            _, p, q = key
            for s in range(2):
                terms.append((j, 1.0, [(_spin_orbital(p // 2, p % 2, s), 1),
                                       (_spin_orbital(q // 2, q % 2, s), 0)]))
        else:
            _, p, q, r, s_ = key
            for s1 in range(2):
                for s2 in range(2):
                    terms.append((j, 0.5, [(_spin_orbital(p // 2, p % 2, s1), 1),
                                           (_spin_orbital(r // 2, r % 2, s2), 1),
                                           (_spin_orbital(s_ // 2, s_ % 2, s2), 0),
                                           (_spin_orbital(q // 2, q % 2, s1), 0)]))
    return terms


def hamiltonian_structure(k):
    """Sparse linear map integrals -> matrix of the k-site piece (k = 1, 2) in
    the monomial basis: arrays (row, col, key_index, coef)."""
    keys = site_integral_keys() if k == 1 else pair_integral_keys()
    S = Space(k)
    mat = S.op_matrix_terms(_hamiltonian_terms(keys))
    rows, cols, js, cs = [], [], [], []
    for (r, c), d in sorted(mat.items()):
        for j, coef in sorted(d.items()):
            if abs(coef) > 1e-14:
                rows.append(r); cols.append(c); js.append(j); cs.append(coef)
    return (np.array(rows), np.array(cols), np.array(js), np.array(cs), keys)


def pair_op_table(A2):
    """For each (a,b) in A2 the action of E_X^a E_Y^b on 2-site basis states:
    arrays (k, src, dst, sign) with src/dst = 16*mX + mY."""
    S2 = Space(2)
    out = []
    for k, (a, b) in enumerate(A2):
        for tup in S2.tuples:
            r = S2.apply_monomials([(0, a), (1, b)], tup)
            if r is not None:
                out.append((k, S2.index(tup), S2.index(r[0]), r[1]))
    return np.array(out, dtype=np.int64)


def site_op_tables(A1):
    """Action of E^m (m in A1) on site 0 and on site 1 of the 2-site space,
    and on the 1-site space: arrays (k, src, dst, sign)."""
    S1, S2 = Space(1), Space(2)
    one, s0, s1 = [], [], []
    for k, m in enumerate(A1):
        for tup in S1.tuples:
            r = S1.apply_monomials([(0, m)], tup)
            if r is not None:
                one.append((k, tup[0], r[0][0], r[1]))
        for tup in S2.tuples:
            r = S2.apply_monomials([(0, m)], tup)
            if r is not None:
                s0.append((k, S2.index(tup), S2.index(r[0]), r[1]))
            r = S2.apply_monomials([(1, m)], tup)
            if r is not None:
                s1.append((k, S2.index(tup), S2.index(r[0]), r[1]))
    return (np.array(one, dtype=np.int64), np.array(s0, dtype=np.int64),
            np.array(s1, dtype=np.int64))


def graded_sign_checks(prod):
    """Check the graded rules used by the contraction formulas against JW:
    E_X^a E_Y^b E_X^c = (-1)^{|b||c|} E_X^a E_X^c E_Y^b on 2 sites."""
    S2 = Space(2)
    ref = (0, 0)
    for a in range(NS):
        for b in range(NS):
            for c in range(NS):
                lhs = S2.apply_monomials([(0, a), (1, b), (0, c)], ref)
                if (a & c) != 0:
                    assert lhs is None
                    continue
                sgn = (-1) ** (parity(b) * parity(c)) * prod[a, c]
                assert lhs == ((a | c, b), sgn), (a, b, c, lhs, sgn)
    return True


class Tables:
    """All generated tables, as numpy arrays."""

    def __init__(self):
        self.prod = local_product_table()
        graded_sign_checks(self.prod)
        self.A1, self.A2 = amplitude_channels()
        assert len(self.A1) == 3 and len(self.A2) == 29
        self.par = np.array([parity(m) for m in range(NS)], dtype=np.int64)
        self.qn = np.array([qn(m) for m in range(NS)], dtype=np.int64)
        self.h1 = hamiltonian_structure(1)
        self.h2 = hamiltonian_structure(2)
        self.pair_ops = pair_op_table(self.A2)
        self.site_ops1, self.site_ops2a, self.site_ops2b = site_op_tables(self.A1)
        # index of each A2 channel by (a, b); 30 "cluster states" = ref + A2
        self.a2_index = {ab: k for k, ab in enumerate(self.A2)}
        self.a1_index = {m: k for k, m in enumerate(self.A1)}
        self.sector36 = sector36(self.A1, self.A2)


# ---------------------------------------------------------------- sector / channel lists
def spin_flip_channels(T):
    """The spin flip (alpha <-> beta on every orbital of a site: bits 0 <-> 1
    and 2 <-> 3 of a monomial) on the amplitude channels.  The flip unitary
    maps E^m to sigma(m) E^flip(m), sigma(m) = (-1)^(b0 b1 + b2 b3) (the two
    creators and the two annihilators of a site swap places), site order
    unchanged; so a closed-shell T (invariant under the flip) has
    t[flip(k)] = sigma(k) t[k].  Returns (flip1, sign1) over A1 and (flip2,
    sign2) over A2, index arrays into the same channel list."""
    def fl(m):
        return ((m & 1) << 1) | ((m >> 1) & 1) | ((m & 4) << 1) | ((m >> 1) & 4)

    def sg(m):
        return -1 if (((m & 3) == 3) + ((m & 12) == 12)) % 2 else 1

    flip1 = np.array([T.a1_index[fl(m)] for m in T.A1])
    sign1 = np.array([sg(m) for m in T.A1])
    flip2 = np.array([T.a2_index[(fl(a), fl(b))] for a, b in T.A2])
    sign2 = np.array([sg(a) * sg(b) for a, b in T.A2])
    return flip1, sign1, flip2, sign2


def sector36(A1, A2):
    """The 36 two-site states with zero total charge and S_z change, in the
    order: ref, A2 (29), (A1, ref) (3), (ref, A1) (3).  Index c; the link
    coefficients of exp(T_XY)|ref> live on c = 0..29."""
    st = [(0, 0)] + list(A2) + [(m, 0) for m in A1] + [(0, m) for m in A1]
    assert len(st) == 36
    return st


def _p(m):
    return bin(m).count("1") & 1


def t9_channels(T):
    """Quartic topology (Hamiltonian piece on X,W; outputs on Y,Z linked by
    exp(T_XY) exp(T_XZ) exp(T_WY) exp(T_WZ)): entries
    (c_xy, c_xz, c_wy, c_wz, g, out, sign) with
    r2[Y,Z][out] += 1/2 sum_{X != W} sign Cl[X,Y][c_xy] Cl[X,Z][c_xz]
                     Cl[W,Y][c_wy] Cl[W,Z][c_wz] G[X,W][g]."""
    st = T.sector36
    idx = {s: i for i, s in enumerate(st)}
    links = st[:30]
    prod = T.prod
    out = []
    for c1, (a1, b1) in enumerate(links):
        for c2, (a2, e1) in enumerate(links):
            if a1 & a2:
                continue
            s12 = prod[a1, a2] * (-1) ** (_p(a2) * _p(b1))
            m = a1 | a2
            for c3, (d1, b2) in enumerate(links):
                if b1 & b2:
                    continue
                for c4, (d2, e2) in enumerate(links):
                    if d1 & d2 or e1 & e2:
                        continue
                    n = d1 | d2
                    if (m, n) not in idx:
                        continue
                    b, c = b1 | b2, e1 | e2
                    if b == 0 or c == 0:
                        continue
                    sg = (s12 * prod[d1, d2] * prod[b1, b2] * prod[e1, e2]
                          * (-1) ** (_p(d1) * (_p(e1) + _p(b1)))
                          * (-1) ** (_p(d2) * (_p(b2) + _p(e1) + _p(b1)))
                          * (-1) ** (_p(b2) * _p(e1)))
                    out.append((c1, c2, c3, c4, idx[(m, n)], T.a2_index[(b, c)], sg))
    return np.array(out, dtype=np.int64)


def t8_channels(T):
    """r1[Y][k] += 1/2 sum_{X != W} sign Cl[X,Y][c_xy] Cl[W,Y][c_wy] G[X,W][g]."""
    st = T.sector36
    idx = {s: i for i, s in enumerate(st)}
    out = []
    for c1, (a, b1) in enumerate(st[:30]):
        for c2, (d, b2) in enumerate(st[:30]):
            if b1 & b2 or (a, d) not in idx:
                continue
            b = b1 | b2
            if b not in T.a1_index:
                continue
            sg = T.prod[b1, b2] * (-1) ** (_p(b1) * _p(d))
            out.append((c1, c2, idx[(a, d)], T.a1_index[b], sg))
    return np.array(out, dtype=np.int64)


def t4_channels(T):
    """r2[Y,Z][out] += sum_X sign Cl[X,Y][c_xy] Cl[X,Z][c_xz] Ht_X[0, m]."""
    st = T.sector36
    out = []
    for c1, (a1, b) in enumerate(st[1:30], start=1):
        for c2, (a2, c) in enumerate(st[1:30], start=1):
            if a1 & a2:
                continue
            m = a1 | a2
            if tuple(T.qn[m]) != (0, 0):
                continue
            sg = T.prod[a1, a2] * (-1) ** (_p(b) * _p(a2))
            out.append((c1, c2, m, T.a2_index[(b, c)], sg))
    return np.array(out, dtype=np.int64)


def t3_channels(T):
    """r1[Y][k] += sum_X Ht_X[0, a] Cl[X,Y][c_xy] with c_xy = (a, A1[k])."""
    st = T.sector36
    idx = {s: i for i, s in enumerate(st)}
    out = []
    for k, m in enumerate(T.A1):
        for a in range(NS):
            if (a, m) in idx and idx[(a, m)] < 30:
                out.append((idx[(a, m)], a, k))
    return np.array(out, dtype=np.int64)


def t2_channels(T):
    """U[nu] += sum_a Cl[X,Y][c_xy] Ht_X[nu_X, a] with c_xy = (a, nu_Y):
    entries (c_xy, nu_X, a, nu)."""
    st = T.sector36
    idx = {s: i for i, s in enumerate(st)}
    out = []
    for nu, (nx, ny) in enumerate(st):
        for a in range(NS):
            if (a, ny) in idx and idx[(a, ny)] < 30:
                out.append((idx[(a, ny)], nx, a, nu))
    return np.array(out, dtype=np.int64)


def t7_channels(T):
    """U[nu] += sum_W sign Cl[X,Y][c_xy] Cl[W,Y][c_wy] Ht_XW[(nu_X,0),(a,d)]:
    entries (c_xy, c_wy, row, col, nu, sign), row/col 2-site indices 16*mX+mW."""
    st = T.sector36
    idx = {s: i for i, s in enumerate(st)}
    out = []
    for nu, (nx, ny) in enumerate(st):
        for c1, (a, b1) in enumerate(st[:30]):
            for c2, (d, b2) in enumerate(st[:30]):
                if b1 & b2 or (b1 | b2) != ny:
                    continue
                # charge/S_z of column must match the row (nu_X, 0)
                if tuple(T.qn[a] + T.qn[d]) != tuple(T.qn[nx]):
                    continue
                sg = T.prod[b1, b2] * (-1) ** (_p(b1) * _p(d))
                out.append((c1, c2, 16 * nx, 16 * a + d, nu, sg))
    return np.array(out, dtype=np.int64)


def sector_pair_ops(T):
    """Pair excitation operators restricted to the 36-state sector:
    (k, src, dst, sign) with src/dst sector indices."""
    st = T.sector36
    idx = {16 * a + b: i for i, (a, b) in enumerate(st)}
    out = []
    for k, s, d, g in T.pair_ops:
        if s in idx and d in idx:
            out.append((k, idx[s], idx[d], g))
    return np.array(out, dtype=np.int64)


# ---------------------------------------------------------------- 2-site block layout
class BlockLayout:
    """Dense charge/S_z sector blocks of the 256-state 2-site space: element
    (r, c) with both states in sector q is stored at base[q] + pos[r]*dim[q] + pos[c]."""

    def __init__(self, T):
        secs = {}
        for s in range(256):
            m, n = divmod(s, 16)
            q = tuple(T.qn[m] + T.qn[n])
            secs.setdefault(q, []).append(s)
        self.sectors = [secs[q] for q in sorted(secs)]
        self.sec_of = np.zeros(256, dtype=np.int64)
        self.pos = np.zeros(256, dtype=np.int64)
        self.base = []
        off = 0
        for i, ss in enumerate(self.sectors):
            self.base.append(off)
            for p, s in enumerate(ss):
                self.sec_of[s] = i; self.pos[s] = p
            off += len(ss) ** 2
        self.size = off
        self.dim = [len(ss) for ss in self.sectors]

    def elem(self, r, c):
        q = self.sec_of[r]
        if self.sec_of[c] != q:
            return -1
        return self.base[q] + self.pos[r] * self.dim[q] + self.pos[c]


def _pack(t, s, g):
    return (int(t) << 17) | (int(s) << 1) | (1 if g < 0 else 0)


def pair_transform_lists(T, L):
    """Work lists for M <- M exp(I) (right) and M <- exp(-I) M (left) on the
    block layout, I = T_X (ops 0-2) + T_W (3-5) + T_XW (6-34).  Entries pack
    (target element, source element, sign bit)."""
    ops = []
    for k in range(3):
        ops.append(T.site_ops2a[T.site_ops2a[:, 0] == k])
    for k in range(3):
        ops.append(T.site_ops2b[T.site_ops2b[:, 0] == k])
    for k in range(29):
        ops.append(T.pair_ops[T.pair_ops[:, 0] == k])
    right, left, rptr, lptr = [], [], [0], [0]
    for tab in ops:
        for _, src, dst, sg in tab:
            # right: O|src> = sg|dst>  =>  M[r, src] += t sg M[r, dst]
            q = L.sec_of[src]
            for r in L.sectors[q]:
                right.append(_pack(L.elem(r, src), L.elem(r, dst), sg))
            # left: M[dst, c] -= t sg M[src, c]
            for c in L.sectors[q]:
                left.append(_pack(L.elem(dst, c), L.elem(src, c), sg))
        rptr.append(len(right)); lptr.append(len(left))
    return (np.array(right, dtype=np.int64), np.array(rptr, dtype=np.int64),
            np.array(left, dtype=np.int64), np.array(lptr, dtype=np.int64))


def pair_sector_lists(T, L, group=4):
    """The pair closure's sweeps per sector: every row r of sector q goes
    through the same sequence M[r, a] += t_o sg M[r, b] (right, exp(I)) and
    every column c through M[b', c] -= t_o sg M[a', c] (left, exp(-I)), with
    the positions a, b inside the sector.  Entries of one operator touch
    distinct targets that are never sources (each O_o is nilpotent), so the
    lists are cut into groups of `group` entries of one operator.  A group is
    padded with entries whose target is the group's first source and whose
    factor is zero (slot 70), which leave M unchanged.  Offsets are in the
    padded shared layout (row stride dim + 1): right entries step along a
    row, left entries along a column (offset = position * (dim + 1)).
    Entry: target offset | source offset << 12 | factor slot << 24, factor
    slot 2 o + (sign < 0)."""
    ops = []
    for k in range(3):
        ops.append(T.site_ops2a[T.site_ops2a[:, 0] == k])
    for k in range(3):
        ops.append(T.site_ops2b[T.site_ops2b[:, 0] == k])
    for k in range(29):
        ops.append(T.pair_ops[T.pair_ops[:, 0] == k])
    nq = len(L.sectors)
    rl, ll = [[] for _ in range(nq)], [[] for _ in range(nq)]
    enc = lambda tg, sc, f: tg | (sc << 12) | (f << 24)
    for o, tab in enumerate(ops):
        cur_r, cur_l = [[] for _ in range(nq)], [[] for _ in range(nq)]
        for _, src, dst, sg in tab:
            q = int(L.sec_of[src])
            assert int(L.sec_of[dst]) == q
            a, b, f = int(L.pos[src]), int(L.pos[dst]), 2 * o + (1 if sg < 0 else 0)
            dp = L.dim[q] + 1
            cur_r[q].append((a, b, f))             # M[r, a] += t sg M[r, b]
            cur_l[q].append((b * dp, a * dp, f))   # M[b, c] -= t sg M[a, c]
        for q in range(nq):
            for cur, lst in ((cur_r[q], rl[q]), (cur_l[q], ll[q])):
                for i in range(0, len(cur), group):
                    chunk = cur[i:i + group]
                    first_src = chunk[0][1]
                    chunk = chunk + [(first_src, first_src, 70)] * (group - len(chunk))
                    lst.extend(enc(*e) for e in chunk)
    def flat(lists):
        ptr = [0]
        for x in lists:
            ptr.append(ptr[-1] + len(x))
        return np.array([e for x in lists for e in x], dtype=np.int64), np.array(ptr, dtype=np.int64)
    r, rp = flat(rl)
    l, lp = flat(ll)
    return r, rp, l, lp


def site_transform_lists(T):
    right, left, rptr, lptr = [], [], [0], [0]
    for k in range(3):
        tab = T.site_ops1[T.site_ops1[:, 0] == k]
        for _, src, dst, sg in tab:
            for r in range(NS):
                right.append(_pack(16 * r + src, 16 * r + dst, sg))
            for c in range(NS):
                left.append(_pack(16 * dst + c, 16 * src + c, sg))
        rptr.append(len(right)); lptr.append(len(left))
    return (np.array(right, dtype=np.int64), np.array(rptr, dtype=np.int64),
            np.array(left, dtype=np.int64), np.array(lptr, dtype=np.int64))


def r1_t8_code(t8, t8p):
    """C++ source of the T8 sum of r1 as straight-line code: for output k the
    entries (c1, c2, g, k, s) of the channel table in table order, each
    acc[k] += (s/2) cx[c1] cw[c2] g[g NN], where cx, cw are the rows
    Cl[X,Y][.], Cl[W,Y][.] and g points at G[X,W][0] in the transposed
    (channel-major) G; the factor order is that of the table-driven form."""
    out = ["template <typename R>",
           "__device__ __forceinline__ void ppq_r1_t8(const R* __restrict__ cx, const R* __restrict__ cw, "
           "const R* __restrict__ g, size_t NN, R* __restrict__ acc) {"]
    for k in range(3):
        for e in range(t8p[k], t8p[k + 1]):
            c1, c2, gi, kk, sg = (int(x) for x in t8[e])
            assert kk == k and sg in (-1, 1)
            h = "R(0.5)" if sg > 0 else "R(-0.5)"
            out.append(f"  acc[{k}] += {h} * cx[{c1}] * cw[{c2}] * g[{gi} * NN];")
    out.append("}")
    return "\n".join(out)


def r2_t4_code(t4, t4p):
    """C++ source of the T4 sum of r2 as straight-line code, for one X: the
    outputs split in two halves (ppq_r2_t4_0: outputs 0-14, ppq_r2_t4_1:
    15-28), each entry (c1, c2, m, o, s) of the table in table order as
    acc[o - o0] += s cy[c1] cz[c2] hx[j], with cy, cz the rows Cl[X,Y][.],
    Cl[X,Z][.] and hx[j] = Ht_X[0, m] for m = 5, 10, 15 (j = 0, 1, 2)."""
    hm = {5: 0, 10: 1, 15: 2}
    out = []
    for half, (o0, o1) in enumerate(((0, 15), (15, 29))):
        out += ["template <typename R>",
                f"__device__ __forceinline__ void ppq_r2_t4_{half}(const R* __restrict__ cy, const R* __restrict__ cz, "
                "const R* __restrict__ hx, R* __restrict__ acc) {"]
        for o in range(o0, o1):
            for e in range(t4p[o], t4p[o + 1]):
                c1, c2, m, oo, sg = (int(x) for x in t4[e])
                assert oo == o and sg in (-1, 1) and m in hm
                out.append(f"  acc[{o - o0}] += R({sg}) * cy[{c1}] * cz[{c2}] * hx[{hm[m]}];")
        out.append("}")
    return "\n".join(out)


def link_code(sop):
    """C++ source of the link coefficients exp(T_XY)|ref> on the 36-state
    sector as straight-line code over a register array: the factors
    (1 + t_k O_k) in order k = 0..28, each operator entry (k, s, d, sign) of
    the table in table order as v[d] += t_k sign v[s] (ppq_link_apply); and
    exp(-T_XY) the same way with v[d] -= t_k sign v[s] (ppq_link_unapply:
    O_k^2 = 0, so 1 - t_k O_k is the inverse factor)."""
    out = []
    for name, op in (("ppq_link_apply", "+="), ("ppq_link_unapply", "-=")):
        out += ["template <typename R>",
                f"__device__ __forceinline__ void {name}(const double* __restrict__ t, R* __restrict__ v) {{"]
        for k in range(29):
            rows = sop[sop[:, 0] == k]
            if not len(rows):
                continue
            out.append(f"  {{ const R tk = R(t[{k}]);")
            for _, src, dst, g in rows:
                sg = "R(-1)" if g < 0 else "R(1)"
                out.append(f"    v[{int(dst)}] {op} tk * {sg} * v[{int(src)}];")
            out.append("  }")
        out.append("}")
    return "\n".join(out)


def pair_sweep_code(T, L):
    """C++ source of the pair closure's per-sector sweeps with one thread's row
    (right, exp(I)) or column (left, exp(-I)) held in registers: for every
    sector q a straight-line sequence over the sector's positions, operator
    by operator in the order of pair_sector_lists (without its padding),
    each entry one multiply-add.  Factors fac[2 o + (sign < 0)] are read into
    locals once per sector.  Right entry: v[a] += fac[f] v[b]; left entry:
    v[b] -= fac[f] v[a] (positions inside the sector)."""
    ops = []
    for k in range(3):
        ops.append(T.site_ops2a[T.site_ops2a[:, 0] == k])
    for k in range(3):
        ops.append(T.site_ops2b[T.site_ops2b[:, 0] == k])
    for k in range(29):
        ops.append(T.pair_ops[T.pair_ops[:, 0] == k])
    nq = len(L.sectors)
    ent = [[] for _ in range(nq)]
    for o, tab in enumerate(ops):
        for _, src, dst, sg in tab:
            q = int(L.sec_of[src])
            ent[q].append((int(L.pos[src]), int(L.pos[dst]), 2 * o + (1 if sg < 0 else 0)))
    out = []
    for side in ("right", "left"):
        out.append("template <typename R>")
        out.append(f"__device__ __forceinline__ void ppq_sweep_{side}(int q, R* __restrict__ M, int base, "
                   "const R* __restrict__ fac) {")
        out.append("  switch (q) {")
        for q in range(nq):
            if not ent[q]:
                continue
            d = L.dim[q]
            step = 1 if side == "right" else d + 1
            fs = sorted({f for _, _, f in ent[q]})
            out.append(f"    case {q}: {{")
            out.append(f"      R v[{d}];")
            out.append(f"#pragma unroll")
            out.append(f"      for (int i = 0; i < {d}; ++i) v[i] = M[base + i * {step}];")
            out.append("      " + " ".join(f"const R f{f} = fac[{f}];" for f in fs))
            for a, b, f in ent[q]:
                if side == "right":
                    out.append(f"      v[{a}] += f{f} * v[{b}];")
                else:
                    out.append(f"      v[{b}] -= f{f} * v[{a}];")
            out.append(f"#pragma unroll")
            out.append(f"      for (int i = 0; i < {d}; ++i) M[base + i * {step}] = v[i];")
            out.append("    } break;")
        out.append("    default: break;")
        out.append("  }")
        out.append("}")
        out.append("")
    return "\n".join(out), ent


def csr_from_structure(struct, elem_of):
    r, c, j, coef, _ = struct
    ent = {}
    for ri, ci, ji, co in zip(r, c, j, coef):
        e = elem_of(int(ri), int(ci))
        assert e >= 0
        ent.setdefault(e, []).append((int(ji), float(co)))
    els = sorted(ent)
    ptr, js, cs = [0], [], []
    for e in els:
        for ji, co in ent[e]:
            js.append(ji); cs.append(co)
        ptr.append(len(js))
    return (np.array(els, dtype=np.int64), np.array(ptr, dtype=np.int64),
            np.array(js, dtype=np.int64), np.array(cs))


def _c_array(name, ctype, arr, per_line=16):
    arr = np.asarray(arr).ravel()
    body = []
    for i in range(0, len(arr), per_line):
        if ctype in ("float", "double"):
            body.append(", ".join(repr(float(x)) + ("f" if ctype == "float" else "") for x in arr[i:i + per_line]))
        else:
            body.append(", ".join(str(int(x)) for x in arr[i:i + per_line]))
    return f"static __device__ const {ctype} {name}[{max(len(arr), 1)}] = {{\n  " + ",\n  ".join(body or ["0"]) + "\n};\n"


def emit_header(path):
    """Write the generated tables as a CUDA header."""
    T = Tables()
    L = BlockLayout(T)
    st = T.sector36
    sidx = {s: i for i, s in enumerate(st)}
    out = ["/* Generated by paper_1609_00077_gb300/tables.py -- do not edit. */",
           "#pragma once", "#include <stdint.h>", ""]
    defs = dict(PPQ_NA1=3, PPQ_NA2=29, PPQ_NG1=20, PPQ_NG2=232, PPQ_NS36=36,
                PPQ_BLK=L.size, PPQ_NLINK=30)
    for k, v in defs.items():
        out.append(f"#define {k} {v}")
    out.append("")
    out.append(_c_array("ppq_A1", "int8_t", T.A1))
    out.append(_c_array("ppq_A2", "int8_t", np.array(T.A2)))
    out.append(_c_array("ppq_S36", "int8_t", np.array(st)))
    out.append(_c_array("ppq_par", "int8_t", T.par))
    # monomial hole / particle counts (for denominators)
    nh = [bin(m & 3).count("1") for m in range(16)]
    npart = [bin(m & 12).count("1") for m in range(16)]
    out.append(_c_array("ppq_nhole", "int8_t", nh))
    out.append(_c_array("ppq_npart", "int8_t", npart))
    # 1-site Hamiltonian CSR (dense 16x16 element index) and transforms
    e1, p1, j1, c1 = csr_from_structure(T.h1, lambda r, c: 16 * r + c)
    out += [f"#define PPQ_H1_NEL {len(e1)}", _c_array("ppq_h1_el", "int16_t", e1),
            _c_array("ppq_h1_ptr", "int16_t", p1), _c_array("ppq_h1_j", "uint8_t", j1),
            _c_array("ppq_h1_c", "float", c1)]
    sr, srp, sl, slp = site_transform_lists(T)
    out += [_c_array("ppq_s_right", "int32_t", sr), _c_array("ppq_s_rptr", "int16_t", srp),
            _c_array("ppq_s_left", "int32_t", sl), _c_array("ppq_s_lptr", "int16_t", slp)]
    # 2-site Hamiltonian CSR on the block layout and transforms
    e2, p2, j2, c2 = csr_from_structure(T.h2, L.elem)
    out += [f"#define PPQ_H2_NEL {len(e2)}", _c_array("ppq_h2_el", "int16_t", e2),
            _c_array("ppq_h2_ptr", "int32_t", p2), _c_array("ppq_h2_j", "uint8_t", j2),
            _c_array("ppq_h2_c", "float", c2)]
    pr, prp, pl, plp = pair_transform_lists(T, L)
    out += [f"#define PPQ_PR_N {len(pr)}", f"#define PPQ_PL_N {len(pl)}",
            _c_array("ppq_p_right", "int32_t", pr), _c_array("ppq_p_rptr", "int32_t", prp),
            _c_array("ppq_p_left", "int32_t", pl), _c_array("ppq_p_lptr", "int32_t", plp)]
    # compact forms for the persistent pair-closure kernel: per-sector sweep
    # lists (groups of 4), state -> (sector, position), sector base and size,
    # and the Hamiltonian CSR with (j, 2c) packed in 16 bits
    sr, srp, sl, slp = pair_sector_lists(T, L)
    assert np.all(np.abs(2 * c2 - np.round(2 * c2)) == 0) and np.abs(2 * c2).max() <= 127
    jc = np.asarray(j2)
    PPQ_NG2_VALUE = defs["PPQ_NG2"]
    assert int(max(j2)) < PPQ_NG2_VALUE
    out += [f"#define PPQ_H2_NNZ {len(jc)}", f"#define PPQ_NSEC {len(L.sectors)}", f"#define PPQ_PSR_N {len(sr)}", f"#define PPQ_PSL_N {len(sl)}",
            _c_array("ppq_ps_right", "int32_t", sr), _c_array("ppq_ps_rptr", "int16_t", srp),
            _c_array("ppq_ps_left", "int32_t", sl), _c_array("ppq_ps_lptr", "int16_t", slp),
            _c_array("ppq_st_sec", "int8_t", L.sec_of), _c_array("ppq_st_pos", "int8_t", L.pos),
            _c_array("ppq_sec_dim", "int8_t", np.array(L.dim))]
    out.append(pair_sweep_code(T, L)[0])
    # thread -> two-site state, grouped by sector (largest first) so that the
    # lanes of a warp walk the same list
    order = sorted(range(256), key=lambda st: (-L.dim[L.sec_of[st]], L.sec_of[st], L.pos[st]))
    # gather terms as code * NG2 + j, code indexing the coefficients below
    codes = [-1.0, -0.5, 0.5, 1.0, 2.0]
    cidx = np.array([codes.index(float(x)) for x in c2], dtype=np.int64)
    out += [_c_array("ppq_th_state", "int16_t", np.array(order)),
            _c_array("ppq_h2_cj", "uint16_t", cidx * PPQ_NG2_VALUE + np.asarray(j2).astype(np.int64)),
            "#define PPQ_H2_NCODE 5", _c_array("ppq_h2_code", "float", np.array(codes))]
    # padded sector layout of the persistent kernel's shared-memory copy: rows
    # of sector q are dim_q + 1 apart (odd or coprime strides, no bank
    # conflicts when one thread walks each row)
    pbase, off = [], 0
    for dq in L.dim:
        pbase.append(off)
        off += dq * (dq + 1)
    def padded(e):
        q = int(np.searchsorted(np.array(L.base), e, side="right") - 1)
        r, c = divmod(int(e) - L.base[q], L.dim[q])
        return pbase[q] + r * (L.dim[q] + 1) + c
    out += [f"#define PPQ_BLKP {off}", _c_array("ppq_sec_pbase", "int16_t", np.array(pbase)),
            _c_array("ppq_h2_elp", "int16_t", np.array([padded(e) for e in e2]))]
    # the gather as one term stream per thread (256 threads): elements dealt
    # out longest first to the least-loaded thread, a thread's terms stored at
    # [j][thread] (coalesced), padded with zero terms to the longest stream.
    # Word: gsv index (11 bits) | padded element offset << 11 (13 bits) |
    # last term of its element << 31; the zero term reads gsv index 1160.
    cnt = np.diff(p2)
    load = [0] * 256
    own = [[] for _ in range(256)]
    for el in sorted(range(len(e2)), key=lambda x: (-int(cnt[x]), x)):
        t = int(np.argmin(load))
        own[t].append(el)
        load[t] += int(cnt[el])
    slen = max(load)
    zero_term = len(codes) * PPQ_NG2_VALUE
    assert zero_term < 2048 and off < 8192
    stream = np.full((slen, 256), zero_term, dtype=np.int64)
    cj_all = cidx * PPQ_NG2_VALUE + np.asarray(j2).astype(np.int64)
    for t in range(256):
        j = 0
        for el in sorted(own[t]):
            for k in range(p2[el], p2[el + 1]):
                w = int(cj_all[k]) | (padded(e2[el]) << 11)
                if k == p2[el + 1] - 1:
                    w |= 1 << 31
                stream[j, t] = w
                j += 1
    out += [f"#define PPQ_H2_SLEN {slen}",
            _c_array("ppq_h2_stream", "uint32_t", stream.ravel())]
    padded_of = padded
    # outputs of the pair closure: G row, T7 entries, column-0 entries, element (0,0)
    g_el = [L.elem(0, 16 * a + b) for a, b in st]
    t7 = t7_channels(T)
    t7rc = sorted(set((int(r), int(c)) for r, c in t7[:, [2, 3]]))
    t7e = {rc: i for i, rc in enumerate(t7rc)}
    t7_el = [L.elem(r, c) for r, c in t7rc]
    col0 = [L.elem(16 * a + b, 0) for a, b in T.A2] + [L.elem(16 * m, 0) for m in T.A1]
    out += [f"#define PPQ_NT7E {len(t7rc)}", f"#define PPQ_NCOL0 {len(col0)}",
            f"#define PPQ_EL00 {L.elem(0, 0)}",
            _c_array("ppq_g_el", "int16_t", g_el), _c_array("ppq_t7_el", "int16_t", t7_el),
            _c_array("ppq_col0_el", "int16_t", col0)]
    out += [f"#define PPQ_EL00P {padded_of(L.elem(0, 0))}",
            _c_array("ppq_g_elp", "int16_t", np.array([padded_of(e) for e in g_el])),
            _c_array("ppq_t7_elp", "int16_t", np.array([padded_of(e) for e in t7_el])),
            _c_array("ppq_col0_elp", "int16_t", np.array([padded_of(e) for e in col0]))]
    # link / transform operators on the 36-state sector
    sop = sector_pair_ops(T)
    sptr = [0]
    for k in range(29):
        sptr.append(int(np.sum(sop[:, 0] <= k)))
    out += [f"#define PPQ_NSOP {len(sop)}",
            _c_array("ppq_sop", "int32_t", [_pack(d, s, g) for _, s, d, g in sop]),
            _c_array("ppq_sop_ptr", "int16_t", sptr)]
    out.append(link_code(sop))
    # topology channel lists
    def by_out(arr, col, nout):
        arr = np.asarray(arr)
        order = np.argsort(arr[:, col], kind="stable")
        arr = arr[order]
        ptr = [int(np.sum(arr[:, col] < o)) for o in range(nout + 1)]
        return arr, ptr
    t2, t2p = by_out(t2_channels(T), 3, 36)
    t3, t3p = by_out(t3_channels(T), 2, 3)
    t4, t4p = by_out(t4_channels(T), 3, 29)
    t8, t8p = by_out(t8_channels(T), 3, 3)
    out += [f"#define PPQ_NT2 {len(t2)}", _c_array("ppq_t2", "int16_t", t2), _c_array("ppq_t2p", "int16_t", t2p),
            f"#define PPQ_NT3 {len(t3)}", _c_array("ppq_t3", "int16_t", t3), _c_array("ppq_t3p", "int16_t", t3p),
            f"#define PPQ_NT4 {len(t4)}", _c_array("ppq_t4", "int16_t", t4), _c_array("ppq_t4p", "int16_t", t4p),
            f"#define PPQ_NT8 {len(t8)}", _c_array("ppq_t8", "int16_t", t8), _c_array("ppq_t8p", "int16_t", t8p)]
    out.append(r1_t8_code(t8, t8p))
    out.append(r2_t4_code(t4, t4p))
    t7c, t7p = by_out(np.array([(c1, c2, t7e[(int(r), int(c))], nu, s) for c1, c2, r, c, nu, s in t7]), 3, 36)
    out += [f"#define PPQ_NT7 {len(t7c)}", _c_array("ppq_t7", "int16_t", t7c), _c_array("ppq_t7p", "int16_t", t7p)]
    # GEMM form of T7: M7[k][Y][Z] = sum_W pt7[Y,W][e] Cl[W,Z][c2] for each
    # distinct (c2, e); channels in the order of ppq_t7 as (c1, k, nu, s)
    k7 = sorted(set((int(r[1]), int(r[2])) for r in t7c))
    k7i = {x: i for i, x in enumerate(k7)}
    t7g = np.array([(int(r[0]), k7i[(int(r[1]), int(r[2]))], int(r[3]), int(r[4])) for r in t7c])
    out += [f"#define PPQ_NK7 {len(k7)}", _c_array("ppq_k7", "int16_t", np.array(k7)),
            _c_array("ppq_t7g", "int16_t", t7g)]
    swap = [T.a2_index[(b, a)] for a, b in T.A2]
    swsg = [(-1) ** (_p(a) * _p(b)) for a, b in T.A2]
    out += [_c_array("ppq_a2_swap", "int8_t", swap), _c_array("ppq_a2_swsg", "int8_t", swsg)]
    t9 = t9_channels(T)
    p9 = sorted(set((int(a), int(b)) for a, b in t9[:, [0, 1]]))
    p9i = {p: i for i, p in enumerate(p9)}
    q9 = sorted(set((p9i[(int(a), int(b))], int(g)) for a, b, g in t9[:, [0, 1, 4]]))
    q9i = {q: i for i, q in enumerate(q9)}
    ch9 = [(q9i[(p9i[(int(r[0]), int(r[1]))], int(r[4]))], int(r[2]), int(r[3]), int(r[5]), int(r[6]))
           for r in t9]
    # GEMM form of the quartic topology: for each c2 the list of (c1, g, q)
    c2list = sorted(((int(p9[p][1]), int(p9[p][0]), int(g), qi) for qi, (p, g) in enumerate(q9)))
    g2ptr = [0]
    for c2 in range(30):
        g2ptr.append(sum(1 for e in c2list if e[0] <= c2))
    out += [_c_array("ppq_q9c", "int16_t", np.array([(c1, g, qi) for _, c1, g, qi in c2list])),
            _c_array("ppq_q9cptr", "int16_t", g2ptr),
            _c_array("ppq_q9cptr_h", "int16_t", g2ptr).replace("static __device__ const", "static const")]
    ch9arr = np.array(ch9)
    # channels grouped by q for the fused GEMM epilogue: (c3, c4, out, s)
    # (ordered by q, then by output o; a run of equal (q, o) is one output group,
    # which lets one thread own each (group, row) and sum in a fixed order)
    c9q = ch9arr[np.lexsort((ch9arr[:, 3], ch9arr[:, 0]))]
    c9qp = [int(np.sum(c9q[:, 0] < q)) for q in range(len(q9) + 1)]
    gstart = [i for i in range(len(c9q)) if i == 0 or tuple(c9q[i, [0, 3]]) != tuple(c9q[i - 1, [0, 3]])]
    c9g = gstart + [len(c9q)]
    gq = c9q[gstart, 0]
    c9gp = [int(np.sum(gq < q)) for q in range(len(q9) + 1)]
    # epilogue group of each channel for the one-q-per-chunk FP64 kernel: the
    # outputs of a q go whole to one of four thread groups (so that no two
    # groups add into the same output), largest output first onto the least
    # loaded group (ties to the lower group)
    c9grp = np.zeros(len(c9q), dtype=np.int64)
    for q in range(len(q9)):
        lo, hi = c9qp[q], c9qp[q + 1]
        outs, cnt = np.unique(c9q[lo:hi, 3], return_counts=True)
        load = [0, 0, 0, 0]
        for k in sorted(range(len(outs)), key=lambda k: (-cnt[k], outs[k])):
            gsel = min(range(4), key=lambda j: (load[j], j))
            load[gsel] += int(cnt[k])
            c9grp[lo:hi][c9q[lo:hi, 3] == outs[k]] = gsel
    out.append(_c_array("ppq_c9grp", "int8_t", c9grp))
    out += [_c_array("ppq_c9q", "int16_t", c9q[:, 1:]), _c_array("ppq_c9qp", "int16_t", c9qp),
            _c_array("ppq_c9g", "int16_t", np.array(c9g)), _c_array("ppq_c9gp", "int16_t", np.array(c9gp))]
    ch9, c9p = by_out(ch9arr, 3, 29)
    out.append(_c_array("ppq_c9p", "int16_t", c9p))
    out += [f"#define PPQ_NP9 {len(p9)}", f"#define PPQ_NQ9 {len(q9)}", f"#define PPQ_NC9 {len(ch9)}",
            _c_array("ppq_p9", "int8_t", np.array(p9)), _c_array("ppq_q9", "int16_t", np.array(q9)),
            _c_array("ppq_c9", "int16_t", np.array(ch9))]
    # host copies for planning the tensor-core work list
    host = lambda a: a.replace("static __device__ const", "static const")
    out += [host(_c_array("ppq_p9_h", "int8_t", np.array(p9))), host(_c_array("ppq_q9_h", "int16_t", np.array(q9))),
            host(_c_array("ppq_c9qp_h", "int16_t", c9qp))]
    # integral gather keys
    k1 = site_integral_keys(); k2 = pair_integral_keys()
    enc1 = [(0, k[1], k[2], 0, 0) if k[0] == "h" else (1,) + k[1:] for k in k1]
    enc2 = [(0, k[1], k[2], 0, 0) if k[0] == "h" else (1,) + k[1:] for k in k2]
    out += [_c_array("ppq_g1key", "int8_t", np.array(enc1)), _c_array("ppq_g2key", "int8_t", np.array(enc2))]
    # amplitude layout descriptor for the C-ABI: kind, first monomial, second
    desc = [(1, m, 0) for m in T.A1] + [(2, a, b) for a, b in T.A2]
    out.append(_c_array("ppq_layout_desc", "int8_t", np.array(desc)).replace("static __device__ const", "static const"))
    # the three-pair (PH) layout: one more column, then the 303 triple channels
    A3 = amplitude_channels3()
    desc3 = ([(1, m, 0, 0) for m in T.A1] + [(2, a, b, 0) for a, b in T.A2]
             + [(3, a, b, c) for a, b, c in A3])
    out.append(f"#define PPQ_NA3 {len(A3)}")
    out.append(host(_c_array("ppq_layout_desc3", "int8_t", np.array(desc3))))
    text = "\n".join(out) + "\n"
    with open(path, "w") as fh:
        fh.write(text)
    return dict(blk=L.size, right=len(pr), left=len(pl), h2=len(j2), t7e=len(t7rc))


if __name__ == "__main__":
    import sys
    print(emit_header(sys.argv[1]))
