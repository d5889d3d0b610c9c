"""Channel tables of the disjoint PH class (test infrastructure; the first
per-class tables of the three-pair path, checked against the site
formulation).

For outputs on labels M and a Hamiltonian piece on labels S with no label in
common, the contribution is sum_{s'} G_S[s'] sigma(mu, s') Lambda(mu, s'),
with the closure row G_S, the interleaving sign sigma and the link
coefficients Lambda(mu, s') = <mu s'| exp(L) |ref> of the clusters L that
join S to M (``SiteInterp.disjoint_term``).  Expanding exp(L) turns Lambda
into a finite sum over *configurations*: sets of (cluster position set,
channel) whose monomials are disjoint on every site and together make mu on M
and s' on S, each with the product of its amplitudes and a sign.  The
configurations depend only on the pattern in which the labels of M and S
interleave, so they are generated once per pattern; G_S[s'] vanishes beyond
two holes on S (two-body Hamiltonian), which bounds a configuration to at most
four clusters.
"""
import itertools

import numpy as np

from tests.ph_site_interp import PAR, PROD


def _holes(m):
    return bin(m & 3).count("1")


def _apply_ordered(ops, k):
    """Product of monomial operators [(position, monomial)] (leftmost applied
    last) on the reference of k sites: (state tuple, sign) or None."""
    st = [0] * k
    sign = 1
    for j, a in reversed(ops):
        if st[j] & a:
            return None
        before = 0
        for i in range(j):
            before ^= PAR[st[i]]
        if PAR[a] and before:
            sign = -sign
        sign *= PROD[a, st[j]]
        st[j] |= a
    return tuple(st), sign


def link_configurations(pattern, A1, A2, A3, max_holes_S=2):
    """pattern: string of 'M' / 'S' for the sites of U in label order.
    Returns {(state tuple): [(((slot), channel index), ...), sign]} over every
    configuration of link clusters whose S-part has at most max_holes_S
    holes; slot = tuple of U positions (sorted), channel index into A1/A2/A3
    by the slot's size."""
    k = len(pattern)
    Mpos = [i for i, c in enumerate(pattern) if c == "M"]
    Spos = [i for i, c in enumerate(pattern) if c == "S"]
    chans = {1: [(m,) for m in A1], 2: list(A2), 3: list(A3)}
    slots = [C for r in (2, 3) for C in itertools.combinations(range(k), r)
             if set(C) & set(Mpos) and set(C) & set(Spos)]
    # every (slot, channel) as a list of (position, monomial)
    items = [(C, c, list(zip(C, mons))) for C in slots for c, mons in enumerate(chans[len(C)])]
    out = {}

    def rec(start, used, chosen):
        # record the current configuration (the empty one is the reference)
        if chosen:
            ops = [op for it in chosen for op in it[2]]
            r = _apply_ordered(ops, k)
            assert r is not None
            st, sg = r
            out.setdefault(st, []).append((tuple((it[0], it[1]) for it in chosen), sg))
        for n in range(start, len(items)):
            C, c, ops = items[n]
            new = list(used)
            ok = True
            for j, a in ops:
                if new[j] & a:
                    ok = False
                    break
                new[j] |= a
            if not ok or sum(_holes(new[j]) for j in Spos) > max_holes_S:
                continue
            rec(n + 1, new, chosen + [items[n]])

    rec(0, [0] * k, [])
    return out


def disjoint_term_from_tables(si, M, S, amp, mats, tables_cache):
    """The disjoint contribution evaluated from the configuration tables."""
    import tests.ph_site_interp as psi
    U = tuple(sorted(set(M) | set(S)))
    pattern = "".join("M" if X in M else "S" for X in U)
    if pattern not in tables_cache:
        tables_cache[pattern] = link_configurations(pattern, si.A1, si.A2, si.A3)
    conf = tables_cache[pattern]
    kS = len(S)
    I_S = si._ops(amp, tuple(S), lambda L: True, mats)
    H_S = si.piece(kS, tuple(range(kS)), S)
    row = psi._expv(I_S.T.tocsr(), H_S.T @ si._ref(kS))
    SecS = si.sector(kS)
    chans = {1: [(m,) for m in si.A1], 2: si.A2, 3: si.A3}[len(M)]
    Mpos = [i for i, X in enumerate(U) if X in M]
    Spos = [i for i, X in enumerate(U) if X in S]
    out = np.zeros(len(chans))
    for c, mu in enumerate(chans):
        odd = [sum(PAR[mu[i]] for i, Y in enumerate(M) if Y < X) & 1 for X in S]
        acc = 0.0
        for n in np.flatnonzero(row):
            sprime = SecS.states[n]
            st = [0] * len(U)
            for i, p in enumerate(Mpos):
                st[p] = mu[i]
            for i, p in enumerate(Spos):
                st[p] = sprime[i]
            sig = -1.0 if sum(PAR[sprime[i]] & odd[i] for i in range(kS)) & 1 else 1.0
            lam = 0.0
            for cfg, sg in conf.get(tuple(st), []):
                prod = float(sg)
                for slot, ch in cfg:
                    prod *= amp[tuple(U[p] for p in slot)][ch]
                lam += prod
            acc += row[n] * sig * lam
        out[c] = acc
    return out


# ---------------------------------------------------------------- per-label factors
def _merge_sign(w, x):
    """E^w E^x = sign E^{w|x} for monomial strings w, x over the same sites
    (canonical order site by site), 0 if they overlap on a site."""
    s = 1
    for j in range(len(w)):
        if w[j] & x[j]:
            return 0
        s *= PROD[w[j], x[j]]
        if PAR[x[j]]:
            for i in range(j + 1, len(w)):
                if PAR[w[i]]:
                    s = -s
    return s


def merge(f, g):
    """Product of two monomial-operator expansions {monomial string: coef}."""
    out = {}
    for w, cw in f.items():
        for x, cx in g.items():
            s = _merge_sign(w, x)
            if s:
                key = tuple(a | b for a, b in zip(w, x))
                out[key] = out.get(key, 0.0) + s * cw * cx
    return out


def link_factors(si, M, S, amp, mats):
    """exp(L) |ref> for the clusters joining S to M, grouped by the labels of
    S they touch: one factor exp(L_a) per label a of S (clusters (a, y) and
    (a, y, y')) and one exp(L_aa') per pair (clusters (a, a', y)), each as a
    monomial-operator expansion over the sites of U = M + S.  The factors
    commute, so exp(L)|ref> is their merged product; a factor depends only on
    its own labels of S and on M, which is what lets a kernel share it across
    every piece S that contains those labels."""
    import tests.ph_site_interp as psi
    U = tuple(sorted(set(M) | set(S)))
    Sec = si.sector(len(U))
    factors = []
    groups = [({a},) for a in S] + [({a, b},) for a, b in itertools.combinations(S, 2)]
    for (part,) in groups:
        Lp = si._ops(amp, U, lambda L, part=part: (L & set(S)) == part and bool(L & set(M)), mats)
        v = psi._expv(Lp, si._ref(len(U)))
        nz = np.flatnonzero(v)
        factors.append({tuple(int(m) for m in Sec.states[i]): v[i] for i in nz})
    return U, factors
