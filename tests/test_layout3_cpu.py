"""The three-pair (K = 3) amplitude layout of the C ABI (ppq_amp_count,
ppq_amp_layout) against the oracle's own K = 3 manifold, and its copy rule
against Jordan-Wigner products (host-only calls; no GPU)."""
from itertools import permutations
from math import comb

import numpy as np
import pytest

import paper_1609_00077_gb300 as ppq
from workloads import build_ppp
from oracle.detcc import enumerate_manifold
from tests.layout import LayoutMap, order_sign
from tests.jw import JW


def _lib_or_skip():
    try:
        ppq.amp_layout(3)
    except ppq.PPQError:
        pytest.skip("libppq.so not built")


@pytest.mark.parametrize("sites", [6, 8])
def test_layout3_covers_the_oracle_manifold(sites):
    _lib_or_skip()
    H = build_ppp('polyene', sites)
    N = H.n_pairs
    man = enumerate_manifold(H.occ_of_pair, H.vir_of_pair, 3)
    desc = ppq.amp_layout(3)
    assert desc.shape == (335, 4) and (desc[:32, :3] == ppq.amp_layout(2)).all()
    lm = LayoutMap(man, H.occ_of_pair, H.vir_of_pair, H.n_orb, desc)
    assert lm.n_amp == ppq.amp_count(N, 3) == 3 * N + 29 * N * N + 303 * N ** 3
    assert len(lm.entries3) == 303 * comb(N, 3)
    assert len(lm.entries) == 3 * N + 29 * comb(N, 2)
    # distinct oracle amplitudes land in distinct slots, all six copies filled
    t = np.random.default_rng(5).uniform(0.5, 1.0, len(man))
    v = lm.to_layout(t)
    assert np.count_nonzero(v) == 3 * N + 2 * 29 * comb(N, 2) + 6 * 303 * comb(N, 3)
    assert np.abs(lm.from_layout(v) - t).max() == 0.0
    assert lm.mirror_error(v) == 0.0


def test_copy_rule_against_jordan_wigner():
    """E_P^a E_Q^b E_R^c |Phi> against the same monomials in the other five
    orders: the sign is -1 per inverted pair of odd monomials."""
    _lib_or_skip()
    H = build_ppp('polyene', 6)
    occ, vir, n = [int(x) for x in H.occ_of_pair], [int(x) for x in H.vir_of_pair], H.n_orb
    jw = JW(n, n // 2, n // 2)
    ref = jw.det(sorted(occ), sorted(occ))

    def mono(P, m):
        ops = []
        if m & 4: ops.append(jw.ad[vir[P]])
        if m & 8: ops.append(jw.ad[n + vir[P]])
        if m & 2: ops.append(jw.a[n + occ[P]])
        if m & 1: ops.append(jw.a[occ[P]])
        return ops

    A3 = [tuple(d[1:]) for d in ppq.amp_layout(3) if d[0] == 3]
    rng = np.random.default_rng(8)
    n_odd = 0
    for k in rng.choice(len(A3), 40, replace=False):
        monos = A3[k]
        base = jw.product(sum((mono(P, monos[P]) for P in range(3)), [])) @ ref
        assert np.abs(base).max() == 1.0
        for perm in permutations(range(3)):
            v = jw.product(sum((mono(perm[i], monos[perm[i]]) for i in range(3)), [])) @ ref
            assert np.array_equal(v, order_sign(monos, perm) * base)
        n_odd += sum(bin(m).count("1") & 1 for m in monos) >= 2
    assert n_odd > 0


def test_layout3_amplitudes_build_the_oracle_state():
    """N = 3: T|Phi> from the oracle's amplitudes (operators tau_D) equals
    T|Phi> from the layout's (E_P^m, E_P^a E_Q^b, E_P^a E_Q^b E_R^c over
    P < Q < R) -- the sign of every slot, including the 303 triple ones."""
    _lib_or_skip()
    H = build_ppp('polyene', 6)
    occ, vir, n = [int(x) for x in H.occ_of_pair], [int(x) for x in H.vir_of_pair], H.n_orb
    man = enumerate_manifold(occ, vir, 3)
    desc = ppq.amp_layout(3)
    lm = LayoutMap(man, occ, vir, n, desc)
    jw = JW(n, n // 2, n // 2)
    ref = jw.det(sorted(occ), sorted(occ))
    t = np.random.default_rng(6).uniform(-1.0, 1.0, len(man))
    want = sum(tk * (jw.excitation(*d, sorted(occ))[0] @ ref) for tk, d in zip(t, man))

    def mono(P, m):
        ops = []
        if m & 4: ops.append(jw.ad[vir[P]])
        if m & 8: ops.append(jw.ad[n + vir[P]])
        if m & 2: ops.append(jw.a[n + occ[P]])
        if m & 1: ops.append(jw.a[occ[P]])
        return ops

    v = lm.to_layout(t)
    N = 3
    t1 = v[:3 * N].reshape(N, 3)
    t2 = v[3 * N:3 * N + 29 * N * N].reshape(N, N, 29)
    t3 = v[3 * N + 29 * N * N:].reshape(N, N, N, 303)
    got = np.zeros_like(ref)
    for P in range(N):
        for k in range(3):
            got += t1[P, k] * (jw.product(mono(P, desc[k, 1])) @ ref)
        for Q in range(P + 1, N):
            for k in range(29):
                a, b = desc[3 + k, 1:3]
                got += t2[P, Q, k] * (jw.product(mono(P, a) + mono(Q, b)) @ ref)
    for k in range(303):
        a, b, c = desc[32 + k, 1:4]
        got += t3[0, 1, 2, k] * (jw.product(mono(0, a) + mono(1, b) + mono(2, c)) @ ref)
    assert np.abs(want).max() > 0.5
    assert np.abs(got - want).max() < 1e-12
