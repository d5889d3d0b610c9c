"""Pins of the CPU oracle against facts fixed by the paper and by mathematics,
independent of the oracle's own formulas.

* PQ is exact for 4 electrons in 4 orbitals and PH for 6 in 6 (Abstract;
  Theory section; Table VI caption): the converged energies equal brute-force
  FCI, and PQ equals PH at 4e/4o.
* A complete manifold (K >= number of pairs) with untruncated integrals is FCI.
* Size consistency (inherited from CC, Theory section): a direct sum of two
  non-interacting fragments has the sum of the fragment energies, and two
  H chains 100 A apart (one RHF, fragment-local pairs) nearly so.
* Invariance to swapping pairs (Theory section) and to MO sign changes;
  non-invariance of PQ to occupied-occupied rotations and to the choice of
  which virtual is paired with which occupied orbital (Theory section), while
  FCI is invariant (negative control); at 4e/4o every pairing is exact.
* Residual at random amplitudes against an independent Jordan-Wigner matrix
  construction of exp(-T) H exp(T) (scipy expm), and O-loc against O-det.
* Manifold sizes against the closed form derived from Eq. decompose.
"""
import json
import os
from math import comb

import numpy as np
import pytest
from scipy.linalg import expm

from workloads import build_ppp, build_hchain, Hamiltonian
from oracle.detcc import Problem, enumerate_manifold, truncated_hamiltonian
from oracle.loccc import LocalAssembly
from oracle.fci import fci_energy

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def solve_total(H, K, K_H=0, **kw):
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=K, K_H=K_H, e_const=H.e_const)
    r = P.solve(r_tol=1e-11, e_tol=1e-13, max_iter=400, **kw)
    assert r['converged']
    return r['e_corr'] + P.e_ref, P, r


def test_pq_exact_at_4e4o_butadiene():
    H = build_ppp('polyene', 4)
    e, _, _ = solve_total(H, K=2)
    assert abs(e - fci_energy(H.h, H.eri, 2, H.e_const)) < 1e-9


def test_pq_exact_at_4e4o_h4_and_equals_ph():
    H = build_hchain(4, 1.5)
    e2, _, _ = solve_total(H, K=2)
    e3, _, _ = solve_total(H, K=3)
    ef = fci_energy(H.h, H.eri, 2, H.e_const)
    assert abs(e2 - ef) < 1e-9 and abs(e3 - ef) < 1e-9


@pytest.mark.slow
def test_ph_exact_at_6e6o_hexatriene():
    H = build_ppp('polyene', 6)
    e, _, _ = solve_total(H, K=3)
    assert abs(e - fci_energy(H.h, H.eri, 3, H.e_const)) < 1e-9
    e2, _, _ = solve_total(H, K=2)
    assert e2 - e > 1e-4   # PQ is not exact at 6e/6o: the truncation is real


def test_complete_manifold_untruncated_is_fci_h6():
    H = build_hchain(6, 1.2)
    e, _, _ = solve_total(H, K=3, K_H=-1)
    assert abs(e - fci_energy(H.h, H.eri, 3, H.e_const)) < 1e-9


def _direct_sum(A, B, interleave=True):
    """Block-diagonal union of two Hamiltonians; pairs interleaved A0 B0 A1 B1."""
    na, nb = A.n_orb, B.n_orb
    n = na + nb
    h = np.zeros((n, n)); eri = np.zeros((n, n, n, n))
    h[:na, :na] = A.h; h[na:, na:] = B.h
    eri[:na, :na, :na, :na] = A.eri; eri[na:, na:, na:, na:] = B.eri
    occ, vir = [], []
    pa = list(zip(A.occ_of_pair, A.vir_of_pair))
    pb = [(i + na, a + na) for i, a in zip(B.occ_of_pair, B.vir_of_pair)]
    order = []
    for k in range(max(len(pa), len(pb))):
        if k < len(pa): order.append(pa[k])
        if k < len(pb): order.append(pb[k])
    if not interleave:
        order = pa + pb
    occ = np.array([o for o, _ in order], dtype=np.int32)
    vir = np.array([v for _, v in order], dtype=np.int32)
    return Hamiltonian("A+B", h, eri, A.e_const + B.e_const, occ, vir,
                       np.concatenate([A.mo_energy, B.mo_energy]))


def test_fragment_additivity_pq_equals_sum_of_fci():
    A = build_ppp('polyene', 4)
    B = build_hchain(4, 1.6)
    AB = _direct_sum(A, B)
    e_ab, _, _ = solve_total(AB, K=2)
    fa = fci_energy(A.h, A.eri, 2, A.e_const)
    fb = fci_energy(B.h, B.eri, 2, B.e_const)
    assert abs(e_ab - (fa + fb)) < 1e-9


def test_fragment_additivity_pq_nontrivial_fragments():
    A = build_hchain(6, 1.3)
    B = build_ppp('polyene', 4)
    ea, _, _ = solve_total(A, K=2)
    eb, _, _ = solve_total(B, K=2)
    AB = _direct_sum(A, B)
    P = LocalAssembly(AB.h, AB.eri, AB.occ_of_pair, AB.vir_of_pair, K=2)
    from oracle.detcc import jacobi_diis, DetCC
    d = DetCC(AB.n_orb, AB.occ_of_pair, AB.vir_of_pair, 2, manifold=P.manifold).denominators(P.f)
    r = jacobi_diis(P.residual, d, len(P.manifold), r_tol=1e-11, e_tol=1e-13, max_iter=400)
    assert r['converged']
    assert abs(r['e_corr'] + P.e_ref + AB.e_const - (ea + eb)) < 1e-9


def test_far_separated_chains_size_consistency():
    """Physical, not block-diagonal: H4 (1.5 A spacing) and H2 (0.74 A) on one
    line 100 A apart, one RHF for all six atoms (every cross integral kept),
    pairs formed inside each fragment.  The neutral fragments interact through
    multipoles (quadrupole-quadrupole, R^-5) and dispersion (R^-6), about 1e-12
    Eh here, so E_PQ(A+B) = E_PQ(A) + E_PQ(B) to 5e-11."""
    from workloads.hchain import ao_integrals_at, chain_positions, BOHR_PER_ANGSTROM
    from workloads.scf import rhf, mo_integrals
    zA = chain_positions(4, 1.5)
    zB = chain_positions(2, 0.74) + zA[-1] + 100.0 * BOHR_PER_ANGSTROM
    S, h, eri, e_nuc = ao_integrals_at(np.concatenate([zA, zB]))
    n = len(zA) + len(zB)

    def jk(P):
        J = (eri.reshape(n * n, n * n) @ P.ravel()).reshape(n, n)
        K = (eri.transpose(0, 2, 1, 3).reshape(n * n, n * n) @ P.ravel()).reshape(n, n)
        return J, K
    e, C, _ = rhf(S, h, n // 2, jk)
    on_a = (C[:len(zA)] ** 2).sum(0) / (C ** 2).sum(0)
    assert np.all(np.minimum(on_a, 1.0 - on_a) < 1e-10)      # every MO on one fragment
    occ, vir = [], []
    for frag in (on_a > 0.5, on_a < 0.5):
        occ += sorted((k for k in range(n // 2) if frag[k]), key=lambda k: -e[k])
        vir += sorted((k for k in range(n // 2, n) if frag[k]), key=lambda k: e[k])
    h_mo, eri_mo = mo_integrals(C, h, eri_ao=eri)
    AB = Hamiltonian("H4 + H2", h_mo, eri_mo, e_nuc, np.array(occ), np.array(vir), e)
    e_ab, _, _ = solve_total(AB, K=2)
    e_a, _, _ = solve_total(build_hchain(4, 1.5), K=2)
    e_b, _, _ = solve_total(build_hchain(2, 0.74), K=2)
    assert abs(e_ab - (e_a + e_b)) < 5e-11


def _permute_pairs(H, perm):
    return Hamiltonian(H.name, H.h, H.eri, H.e_const, H.occ_of_pair[perm],
                       H.vir_of_pair[perm], H.mo_energy)


def test_pair_swap_invariance():
    H = build_hchain(8, 1.4)
    e0, _, _ = solve_total(H, K=2)
    e1, _, _ = solve_total(_permute_pairs(H, np.array([2, 0, 3, 1])), K=2)
    assert abs(e0 - e1) < 1e-10


def _rotate(H, U):
    h = U.T @ H.h @ U
    eri = np.einsum('pqrs,pi,qj,rk,sl->ijkl', H.eri, U, U, U, U, optimize=True)
    return Hamiltonian(H.name, h, eri, H.e_const, H.occ_of_pair, H.vir_of_pair, H.mo_energy)


def test_orbital_sign_invariance():
    H = build_ppp('polyene', 8)
    e0, _, _ = solve_total(H, K=2)
    U = np.diag([1, -1, 1, 1, -1, 1, -1, 1.0])
    e1, _, _ = solve_total(_rotate(H, U), K=2)
    assert abs(e0 - e1) < 1e-10


def test_occupied_rotation_changes_pq_not_fci():
    H = build_ppp('polyene', 6)
    c, s = np.cos(0.3), np.sin(0.3)
    U = np.eye(6); U[0, 0] = U[1, 1] = c; U[0, 1] = s; U[1, 0] = -s
    Hr = _rotate(H, U)
    e0, _, _ = solve_total(H, K=2)
    e1, _, _ = solve_total(Hr, K=2)
    assert abs(e0 - e1) > 1e-5
    assert abs(fci_energy(H.h, H.eri, 3) - fci_energy(Hr.h, Hr.eri, 3)) < 1e-10


def _repair(H, perm):
    vir = np.asarray(H.vir_of_pair)[perm]
    return Hamiltonian(H.name, H.h, H.eri, H.e_const, H.occ_of_pair, vir, H.mo_energy)


def test_pairing_choice_changes_pq_but_not_exactness():
    # 6e/6o: the energy depends on the occupied-virtual pairing
    H = build_ppp('polyene', 6)
    e0, _, _ = solve_total(H, K=2)
    e1, _, _ = solve_total(_repair(H, np.array([2, 0, 1])), K=2)
    assert abs(e0 - e1) > 1e-5
    # 4e/4o: PQ is exact for any pairing
    B = build_ppp('polyene', 4)
    efci = fci_energy(B.h, B.eri, 2) + B.e_const
    for perm in ([0, 1], [1, 0]):
        e, _, _ = solve_total(_repair(B, np.array(perm)), K=2)
        assert abs(e - efci) < 1e-9


def test_manifold_counts_closed_form_and_tables():
    with open(os.path.join(GOLDEN, "counts_tables_I_II.json")) as fh:
        g = json.load(fh)
    for N in range(1, 7):
        occ, vir = np.arange(N), np.arange(N, 2 * N)
        assert len(enumerate_manifold(occ, vir, 1)) == 3 * N
        assert len(enumerate_manifold(occ, vir, 2)) == 3 * N + 29 * comb(N, 2)
        if N <= 4:
            assert len(enumerate_manifold(occ, vir, 3)) == 3 * N + 29 * comb(N, 2) + 303 * comb(N, 3)
    # 4e/4o and 6e/6o: the truncated manifold is the full M_s = 0 space minus Phi
    assert len(enumerate_manifold(np.arange(2), np.arange(2, 4), 2)) == comb(4, 2) ** 2 - 1
    assert len(enumerate_manifold(np.arange(3), np.arange(3, 6), 3)) == comb(6, 3) ** 2 - 1
    # Eq. decompose: opposite-spin doubles of PQ fall in 8 label patterns
    occ, vir = np.arange(4), np.arange(4, 8)
    lab = {**{i: i for i in range(4)}, **{4 + i: i for i in range(4)}}
    pats = set()
    for ah, ap, bh, bp in enumerate_manifold(occ, vir, 2):
        if len(ah) == 1 and len(bh) == 1:
            i, j, a, b = lab[ah[0]], lab[bh[0]], lab[ap[0]], lab[bp[0]]
            names = {}
            pats.add(tuple(names.setdefault(x, len(names)) for x in (i, j, a, b)))
    assert len(pats) == g["eq_decompose_PQ_doubles_label_patterns"]


# ---------------------------------------------------------------------------
# residual at random amplitudes against a Jordan-Wigner construction


def _jw_ops(nso):
    I = np.eye(2); Z = np.diag([1.0, -1.0]); a = np.array([[0, 1.0], [0, 0]])
    ops = []
    for k in range(nso):
        m = np.array([[1.0]])
        for j in range(nso):
            m = np.kron(m, Z if j < k else (a if j == k else I))
        ops.append(m)
    return ops


def test_residual_random_t_against_jordan_wigner_expm():
    """N = 2 (8 spin orbitals): build H, every tau_D and exp(+-T) as dense
    2^8 matrices with numpy kron and scipy expm, independent of the string
    code, and compare the linked residual and energy at random amplitudes."""
    H = build_hchain(4, 1.7)
    n, N = 4, 2
    for K, K_H in ((1, 2), (2, 2), (2, -1)):
        P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=K, K_H=K_H)
        rng = np.random.default_rng(1234)
        t = rng.uniform(-0.1, 0.1, P.cc.n_amp)
        R, e = P.residual(t)
        a = _jw_ops(2 * n)          # spin orbital (p, spin) -> p + n*spin
        ad = [x.T for x in a]
        Hm = np.zeros((256, 256))
        for p in range(n):
            for q in range(n):
                for s in range(2):
                    Hm += P.hp[p, q] * ad[p + n * s] @ a[q + n * s]
        for p in range(n):
            for q in range(n):
                for r in range(n):
                    for u in range(n):
                        if P.vt[p, q, r, u] == 0.0:
                            continue
                        for s1 in range(2):
                            for s2 in range(2):
                                Hm += 0.5 * P.vt[p, q, r, u] * (
                                    ad[p + n * s1] @ ad[r + n * s2] @ a[u + n * s2] @ a[q + n * s1])
        vac = np.zeros(256); vac[0] = 1.0
        ref = vac.copy()
        # |Phi> = a+ (alpha occ ascending) a+ (beta occ ascending) |vac>
        occ_sorted = sorted(int(i) for i in H.occ_of_pair)
        creators = [ad[i] for i in occ_sorted] + [ad[i + n] for i in occ_sorted]
        for c in reversed(creators):
            ref = c @ ref
        T = np.zeros((256, 256))
        taus = []
        for (ah, ap, bh, bp) in P.cc.manifold:
            op = np.eye(256)
            seq = ([ad[x] for x in ap] + [a[x] for x in reversed(ah)]
                   + [ad[x + n] for x in bp] + [a[x + n] for x in reversed(bh)])
            for m in seq:
                op = op @ m
            # normalise so that tau|Phi> is the determinant with a+ ordered
            # alpha-ascending then beta-ascending, as in the string basis
            det = vac.copy()
            occ_a = sorted(set(occ_sorted) - set(ah) | set(ap))
            occ_b = sorted(set(occ_sorted) - set(bh) | set(bp))
            for c in reversed([ad[x] for x in occ_a] + [ad[x + n] for x in occ_b]):
                det = c @ det
            sgn = float(det @ (op @ ref))
            assert abs(abs(sgn) - 1.0) < 1e-12
            taus.append((sgn * op, det))
        for tk, (op, _) in zip(t, taus):
            T += tk * op
        Hbar = expm(-T) @ Hm @ expm(T)
        R_jw = np.array([det @ Hbar @ ref for _, det in taus])
        e_jw = ref @ Hbar @ ref - ref @ Hm @ ref
        assert np.abs(R - R_jw).max() < 1e-12
        assert abs(e - e_jw) < 1e-12


@pytest.mark.parametrize("kind,size,K", [("hchain", 10, 2), ("polyene", 10, 2), ("hchain", 12, 2)])
def test_local_assembly_equals_detcc(kind, size, K):
    H = build_hchain(size, 1.6) if kind == "hchain" else build_ppp('polyene', size)
    if size > 10 and os.environ.get("PPQ_LONG_CHECKS") != "1":
        pytest.skip("853 776 determinants for O-det; set PPQ_LONG_CHECKS=1")
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=K)
    L = LocalAssembly(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=K)
    rng = np.random.default_rng(1234)
    t = rng.uniform(-0.1, 0.1, P.cc.n_amp)
    R1, e1 = P.residual(t)
    R2, e2 = L.residual(t)
    assert np.abs(R1 - R2).max() < 1e-12
    assert abs(e1 - e2) < 1e-12


def test_local_assembly_truncated_integrals_h10():
    """K_H = 2 < K + ... with a non-trivial Moebius sum (N = 5 > K + K_H)."""
    H = build_hchain(10, 2.2)
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=2, K_H=2)
    L = LocalAssembly(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=2, K_H=2)
    t = np.random.default_rng(7).uniform(-0.05, 0.05, P.cc.n_amp)
    R1, e1 = P.residual(t)
    R2, e2 = L.residual(t)
    assert np.abs(R1 - R2).max() < 1e-12 and abs(e1 - e2) < 1e-12


def test_fci_lanczos_branch():
    # The Lanczos branch of fci_energy (spaces above 800 determinants) against
    # the dense eigensolver on the same sigma products (the lowest 7 orbitals of
    # octatetraene, 3 + 3 electrons: 1225 determinants), and against the
    # additivity of FCI over
    # two non-interacting fragments: butadiene + H4 has 4900 determinants
    # (Lanczos) while each fragment has 36 (dense).
    from oracle.fci import Strings, sigma
    H = build_ppp('polyene', 8)
    h7, eri7 = H.h[:7, :7].copy(), H.eri[:7, :7, :7, :7].copy()
    S = Strings(7, 3)
    dim = S.n * S.n
    assert dim == 1225
    Hm = np.empty((dim, dim))
    for j in range(dim):
        c = np.zeros(dim); c[j] = 1.0
        Hm[:, j] = sigma(S, h7, eri7, c.reshape(S.n, S.n)).ravel()
    e_dense = float(np.linalg.eigvalsh(0.5 * (Hm + Hm.T))[0])
    assert abs(fci_energy(h7, eri7, 3) - e_dense) < 1e-10
    A, B = build_ppp('polyene', 4), build_hchain(4, 1.6)
    AB = _direct_sum(A, B)
    e_ab = fci_energy(AB.h, AB.eri, 4, AB.e_const)
    assert abs(e_ab - (fci_energy(A.h, A.eri, 2, A.e_const) + fci_energy(B.h, B.eri, 2, B.e_const))) < 1e-9


@pytest.mark.parametrize("sites,K", [(6, 2), (6, 3), (8, 2)])
def test_residual_is_spin_flip_symmetric_for_closed_shell_hamiltonians(sites, K):
    """A spin-free Hamiltonian in RHF orbitals commutes with the spin flip
    (alpha <-> beta on every orbital), which maps the reference to itself up
    to a global sign and each excitation (a_holes, a_parts, b_holes,
    b_parts) to (b_holes, b_parts, a_holes, a_parts) with no sign (both
    spin strings hold an even number of operators).  So amplitudes equal on
    spin-flip partners give residuals equal on them, for every residual
    element and for K = 2 and 3; a spin-asymmetric perturbation breaks it."""
    H = build_ppp('polyene', sites)
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=K)
    man = P.cc.manifold
    idx = {m: i for i, m in enumerate(man)}
    flip = np.array([idx[(bh, bp, ah, ap)] for ah, ap, bh, bp in man])
    assert (flip != np.arange(len(man))).sum() > len(man) // 2 and (flip[flip] == np.arange(len(man))).all()
    rng = np.random.default_rng(sites + 10 * K)
    t = rng.uniform(-0.1, 0.1, len(man))
    t = 0.5 * (t + t[flip])
    R, e = P.residual(t)
    assert np.abs(R).max() > 1e-2
    assert np.abs(R - R[flip]).max() < 1e-13
    j = int(np.nonzero(flip != np.arange(len(man)))[0][0])
    t2 = t.copy()
    t2[j] += 0.05
    R2, _ = P.residual(t2)
    assert np.abs(R2 - R2[flip]).max() > 1e-6
