"""Parity of the three-pair (PH) CUDA path, through the C ABI, with the CPU oracle.

Residuals are compared element by element at seeded random amplitudes
(uniform +-0.1).  Tolerances:
  FP64: 1e-11 absolute -- the kernels sum the same exact terms as the oracle
    in another order (local problems combined by inclusion-exclusion, with
    coefficients of at most a few hundred at these sizes), |terms| <= ~1;
  FP32: 2e-5 * max|R| -- FP32 local problems, FP64 assembly.
Energies after convergence: 1e-9 Eh on the FP64 path, 1e-8 Eh mixed.

Cases:
  * N = 2, 3, 4 (butadiene, hexatriene, octatetraene PPP, H8) against O-det,
    integrals truncated to three and to two labels: every local problem is the
    whole system or a subset of it;
  * N = 6 with two-label integrals against O-loc: inclusion-exclusion over
    subsets of up to five labels with nonzero coefficients for every size;
  * N = 7, three-label integrals, the stored oracle elements of one label
    triple (tests/golden/ph_c14h16_triple.npz, written by the committed script
    beside it from O-loc alone): every coefficient nonzero;
  * a direct sum of hexatriene and octatetraene (N = 7, pairs interleaved) at
    random amplitudes inside the fragments: each fragment's elements equal its
    own oracle residual, the mixed elements vanish, the energies add;
  * ph_solve: FCI at 6e/6o (PH is exact there), the oracle's PH energy for
    octatetraene, additivity over the direct sum, mixed against FP64, and the
    excitation-rank mask (ranks <= 2 and <= 4) against the oracle on the
    reduced manifold.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1609_00077_gb300 as ppq
from workloads import build_ppp, build_hchain
from oracle.detcc import Problem, enumerate_manifold
from oracle.loccc import LocalAssembly
from oracle.fci import fci_energy
from tests.layout import LayoutMap
from tests.test_oracle_pins import _direct_sum

HERE = os.path.dirname(os.path.abspath(__file__))
SYSTEMS = {"C4H6": lambda: build_ppp('polyene', 4), "C6H8": lambda: build_ppp('polyene', 6),
           "C8H10": lambda: build_ppp('polyene', 8), "H8": lambda: build_hchain(8, 1.5)}


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _layout3():
    return ppq.amp_layout(3)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,K_H", [("C4H6", 3), ("C6H8", 3), ("C6H8", 2), ("C8H10", 3), ("C8H10", 2),
                                      ("H8", 3), ("H8", 2)])
def test_ph_residual_matches_oracle(name, K_H, precision):
    H = SYSTEMS[name]()
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=3, K_H=K_H)
    t = np.random.default_rng(1234 + 7919 * H.n_pairs + 17 * K_H).uniform(-0.1, 0.1, P.cc.n_amp)
    R, e = P.residual(t)
    lm = LayoutMap(P.cc.manifold, H.occ_of_pair, H.vir_of_pair, H.n_orb, _layout3())
    r, e2 = ppq.ph_residual(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), dev(lm.to_layout(t)),
                            precision=precision, K_H=K_H)
    rv = r.cpu().numpy()
    R2 = lm.from_layout(rv)
    tol = 1e-11 if precision == 0 else 2e-5 * np.abs(R).max()
    assert np.abs(R).max() > 0.05
    assert np.abs(R2 - R).max() < tol
    assert abs(e2 - e) < (1e-11 if precision == 0 else 1e-6)
    assert lm.mirror_error(rv) <= (0.0 if precision == 0 else 1e-12)


def test_ph_residual_n6_two_label_integrals_against_local_assembly():
    H = build_ppp('polyene', 12)
    LA = LocalAssembly(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=3, K_H=2)
    t = np.random.default_rng(5).uniform(-0.1, 0.1, len(LA.manifold))
    R, e = LA.residual(t)
    lm = LayoutMap(LA.manifold, H.occ_of_pair, H.vir_of_pair, H.n_orb, _layout3())
    r, e2 = ppq.ph_residual(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), dev(lm.to_layout(t)), K_H=2)
    assert np.abs(lm.from_layout(r.cpu().numpy()) - R).max() < 1e-11
    assert abs(e2 - e) < 1e-11


def test_ph_residual_n7_triple_against_stored_oracle_elements():
    path = os.path.join(HERE, "golden", "ph_c14h16_triple.npz")
    if not os.path.exists(path):
        pytest.skip("golden file not generated")
    g = np.load(path)
    occ, vir = g["occ"], g["vir"]
    man = enumerate_manifold(occ, vir, 3)
    lm = LayoutMap(man, occ, vir, g["h"].shape[0], _layout3())
    r, _ = ppq.ph_residual(occ, vir, dev(g["h"]), dev(g["eri"]), dev(lm.to_layout(g["t"])), K_H=3)
    R2 = lm.from_layout(r.cpu().numpy())[g["idx"]]
    assert len(g["idx"]) == 303 and np.abs(g["R"]).max() > 0.01
    assert np.abs(R2 - g["R"]).max() < 1e-11


def _label_maps(A, B):
    """Labels of A and B inside the interleaved direct sum (A0 B0 A1 B1 ...)."""
    la, lb, k = [], [], 0
    for i in range(max(A.n_pairs, B.n_pairs)):
        if i < A.n_pairs: la.append(k); k += 1
        if i < B.n_pairs: lb.append(k); k += 1
    return la, lb


def _embed(v, lmap, N, NF):
    """Sorted-label entries of a fragment's K = 3 layout vector placed in the
    direct sum's layout (labels mapped monotonically, so channels and signs
    carry over)."""
    out = np.zeros(3 * N + 29 * N * N + 303 * N ** 3)
    o2, o3 = 3 * N, 3 * N + 29 * N * N
    f2, f3 = 3 * NF, 3 * NF + 29 * NF * NF
    for a in range(NF):
        out[3 * lmap[a]:3 * lmap[a] + 3] = v[3 * a:3 * a + 3]
        for b in range(a + 1, NF):
            out[o2 + (lmap[a] * N + lmap[b]) * 29:][:29] = v[f2 + (a * NF + b) * 29:][:29]
            for c in range(b + 1, NF):
                q, qf = (lmap[a] * N + lmap[b]) * N + lmap[c], (a * NF + b) * NF + c
                out[o3 + q * 303:][:303] = v[f3 + qf * 303:][:303]
    return out


def _unique_mask(N, labels=None):
    m = np.zeros(3 * N + 29 * N * N + 303 * N ** 3, dtype=bool)
    inside = set(range(N)) if labels is None else set(labels)
    for a in range(N):
        if a in inside: m[3 * a:3 * a + 3] = True
        for b in range(a + 1, N):
            if {a, b} <= inside: m[3 * N + (a * N + b) * 29:][:29] = True
            for c in range(b + 1, N):
                if {a, b, c} <= inside:
                    m[3 * N + 29 * N * N + ((a * N + b) * N + c) * 303:][:303] = True
    return m


def test_ph_residual_direct_sum_n7():
    A, B = build_ppp('polyene', 6), build_ppp('polyene', 8)
    AB = _direct_sum(A, B)
    N = AB.n_pairs
    la, lb = _label_maps(A, B)
    parts = []
    for F, lmap, seed in ((A, la, 11), (B, lb, 12)):
        P = Problem(F.h, F.eri, F.occ_of_pair, F.vir_of_pair, K=3, K_H=3)
        t = np.random.default_rng(seed).uniform(-0.1, 0.1, P.cc.n_amp)
        R, e = P.residual(t)
        lm = LayoutMap(P.cc.manifold, F.occ_of_pair, F.vir_of_pair, F.n_orb, _layout3())
        parts.append((lmap, F.n_pairs, lm.to_layout(t), lm.to_layout(R), e))
    t_ab = sum(_embed(v, lmap, N, NF) for lmap, NF, v, _, _ in parts)
    r, e_ab = ppq.ph_residual(AB.occ_of_pair, AB.vir_of_pair, dev(AB.h), dev(AB.eri), dev(t_ab), K_H=3)
    r = r.cpu().numpy()
    expect = sum(_embed(Rv, lmap, N, NF) for lmap, NF, _, Rv, _ in parts)
    uniq = _unique_mask(N)
    inside = _unique_mask(N, la) | _unique_mask(N, lb)
    assert np.abs(expect[inside]).max() > 0.05
    assert np.abs(r[uniq] - expect[uniq]).max() < 1e-11       # fragment elements; mixed ones zero
    assert np.abs(r[uniq & ~inside]).max() < 1e-11
    assert abs(e_ab - (parts[0][4] + parts[1][4])) < 1e-11


def test_ph_residual_is_bit_reproducible():
    H = build_ppp('polyene', 8)
    L = ppq.amp_count(4, 3)
    t = dev(np.random.default_rng(2).uniform(-0.1, 0.1, L))
    r1, e1 = ppq.ph_residual(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), t)
    r2, e2 = ppq.ph_residual(H.occ_of_pair, H.vir_of_pair, H.h, H.eri, t.cpu().numpy())
    assert torch.equal(r1.cpu(), torch.from_numpy(r2)) and e1 == e2


def _oracle_ph_energy(H, K_H=3):
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=3, K_H=K_H, e_const=H.e_const)
    res = P.solve(r_tol=1e-11, e_tol=1e-13, max_iter=300)
    assert res['converged']
    return res['e_corr'] + P.e_ref


def test_ph_solve_is_fci_at_6e6o():
    H = build_ppp('polyene', 6)
    fci = fci_energy(H.h, H.eri, 3, H.e_const)
    rc, e, _, info = ppq.ph_solve(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), H.e_const, precision=0)
    assert rc == 0 and abs(e - fci) < 1e-9, (e, fci)
    rc, em, _, info = ppq.ph_solve(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), H.e_const, precision=1)
    assert rc == 0 and abs(em - fci) < 1e-8 and info["evals_fp32"] > 0


@pytest.mark.parametrize("K_H", [3, 2])
def test_ph_solve_octatetraene_matches_oracle(K_H):
    H = build_ppp('polyene', 8)
    eo = _oracle_ph_energy(H, K_H)
    rc, e, t, info = ppq.ph_solve(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), H.e_const, precision=0,
                                  K_H=K_H)
    assert rc == 0 and abs(e - eo) < 1e-9, (e, eo)
    assert info["res_norm"] <= 1e-10
    rc, em, _, info = ppq.ph_solve(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), H.e_const, precision=1,
                                   K_H=K_H)
    assert rc == 0 and abs(em - eo) < 1e-8


def test_ph_solve_direct_sum_is_additive_n7():
    A, B = build_ppp('polyene', 6), build_ppp('polyene', 8)
    AB = _direct_sum(A, B)
    ea = fci_energy(A.h, A.eri, 3, A.e_const)
    eb = _oracle_ph_energy(B)
    rc, e, _, info = ppq.ph_solve(AB.occ_of_pair, AB.vir_of_pair, dev(AB.h), dev(AB.eri), AB.e_const,
                                  precision=0, max_iter=300)
    assert rc == 0 and abs(e - (ea + eb)) < 1e-9, (e, ea + eb)


@pytest.mark.parametrize("max_rank", [2, 4])
def test_ph_solve_excitation_rank_mask_matches_oracle(max_rank):
    # PH with the excitations above max_rank disabled (Conclusions: PH with
    # singles and doubles is a local CCSD) against the oracle on the same
    # reduced manifold; the dropped amplitudes stay zero
    H = build_ppp('polyene', 8)
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=3, K_H=3, e_const=H.e_const, max_rank=max_rank)
    res = P.solve(r_tol=1e-11, e_tol=1e-13, max_iter=400)
    assert res['converged']
    eo = res['e_corr'] + P.e_ref
    rc, e, t, info = ppq.ph_solve(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), H.e_const, precision=0,
                                  max_rank=max_rank)
    assert rc == 0 and abs(e - eo) < 1e-9, (e, eo)
    lm = LayoutMap(P.cc.manifold, H.occ_of_pair, H.vir_of_pair, H.n_orb, _layout3())
    assert np.abs(lm.from_layout(t) - res['t']).max() < 1e-7
    full = enumerate_manifold(H.occ_of_pair, H.vir_of_pair, 3)
    dropped = [k for k, (ah, ap, bh, bp) in enumerate(full) if len(ah) + len(bh) > max_rank]
    lf = LayoutMap(full, H.occ_of_pair, H.vir_of_pair, H.n_orb, _layout3())
    assert len(dropped) > 0 and np.abs(lf.from_layout(t)[dropped]).max() == 0.0
    rc, em, _, _ = ppq.ph_solve(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), H.e_const, precision=1,
                                max_rank=max_rank)
    assert rc == 0 and abs(em - eo) < 1e-8
