"""PQ with untruncated two-electron integrals (K_H = FULL, the integral
truncation the paper controls separately from the amplitudes) on the GPU,
through the C ABI, against the oracle.

Every (pq|rs) is kept, so a linked term carries up to K + 4 = 6 labels; the
label-subset expansion evaluates it from local problems of up to six labels.
Tolerances as tests/test_gpu_ph.py (FP64 1e-11, FP32 2e-5 max|R|; energies
1e-9 Eh FP64, 1e-8 Eh mixed).  Checks: residual elements at random amplitudes
against O-det for N = 2, 3, 4; the stored O-det residual of C14H16 (N = 7,
every subset size enters; tests/golden/pq_full_c14h16.npz, written by the
committed script beside it); PQ = FCI at 4e/4o with the untruncated
Hamiltonian; pq_solve with K_H = -1 equal to the oracle's solve at N = 4, and
different from the two-label model there (control).
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
from oracle.fci import fci_energy
from tests.layout import LayoutMap

HERE = os.path.dirname(os.path.abspath(__file__))
SYSTEMS = {"C4H6": lambda: build_ppp('polyene', 4), "C6H8": lambda: build_ppp('polyene', 6),
           "C8H10": lambda: build_ppp('polyene', 8), "H8": lambda: build_hchain(8, 1.5)}


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_full_residual_matches_oracle(name, precision):
    H = SYSTEMS[name]()
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=2, K_H=-1)
    t = np.random.default_rng(77 + H.n_pairs).uniform(-0.1, 0.1, P.cc.n_amp)
    R, e = P.residual(t)
    lm = LayoutMap(P.cc.manifold, H.occ_of_pair, H.vir_of_pair, H.n_orb, ppq.amp_layout(2))
    r, e2 = ppq.subset_residual(2, -1, H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), dev(lm.to_layout(t)),
                                precision=precision)
    R2 = lm.from_layout(r.cpu().numpy())
    tol = 1e-11 if precision == 0 else 2e-5 * np.abs(R).max()
    assert np.abs(R2 - R).max() < tol
    assert abs(e2 - e) < (1e-11 if precision == 0 else 1e-6)


def test_full_residual_n7_against_stored_oracle():
    path = os.path.join(HERE, "golden", "pq_full_c14h16.npz")
    if not os.path.exists(path):
        pytest.skip("golden file not generated")
    g = np.load(path)
    occ, vir = g["occ"], g["vir"]
    lm = LayoutMap(enumerate_manifold(occ, vir, 2), occ, vir, g["h"].shape[0], ppq.amp_layout(2))
    r, e = ppq.subset_residual(2, -1, occ, vir, dev(g["h"]), dev(g["eri"]), dev(lm.to_layout(g["t"])))
    assert np.abs(lm.from_layout(r.cpu().numpy()) - g["R"]).max() < 1e-11
    assert abs(e - float(g["e_corr"])) < 1e-11


def test_pq_full_is_fci_at_4e4o():
    H = build_ppp('polyene', 4)
    fci = fci_energy(H.h, H.eri, 2, H.e_const)
    rc, e, _, _ = ppq.pq_solve(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), H.e_const, K_H=-1, precision=0)
    assert rc == 0 and abs(e - fci) < 1e-9


def test_pq_full_solve_matches_oracle_n4():
    H = build_ppp('polyene', 8)
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=2, K_H=-1, e_const=H.e_const)
    res = P.solve(r_tol=1e-11, e_tol=1e-13, max_iter=300)
    assert res['converged']
    eo = res['e_corr'] + P.e_ref
    for prec, tol in ((0, 1e-9), (1, 1e-8)):
        rc, e, _, info = ppq.pq_solve(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), H.e_const, K_H=-1,
                                      precision=prec)
        assert rc == 0 and abs(e - eo) < tol, (prec, e, eo)
    rc, e2, _, _ = ppq.pq_solve(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), H.e_const, precision=0)
    assert rc == 0 and abs(e2 - eo) > 1e-5     # the four-label integrals change the energy
