"""Integrals as three-index factors (pq_solve_cd, ph_solve_cd): the solvers
contract the Fock matrix and every gathered integral block from B[Q][p][q]
((pq|rs) = sum_Q B[Q,p,q] B[Q,r,s]) and never form the n^4 array.

Checks against the dense-integral path (the same kernels downstream of the
staging) and the oracle: PPP factors are exact (one Cholesky vector per site),
so energies agree with the dense solve to rounding (1e-10 Eh) and with the
oracle to 1e-9; H-chain factors from a pivoted Cholesky to 1e-12 agree to
1e-9.  The bench workload (C140H142, 140 factors instead of 3.07 GB of
integrals) agrees with the dense mixed solve to 1e-8 Eh.  A non-finite factor
returns status 3 before any solve.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1609_00077_gb300 as ppq
from workloads import build_ppp, build_hchain, ppp_cholesky_vectors, cholesky_vectors, ppp_eri_device
from oracle.detcc import Problem


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _oracle(H, K, K_H=0):
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=K, K_H=K_H, e_const=H.e_const)
    r = P.solve(r_tol=1e-11, e_tol=1e-13, max_iter=300)
    assert r['converged']
    return r['e_corr'] + P.e_ref


@pytest.mark.parametrize("K_H", [0, -1])
def test_pq_cd_ppp_matches_dense_and_oracle(K_H):
    H = build_ppp('polyene', 8)
    B = ppp_cholesky_vectors(H)
    rc, e_cd, t_cd, _ = ppq.pq_solve_cd(H.occ_of_pair, H.vir_of_pair, H.h, B, H.e_const, precision=0, K_H=K_H)
    rc2, e_d, t_d, _ = ppq.pq_solve(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), H.e_const, precision=0,
                                    K_H=K_H)
    assert rc == 0 and rc2 == 0
    assert abs(e_cd - e_d) < 1e-10 and np.abs(t_cd - t_d).max() < 1e-8
    assert abs(e_cd - _oracle(H, 2, K_H)) < 1e-9


def test_pq_cd_hchain_pivoted_cholesky():
    H = build_hchain(8, 1.5)
    B = cholesky_vectors(H.eri, 1e-12)
    rc, e_cd, _, _ = ppq.pq_solve_cd(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(B), H.e_const, precision=1)
    assert rc == 0 and abs(e_cd - _oracle(H, 2)) < 1e-8


def test_ph_cd_matches_dense():
    H = build_ppp('polyene', 8)
    B = ppp_cholesky_vectors(H)
    rc, e_cd, _, _ = ppq.ph_solve_cd(H.occ_of_pair, H.vir_of_pair, H.h, B, H.e_const, precision=0)
    rc2, e_d, _, _ = ppq.ph_solve(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), H.e_const, precision=0)
    assert rc == 0 and rc2 == 0 and abs(e_cd - e_d) < 1e-10


def test_pq_cd_bench_workload_c140h142():
    H = build_ppp('polyene', 140, with_eri=False, orbitals="local")
    B = ppp_cholesky_vectors(H)
    assert B.shape == (140, 140, 140)
    eri = ppp_eri_device(H, torch)
    h = dev(H.h)
    rc, e_d, _, _ = ppq.pq_solve(H.occ_of_pair, H.vir_of_pair, h, eri, H.e_const, precision=1)
    del eri
    torch.cuda.empty_cache()
    rc2, e_cd, _, info = ppq.pq_solve_cd(H.occ_of_pair, H.vir_of_pair, H.h, B, H.e_const, precision=1)
    assert rc == 0 and rc2 == 0 and abs(e_cd - e_d) < 1e-8, (e_cd, e_d)


def test_cd_nonfinite_factor_is_status_3():
    H = build_ppp('polyene', 6)
    B = ppp_cholesky_vectors(H)
    B[1, 2, 3] = np.nan
    rc, _, _, info = ppq.pq_solve_cd(H.occ_of_pair, H.vir_of_pair, H.h, B, H.e_const)
    assert rc == 3 and info["status"] == 3
