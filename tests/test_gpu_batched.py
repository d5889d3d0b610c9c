"""Batched solve: many Hamiltonians of different pair counts in one call give
the same energies and amplitudes as one-by-one solves (and, for the small
members, as the oracle)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1609_00077_gb300 as ppq
from workloads import build_hchain, build_ppp
from oracle.detcc import Problem


def _systems():
    rng = np.random.default_rng(1609)
    out = []
    for k in range(10):
        n = int(rng.choice([4, 6, 8, 10, 12, 14]))
        d = float(rng.uniform(0.9, 1.3))
        out.append(build_hchain(n, d))
    out.append(build_ppp('polyene', 8))
    out.append(build_ppp('polyene', 40, orbitals="local"))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_equals_individual(precision):
    Hs = _systems()
    syst = [(H.occ_of_pair, H.vir_of_pair, torch.from_numpy(H.h).cuda(),
             torch.from_numpy(H.eri).cuda(), H.e_const) for H in Hs]
    rc, e_b, infos, amps = ppq.pq_solve_batched(syst, precision=precision, max_iter=400,
                                                with_amplitudes=True)
    n_ok = 0
    for k, (H, s) in enumerate(zip(Hs, syst)):
        rc1, e1, t1, i1 = ppq.pq_solve(*s, precision=precision, max_iter=400)
        assert rc1 == infos[k]['status'], (H.name, rc1, infos[k]['status'])
        if rc1 == 0:
            n_ok += 1
            assert abs(e1 - e_b[k]) < 1e-9, (H.name, e1, e_b[k])
            assert np.abs(t1 - amps[k]).max() < 1e-6
    assert rc == max(i['status'] for i in infos)
    assert n_ok >= len(Hs) - 2
    # small members against the oracle
    for k, H in enumerate(Hs):
        if H.n_pairs <= 4 and infos[k]['status'] == 0:
            P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=2, e_const=H.e_const)
            r = P.solve(r_tol=1e-11, e_tol=1e-13, max_iter=400)
            assert r['converged'] and abs(r['e_corr'] + P.e_ref - e_b[k]) < 1e-9


def test_batched_reports_per_system_status():
    H = build_hchain(8, 1.2)
    syst = [(H.occ_of_pair, H.vir_of_pair, torch.from_numpy(H.h).cuda(),
             torch.from_numpy(H.eri).cuda(), H.e_const)] * 3
    rc, e_b, infos = ppq.pq_solve_batched(syst, max_iter=2)
    assert rc == 1 and all(i['status'] == 1 for i in infos)
    assert np.all(e_b == e_b[0])
