"""Batched solve: many Hamiltonians of different pair counts in one call give
the same energies and amplitudes as one-by-one solves (and, for the small
members, as the oracle).  The largest member (N = 20) is checked by the
oracle at the amplitudes the batched mixed-precision solve returns."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1609_00077_gb300 as ppq
from workloads import build_hchain, build_ppp
from oracle.detcc import Problem, enumerate_manifold
from tests.layout import LayoutMap
from tests.oloc_sampled import save_orbitals

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def test_batched_largest_member_against_oracle(tmp_path):
    """PPP C40H42 with Boys-localised pairs (N = 20) inside a mixed-precision
    batch: at the returned amplitudes the oracle's energy (every label set of
    at most two labels) equals the batched energy to 1e-8 Eh, and the oracle's
    residual elements of two sampled pairs, one per 128-row tile, vanish to
    1e-8 (the solve stops at ||R|| <= 1e-10 in FP64)."""
    Hs = _systems()
    syst = [(H.occ_of_pair, H.vir_of_pair, torch.from_numpy(H.h).cuda(),
             torch.from_numpy(H.eri).cuda(), H.e_const) for H in Hs]
    rc, e_b, infos, amps = ppq.pq_solve_batched(syst, precision=1, max_iter=400, with_amplitudes=True)
    k = len(Hs) - 1
    H = Hs[k]
    assert H.n_pairs == 20 and infos[k]['status'] == 0
    man = enumerate_manifold(H.occ_of_pair, H.vir_of_pair, 2)
    lm = LayoutMap(man, H.occ_of_pair, H.vir_of_pair, H.n_orb, ppq.amp_layout())
    np.save(tmp_path / "t.npy", lm.from_layout(amps[k]))
    save_orbitals(tmp_path / "orb.npz", H)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    subprocess.run([sys.executable, "-m", "tests.oloc_sampled", "--size", "40",
                    "--orbitals-from", str(tmp_path / "orb.npz"),
                    "--pairs", "0,1", "18,19", "--t-in", str(tmp_path / "t.npy"), "--energy",
                    "--out", str(tmp_path / "o.npz")], cwd=ROOT, env=env, check=True, timeout=1800)
    got = np.load(tmp_path / "o.npz")
    assert len(got["idx"]) == 2 * 29
    assert abs(float(got["e_c"] + got["e_ref"] + got["e_const"]) - e_b[k]) < 1e-8
    assert np.abs(got["vals"]).max() < 1e-8
