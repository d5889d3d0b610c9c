"""The process-split sampled oracle (tests/oloc_sampled.py) as GPU tests run
it -- a command in a fresh process -- against the oracle's serial local
assembly over every label set, at N = 6."""
import os
import subprocess
import sys

import numpy as np

from oracle.detcc import enumerate_manifold
from oracle.loccc import LocalAssembly
from tests.oloc_sampled import workload, amplitudes, pair_subsets

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_pair_subsets_count():
    # 1 + (N - 2) + C(N - 2, 2) label sets per pair for PQ; shared ones once
    assert len(pair_subsets(70, [(33, 34)], 4)) == 1 + 68 + 68 * 67 // 2
    assert len(pair_subsets(6, [(0, 1), (0, 1)], 4)) == 1 + 4 + 6


def _run(args, cwd):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    subprocess.run([sys.executable, "-m", "tests.oloc_sampled"] + args, cwd=cwd, env=env,
                   check=True, timeout=600)


def test_sampled_command_matches_serial_oracle(tmp_path):
    H = workload("polyene", 12, "canonical")
    man = enumerate_manifold(H.occ_of_pair, H.vir_of_pair, 2)
    L = LocalAssembly(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=2)
    # seeded amplitudes
    out = tmp_path / "s.npz"
    _run(["--size", "12", "--pairs", "0,1", "2,5", "--tag", "3", "--workers", "2", "--out", str(out)], ROOT)
    got = np.load(out)
    R, _ = L.residual(amplitudes(len(man), H.n_pairs, 3))
    assert len(got["idx"]) == 2 * 29
    assert np.abs(R[got["idx"]]).max() > 1e-3
    assert np.abs(got["vals"] - R[got["idx"]]).max() < 1e-13
    assert np.isnan(got["e_c"]) and abs(got["e_ref"] - L.e_ref) < 1e-12
    # given amplitudes, with the energy
    t = np.random.default_rng(11).uniform(-0.05, 0.05, len(man))
    np.save(tmp_path / "t.npy", t)
    _run(["--size", "12", "--pairs", "1,4", "--t-in", str(tmp_path / "t.npy"), "--energy",
          "--workers", "3", "--out", str(out)], ROOT)
    got = np.load(out)
    R, e = L.residual(t)
    assert np.abs(got["vals"] - R[got["idx"]]).max() < 1e-13
    assert abs(got["e_c"] - e) < 1e-12 and abs(e) > 1e-3


def test_sampled_command_with_the_callers_orbitals(tmp_path):
    """--orbitals-from: the command transforms the PPP model with the
    caller's orbitals and pairing (as the GPU tests pass them)."""
    from workloads import build_ppp
    from tests.oloc_sampled import save_orbitals
    H = build_ppp('polyene', 12, orbitals='local')
    save_orbitals(tmp_path / "orb.npz", H)
    man = enumerate_manifold(H.occ_of_pair, H.vir_of_pair, 2)
    t = np.random.default_rng(12).uniform(-0.05, 0.05, len(man))
    np.save(tmp_path / "t.npy", t)
    _run(["--size", "12", "--orbitals-from", str(tmp_path / "orb.npz"), "--pairs", "2,3",
          "--t-in", str(tmp_path / "t.npy"), "--energy", "--workers", "2", "--out", str(tmp_path / "o.npz")], ROOT)
    got = np.load(tmp_path / "o.npz")
    R, e = LocalAssembly(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=2).residual(t)
    assert np.abs(got["vals"] - R[got["idx"]]).max() < 1e-12
    assert abs(got["e_c"] - e) < 1e-12 and abs(got["e_const"] - H.e_const) < 1e-12
