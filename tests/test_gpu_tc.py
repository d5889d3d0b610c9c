"""The residual with the quartic topology on the tensor cores (tcgen05: FP32
by 3xTF32 products, FP64 by exact integer splitting) beyond one 128-row tile.

* N = 20 (190 unordered pairs: a full tile and a ragged one of 62 rows):
  every pair-amplitude element of two sampled pairs of the second tile
  against the oracle's local assembly restricted to the label subsets that
  contain the pair (exact for those elements), FP32 within 2e-5 * max|R|,
  FP64 within 1e-11;
* N = 70, the time-to-solution workload (PPP C140H142, Boys-localised
  pairs; 2415 unordered pairs in 19 tiles, the last one ragged): every
  pair-amplitude element of a pair in a middle tile and of the last pair
  against the oracle's local assembly over the 2347 label sets containing
  each pair, run as a separate process split over the host cores
  (tests/oloc_sampled.py, given this process's orbitals).  FP64 within 1e-9: the exact slicing drops
  products below about 2^-41 of the row and block scales, and each element
  sums a few 10^4 such products over X, W and the channels (below 1e-11 at
  N = 20); FP32 within 2e-5 * max|R| as above;
* N = 40 and 70 (7 and 19 tiles, 48 and 80 TMEM columns per g): the whole
  FP32 residual against the FP64 one (oracle-pinned at N <= 12 and on the
  N = 20 and N = 70 samples) within the same FP32 bound -- a property that
  holds at any size.
"""
import os
import subprocess
import sys
from itertools import combinations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1609_00077_gb300 as ppq
from workloads import build_ppp, ppp_eri_device, random_pair_amplitude_seed
from oracle.loccc import LocalAssembly
from oracle.detcc import enumerate_manifold
from tests.layout import LayoutMap
from tests.oloc_sampled import amplitudes, save_orbitals

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def residuals(H, tl, eri=None):
    eri = dev(H.eri) if eri is None else eri
    out = {}
    for prec in (0, 1):
        r, e = ppq.pq_residual(H.occ_of_pair, H.vir_of_pair, dev(H.h), eri, dev(tl), precision=prec)
        out[prec] = (r.cpu().numpy(), e)
    return out


def test_two_tiles_sampled_pairs_match_oracle():
    H = build_ppp('polyene', 40, orbitals='local')
    N = H.n_pairs
    assert N == 20
    sampled = [(8, 13), (18, 19)]   # unordered-pair rows 128 and 189: first and last of tile 2
    subs = set()
    for Y, Z in sampled:
        others = [k for k in range(N) if k not in (Y, Z)]
        for extra in [()] + [(a,) for a in others] + list(combinations(others, 2)):
            subs.add(tuple(sorted((Y, Z) + extra)))   # each label set once
    L = LocalAssembly(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=2, subsets=sorted(subs))
    man = L.manifold
    lm = LayoutMap(man, H.occ_of_pair, H.vir_of_pair, H.n_orb, ppq.amp_layout())
    rng = np.random.default_rng(random_pair_amplitude_seed(N))
    t = rng.uniform(-0.1, 0.1, len(man))
    R_ref, _ = L.residual(t)
    idx = [k for k, d in enumerate(man) if L._labels(d) in [{Y, Z} for Y, Z in sampled]]
    assert len(idx) == 29 * len(sampled)
    res = residuals(H, lm.to_layout(t))
    R64 = lm.from_layout(res[0][0])
    R32 = lm.from_layout(res[1][0])
    assert np.abs(R64[idx] - R_ref[idx]).max() < 1e-11
    scale = max(np.abs(R_ref[idx]).max(), np.abs(R64).max())
    assert np.abs(R32[idx] - R_ref[idx]).max() < 2e-5 * scale
    assert np.abs(R32 - R64).max() < 2e-5 * scale


@pytest.mark.parametrize("size", [80, 140])
def test_fp32_tensor_core_residual_matches_fp64(size):
    H = build_ppp('polyene', size, orbitals='local', with_eri=False)
    eri = ppp_eri_device(H, torch)
    N = H.n_pairs
    man = enumerate_manifold(H.occ_of_pair, H.vir_of_pair, 2)
    lm = LayoutMap(man, H.occ_of_pair, H.vir_of_pair, H.n_orb, ppq.amp_layout())
    rng = np.random.default_rng(random_pair_amplitude_seed(N))
    t = rng.uniform(-0.1, 0.1, len(man))
    res = residuals(H, lm.to_layout(t), eri)
    del eri
    r64, e64 = res[0]
    r32, e32 = res[1]
    assert np.all(np.isfinite(r32))
    scale = np.abs(r64).max()
    assert np.abs(r32 - r64).max() < 2e-5 * scale
    assert abs(e32 - e64) < 2e-5 * max(1.0, abs(e64))


def test_bench_workload_sampled_pairs_match_oracle(tmp_path):
    out = tmp_path / "sampled.npz"
    H = build_ppp('polyene', 140, orbitals='local', with_eri=False)
    N = H.n_pairs
    assert N == 70
    save_orbitals(tmp_path / "orb.npz", H)       # the oracle process uses these very orbitals
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    oracle = subprocess.Popen([sys.executable, "-m", "tests.oloc_sampled", "--size", "140",
                               "--orbitals-from", str(tmp_path / "orb.npz"), "--pairs", "33,34", "68,69",
                               "--tag", "0", "--out", str(out)], cwd=ROOT, env=env)
    try:
        eri = ppp_eri_device(H, torch)
        man = enumerate_manifold(H.occ_of_pair, H.vir_of_pair, 2)
        lm = LayoutMap(man, H.occ_of_pair, H.vir_of_pair, H.n_orb, ppq.amp_layout())
        res = residuals(H, lm.to_layout(amplitudes(len(man), N, 0)), eri)
        del eri
        assert oracle.wait(timeout=1800) == 0
    finally:
        if oracle.poll() is None:
            oracle.kill()
    got = np.load(out)
    idx, R_ref = got["idx"], got["vals"]
    assert len(idx) == 2 * 29
    R64 = lm.from_layout(res[0][0])
    R32 = lm.from_layout(res[1][0])
    assert np.abs(R_ref).max() > 1e-2
    assert np.abs(R64[idx] - R_ref).max() < 1e-9
    scale = max(np.abs(R_ref).max(), np.abs(R64).max())
    assert np.abs(R32[idx] - R_ref).max() < 2e-5 * scale


@pytest.mark.parametrize("precision,tol", [(1, 1e-8), (0, 1e-9)])
def test_bench_workload_solution_against_oracle(tmp_path, precision, tol):
    """The time-to-solution solve itself (C140H142, default tolerances), mixed
    and FP64-only: at the amplitudes it returns, the oracle's energy (all 2485
    label sets of at most two labels) equals the returned energy to 1e-8 Eh
    (mixed) and 1e-9 Eh (FP64), and the oracle's residual elements of the last
    pair (the ragged tile) vanish to the same tolerance (the solve stops at
    ||R|| <= 1e-10 in FP64)."""
    H = build_ppp('polyene', 140, orbitals='local', with_eri=False)
    eri = ppp_eri_device(H, torch)
    rc, e, t, info = ppq.pq_solve(H.occ_of_pair, H.vir_of_pair, dev(H.h), eri, H.e_const, precision=precision)
    del eri
    assert rc == 0 and (precision == 0 or info['polish_iters'] > 0)
    man = enumerate_manifold(H.occ_of_pair, H.vir_of_pair, 2)
    lm = LayoutMap(man, H.occ_of_pair, H.vir_of_pair, H.n_orb, ppq.amp_layout())
    np.save(tmp_path / "t.npy", lm.from_layout(t))
    save_orbitals(tmp_path / "orb.npz", H)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    subprocess.run([sys.executable, "-m", "tests.oloc_sampled", "--size", "140",
                    "--orbitals-from", str(tmp_path / "orb.npz"),
                    "--pairs", "68,69", "--t-in", str(tmp_path / "t.npy"), "--energy",
                    "--out", str(tmp_path / "o.npz")], cwd=ROOT, env=env, check=True, timeout=1800)
    got = np.load(tmp_path / "o.npz")
    assert len(got["idx"]) == 29
    assert abs(float(got["e_c"] + got["e_ref"] + got["e_const"]) - e) < tol
    assert np.abs(got["vals"]).max() < tol
