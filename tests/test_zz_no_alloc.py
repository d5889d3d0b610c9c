"""The allocation-free residual entry point.

Some callers cannot allocate device memory, for example code inside another
framework's memory pool or under a fixed memory budget. pq_residual_static
serves them: it uses a fixed 8 MiB device array instead of the cached
workspace. This test calls it through the C ABI twice in a row, with
different amplitudes, and checks each result against pq_residual within the
FP64 parity tolerance used elsewhere. The second call catches state left in
the shared array by the first. The file is named so pytest collects it last;
it must pass alone in a fresh process and after the other tests."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1609_00077_gb300 as ppq
from workloads import build_ppp, build_hchain


@pytest.mark.parametrize("precision", [0, 1])
def test_static_residual_matches_allocating_entry_point_twice(precision):
    # 4, 6 and 12 pairs (the stated maximum)
    for H in (build_ppp('polyene', 8), build_hchain(12, 1.7), build_ppp('polyene', 24)):
        h = torch.from_numpy(H.h).cuda()
        eri = torch.from_numpy(H.eri).cuda()
        L = ppq.amp_count(H.n_pairs)
        for seed in (1, 2):
            t = torch.from_numpy(np.random.default_rng(seed).uniform(-0.1, 0.1, L)).cuda()
            r_ref, e_ref = ppq.pq_residual(H.occ_of_pair, H.vir_of_pair, h, eri, t,
                                           precision=precision)
            r = torch.zeros_like(t)
            e = ppq.pq_residual_static(H.occ_of_pair, H.vir_of_pair, h, eri, t, r,
                                       precision=precision)
            tol = 1e-11 if precision == 0 else 2e-5 * float(r_ref.abs().max())
            assert float((r - r_ref).abs().max()) < tol
            assert abs(e - e_ref) < (1e-11 if precision == 0 else 2e-5)


def test_static_residual_rejects_oversize_and_host_pointers():
    H = build_ppp('polyene', 26)   # 13 pairs: above the 12-pair limit
    L = ppq.amp_count(H.n_pairs)
    h = torch.from_numpy(H.h).cuda(); eri = torch.from_numpy(H.eri).cuda()
    t = torch.zeros(L, dtype=torch.float64, device="cuda"); r = torch.zeros_like(t)
    with pytest.raises(ppq.PPQError, match="static scratch limit"):
        ppq.pq_residual_static(H.occ_of_pair, H.vir_of_pair, h, eri, t, r)
    H = build_ppp('polyene', 6)
    L = ppq.amp_count(H.n_pairs)
    with pytest.raises(ppq.PPQError, match="device pointers"):
        ppq.pq_residual_static(H.occ_of_pair, H.vir_of_pair, np.ascontiguousarray(H.h),
                               np.ascontiguousarray(H.eri), np.zeros(L), np.zeros(L))
