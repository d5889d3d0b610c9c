"""Natural occupation numbers and the single-pair starting guess (the paper's
occupation analysis of the acenes and its perfect-pairing guess for H50,
Results section) on the GPU, through the C ABI.

* ppq_natural_occupations: eigenvalues of symmetric matrices against numpy's
  (1e-12 relative), eigenvectors orthonormal and diagonalising;
* at 4e/4o PQ is exact, so the relaxed density of pq_gradient is the FCI
  one-particle density: its natural occupations equal those of the oracle's
  FCI density (1e-8) and sum to the electron count;
* guess = 2 (start from the single-pair, K = 1, truncation solved first)
  reaches the same PQ energy as the zero start (1e-9 Eh).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1609_00077_gb300 as ppq
from workloads import build_ppp, build_hchain
from oracle.gradient import fci_one_rdm


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("n", [1, 7, 40, 140])
def test_eigenvalues_of_symmetric_matrices(n):
    rng = np.random.default_rng(n)
    A = rng.normal(size=(n, n))
    A = A + A.T
    w = ppq.natural_occupations(dev(A))
    ref = np.sort(np.linalg.eigvalsh(A))[::-1]
    assert np.abs(w - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())
    if n <= 120:
        w2, V = ppq.natural_occupations(A, vectors=True)
        assert np.abs(V.T @ V - np.eye(n)).max() < 1e-12
        assert np.abs(V.T @ A @ V - np.diag(w2)).max() < 1e-10 * max(1.0, np.abs(ref).max())


def test_natural_occupations_pq_equal_fci_at_4e4o():
    H = build_hchain(4, 1.5)
    rc, e, dh, _, _, _ = ppq.pq_gradient(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), H.e_const,
                                         want_eri=False, r_tol=1e-11, e_tol=1e-13)
    assert rc == 0
    occ = ppq.natural_occupations(dh)
    ref = np.sort(np.linalg.eigvalsh(fci_one_rdm(H.h, H.eri, 2)))[::-1]
    assert abs(occ.sum() - 4.0) < 1e-9
    assert np.abs(occ - ref).max() < 1e-8
    assert 1.0 < occ[0] < 2.0 and 0.0 < occ[-1] < 0.5


@pytest.mark.parametrize("name", ["C8H10", "H10"])
def test_single_pair_guess_reaches_the_same_energy(name):
    H = build_ppp('polyene', 8) if name == "C8H10" else build_hchain(10, 1.4)
    rc0, e0, _, i0 = ppq.pq_solve(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), H.e_const, precision=0)
    rc2, e2, _, i2 = ppq.pq_solve(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), H.e_const, precision=0,
                                  guess=2)
    assert rc0 == 0 and rc2 == 0 and abs(e2 - e0) < 1e-9
