"""Adjoint (Lambda) kernels against the oracle.

grad_t L(t, lambda) = dE_c/dt + J^T lambda at random (t, lambda) is compared
element by element with the oracle's complex-step Jacobian (exact for the
polynomial residual), and the Lambda amplitudes solved at converged t are
compared with the oracle's dense solve of J^T lambda = -dE_c/dt.
Tolerance 1e-10 absolute for the gradient (FP64, |entries| <= ~1), 1e-8 for
lambda (both sides converged to ~1e-11 and amplified by ||J^-1|| ~ 10).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1609_00077_gb300 as ppq
from workloads import build_ppp, build_hchain
from oracle.detcc import Problem
from oracle.gradient import jacobian, solve_lambda
from tests.layout import LayoutMap

SYSTEMS = {
    "H4": lambda: build_hchain(4, 1.5),
    "C6H8": lambda: build_ppp('polyene', 6),
    "C8H10": lambda: build_ppp('polyene', 8),
    "H8": lambda: build_hchain(8, 1.3),
}


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_lagrangian_gradient_random_point(name):
    H = SYSTEMS[name]()
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=2)
    lm = LayoutMap(P.cc.manifold, H.occ_of_pair, H.vir_of_pair, H.n_orb, ppq.amp_layout())
    rng = np.random.default_rng(20 + H.n_pairs)
    t = rng.uniform(-0.1, 0.1, P.cc.n_amp)
    lam = rng.uniform(-0.1, 0.1, P.cc.n_amp)
    J, b = jacobian(P, t)
    g_ref = b + J.T @ lam
    g, e = ppq.pq_lagrangian_gradient(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri),
                                      dev(lm.to_layout(t)), dev(lm.to_layout(lam)))
    g = g.cpu().numpy()
    assert lm.mirror_error(g) < 1e-12
    assert np.abs(lm.from_layout(g) - g_ref).max() < 1e-10


@pytest.mark.parametrize("name", ["H4", "C8H10", "H8"])
def test_lambda_matches_oracle(name):
    H = SYSTEMS[name]()
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=2, e_const=H.e_const)
    ro = P.solve(r_tol=1e-12, e_tol=1e-14, max_iter=400)
    assert ro['converged']
    lam_ref = solve_lambda(P, ro['t'])
    lm = LayoutMap(P.cc.manifold, H.occ_of_pair, H.vir_of_pair, H.n_orb, ppq.amp_layout())
    h, eri = dev(H.h), dev(H.eri)
    rc, e, t, info = ppq.pq_solve(H.occ_of_pair, H.vir_of_pair, h, eri, H.e_const,
                                  r_tol=1e-12, e_tol=1e-14, max_iter=400)
    assert rc == 0
    rc, lam, li = ppq.pq_lambda(H.occ_of_pair, H.vir_of_pair, h, eri, t, r_tol=1e-11, max_iter=400)
    assert rc == 0, li
    assert np.abs(lm.from_layout(lam) - lam_ref).max() < 1e-8
