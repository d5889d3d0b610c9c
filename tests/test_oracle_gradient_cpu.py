"""Pins of the gradient oracle (oracle/gradient.py) on the CPU, against
independent numerical and physical facts.

* The complex-step Jacobian dR/dt equals central finite differences of the
  residual.
* The FCI one-particle density matrix is Hermitian with trace equal to the
  number of electrons, and (Hellmann-Feynman) its contraction with a
  symmetric change of h is the derivative of the FCI energy; the two-particle
  one rebuilds the FCI energy with it, traces down to (n_el - 1) gamma, and
  gives the derivative along a symmetric change of (pq|rs).
* The Lambda amplitudes turn the Lagrangian into the total derivative of the
  converged energy: for a change of h and (pq|rs), the partial derivative of
  E_ref + E_c(t) + lambda . R(t) at the converged t equals the central
  difference of re-converged PQ energies (Theory section: lambda on the same
  manifold as t).
"""
import numpy as np

from workloads import build_ppp, build_hchain
from oracle.detcc import Problem
from oracle.fci import fci_energy
from oracle.gradient import jacobian, fci_one_rdm, fci_two_rdm, solve_lambda, energy


def _sym(n, rng):
    dh = rng.normal(size=(n, n)); dh = dh + dh.T
    dv = rng.normal(size=(n, n, n, n))
    dv = dv + dv.transpose(1, 0, 2, 3); dv = dv + dv.transpose(0, 1, 3, 2); dv = dv + dv.transpose(2, 3, 0, 1)
    return dh, dv


def test_complex_step_jacobian_matches_central_differences():
    H = build_ppp('polyene', 6)
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=2)
    t = np.random.default_rng(2).uniform(-0.05, 0.05, P.cc.n_amp)
    J, b = jacobian(P, t)
    eps = 1e-5
    for k in (0, 5, 17, 40, P.cc.n_amp - 1):
        tp, tm = t.copy(), t.copy()
        tp[k] += eps; tm[k] -= eps
        (Rp, ep), (Rm, em) = P.residual(tp), P.residual(tm)
        assert np.abs(J[:, k] - (Rp - Rm) / (2 * eps)).max() < 1e-8
        assert abs(b[k] - (ep - em) / (2 * eps)) < 1e-8


def test_fci_one_rdm_trace_symmetry_and_hellmann_feynman():
    H = build_hchain(6, 1.3)
    g = fci_one_rdm(H.h, H.eri, 3)
    assert abs(np.trace(g) - 6.0) < 1e-10
    assert np.abs(g - g.T).max() < 1e-10
    w = np.linalg.eigvalsh(g)
    assert w.min() > -1e-10 and w.max() < 2.0 + 1e-10
    dh, _ = _sym(H.n_orb, np.random.default_rng(3))
    eps = 1e-5
    fd = (fci_energy(H.h + eps * dh, H.eri, 3) - fci_energy(H.h - eps * dh, H.eri, 3)) / (2 * eps)
    assert abs(fd - np.sum(g * dh)) < 1e-7


def test_fci_two_rdm_energy_trace_and_hellmann_feynman():
    H = build_hchain(6, 1.3)
    g = fci_one_rdm(H.h, H.eri, 3)
    G = fci_two_rdm(H.h, H.eri, 3)
    e = fci_energy(H.h, H.eri, 3)
    assert abs(np.sum(H.h * g) + 0.5 * np.sum(H.eri * G) - e) < 1e-10
    assert np.abs(np.einsum('pqrr->pq', G) - 5.0 * g).max() < 1e-10
    _, dv = _sym(H.n_orb, np.random.default_rng(4))
    dv *= 0.01
    eps = 1e-4
    fd = (fci_energy(H.h, H.eri + eps * dv, 3) - fci_energy(H.h, H.eri - eps * dv, 3)) / (2 * eps)
    assert abs(fd - 0.5 * np.sum(G * dv)) < 1e-7


def test_lambda_makes_the_lagrangian_derivative_total():
    H = build_ppp('polyene', 6)       # N = 3: PQ is not FCI here
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=2, e_const=H.e_const)
    r = P.solve(r_tol=1e-13, e_tol=1e-15, max_iter=600)
    assert r['converged']
    t = r['t']
    lam = solve_lambda(P, t)
    rng = np.random.default_rng(11)
    dh, dv = _sym(H.n_orb, rng)
    dh *= 0.05; dv *= 0.005
    eps = 1e-4

    def lagrangian(s):
        Q = Problem(H.h + s * dh, H.eri + s * dv, H.occ_of_pair, H.vir_of_pair, K=2, e_const=H.e_const)
        R, ec = Q.residual(t)
        return Q.e_ref + ec + lam @ R

    partial = (lagrangian(eps) - lagrangian(-eps)) / (2 * eps)
    E = lambda s: energy(H.h + s * dh, H.eri + s * dv, H.occ_of_pair, H.vir_of_pair, 2, H.e_const)
    total = (E(eps) - E(-eps)) / (2 * eps)
    assert abs(partial - total) < 1e-7
    # without lambda the partial derivative misses the amplitude response
    def no_lambda(s):
        Q = Problem(H.h + s * dh, H.eri + s * dv, H.occ_of_pair, H.vir_of_pair, K=2, e_const=H.e_const)
        return Q.e_ref + Q.residual(t)[1]
    assert abs((no_lambda(eps) - no_lambda(-eps)) / (2 * eps) - total) > 1e-6
