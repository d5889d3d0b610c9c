"""Oracle for the Lambda (left) equations and energy gradients of PQ/PH
(test infrastructure only; see the package header).

The Lagrangian of the projected CC equations is
    L(t, lambda) = E_c(t) + sum_mu lambda_mu R_mu(t),
stationary in t at the Lambda solution (Theory section: lambda lives on the
same truncated manifold as t, Table I).  Because R and E_c are polynomials in
t, derivatives with respect to t are taken exactly by the complex step
dF/dt_k = Im F(t + i h e_k) / h (no subtraction, h = 1e-30), through the same
determinant-space evaluator O-det.

    J[nu, mu]  = dR_nu / dt_mu        (complex step, column by column)
    b[mu]      = dE_c / dt_mu
    J^T lambda = -b                    (dense solve)
    grad_t L   = b + J^T lambda        (zero at the solution)

Integral gradients of the total energy are checked by central finite
differences of converged energies (perturbing all symmetry copies together),
and at four electrons in four orbitals by the FCI one-particle density matrix
(Hellmann-Feynman: PQ is FCI there, so dE/dh_pq equals the FCI 1-RDM).
"""
import numpy as np

from .detcc import Problem
from .fci import Strings, sigma


def _complex_step(f, t, k, h=1e-30):
    tc = t.astype(complex)
    tc[k] += 1j * h
    return f(tc)


def jacobian(P, t, h=1e-30):
    """(J, b) at amplitudes t for Problem P: J[nu, mu] = dR_nu/dt_mu,
    b[mu] = dE_c/dt_mu."""
    n = P.cc.n_amp
    J = np.empty((n, n))
    b = np.empty(n)
    for k in range(n):
        Rc, ec = _complex_step(lambda tc: P.cc.residual(tc, P.hp, P.vt), t, k, h)
        J[:, k] = np.imag(Rc) / h
        b[k] = np.imag(ec) / h
    return J, b


def grad_t_lagrangian(P, t, lam, h=1e-30):
    """grad_t L = dE_c/dt + J^T lambda at arbitrary (t, lambda)."""
    J, b = jacobian(P, t, h)
    return b + J.T @ lam


def solve_lambda(P, t):
    """Lambda amplitudes at converged t: J^T lambda = -dE_c/dt."""
    J, b = jacobian(P, t)
    return np.linalg.solve(J.T, -b)


def _fci_ground(h, eri, n_alpha):
    """(strings, C[I_alpha, I_beta]) of the lowest FCI state (dense
    diagonalisation, small spaces)."""
    n = h.shape[0]
    S = Strings(n, n_alpha)
    dim = S.n * S.n
    Hm = np.empty((dim, dim))
    for j in range(dim):
        c = np.zeros(dim); c[j] = 1.0
        Hm[:, j] = sigma(S, h, eri, c.reshape(S.n, S.n)).ravel()
    w, v = np.linalg.eigh(0.5 * (Hm + Hm.T))
    return S, v[:, 0].reshape(S.n, S.n)


def _spin_summed(S, C):
    """E_pq C for every p, q (spin-summed one-body operators on C)."""
    E = S.E()
    n = len(E)
    return [[E[p][q] @ C + (E[p][q] @ C.T).T for q in range(n)] for p in range(n)]


def fci_one_rdm(h, eri, n_alpha):
    """Spin-summed FCI 1-RDM gamma_pq = <Psi| sum_s a+_ps a_qs |Psi> of the
    lowest state (dense diagonalisation, small spaces)."""
    S, C = _fci_ground(h, eri, n_alpha)
    X = _spin_summed(S, C)
    n = h.shape[0]
    return np.array([[np.sum(C * X[p][q]) for q in range(n)] for p in range(n)])


def fci_two_rdm(h, eri, n_alpha):
    """Spin-summed FCI 2-RDM in the chemists' order of the Hamiltonian,
    Gamma_pqrs = sum_{s,t} <Psi| a+_ps a+_rt a_st a_qs |Psi>
               = <Psi| E_pq E_rs |Psi> - delta_qr gamma_ps,
    so that E = sum h_pq gamma_pq + 1/2 sum (pq|rs) Gamma_pqrs."""
    S, C = _fci_ground(h, eri, n_alpha)
    X = _spin_summed(S, C)
    n = h.shape[0]
    V = np.array([[X[p][q].ravel() for q in range(n)] for p in range(n)])   # E_pq Psi
    g = np.einsum('i,pqi->pq', C.ravel(), V)
    # <Psi| E_pq E_rs |Psi> = (E_qp Psi) . (E_rs Psi)
    G = np.einsum('qpi,rsi->pqrs', V, V)
    G -= np.einsum('qr,ps->pqrs', np.eye(n), g)
    return G


def energy(h, eri, occ, vir, K, e_const=0.0, K_H=0, **kw):
    P = Problem(h, eri, occ, vir, K=K, K_H=K_H, e_const=e_const)
    r = P.solve(r_tol=1e-12, e_tol=1e-14, max_iter=600, **kw)
    assert r['converged']
    return r['e_corr'] + P.e_ref
