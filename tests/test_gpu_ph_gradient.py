"""The PH reverse pass (ph_lagrangian_gradient) and energy gradients
(ph_gradient) against the oracle and against facts the mathematics fixes.

* grad_t L = dE_c/dt + J^T lambda element by element against the oracle's
  complex-step Jacobian through O-det (N = 2 with three- and two-label
  integrals, N = 3), tolerance 1e-10 (FP64; the same exact terms in another
  order);
* at N = 7 (every subset size enters with a nonzero coefficient) the
  directional derivative along a random direction equals the central
  difference of L = E_c + lambda . R from FP64 GPU residuals (themselves held
  to the oracle element by element in test_gpu_ph.py), tolerance 1e-6
  relative; and two calls give identical bits;
* hexatriene 6e/6o: PH is FCI there, so by Hellmann-Feynman dE/dh is the FCI
  one-particle density matrix, dE/d(pq|rs) half the FCI two-particle one
  (both symmetrised), and dE/dkappa vanishes (FCI is invariant to orbital
  rotations); tolerance 1e-8;
* octatetraene (N = 4): central differences (step 1e-4) of converged oracle PH
  energies along a random symmetric direction in (h, (pq|rs)) (scaled by 0.1
  and 0.01 as in the PQ tests: the energy's third derivative along an
  unscaled random (pq|rs) direction makes the difference quotient miss by
  3e-2 at this step, by 3e-4 at 1e-5) and along a random orbital rotation,
  tolerance 1e-6;
* naphthalene (N = 5): central differences of converged GPU energies along
  random directions and for single symmetric elements of h and (pq|rs); the
  torch.autograd function (ph_energy) returns the same dE/dh, dE/d(pq|rs)
  and, through an orbital rotation, dE/dkappa.
"""
import numpy as np
import pytest
from scipy.linalg import expm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1609_00077_gb300 as ppq
from workloads import build_ppp
from oracle.detcc import Problem
from oracle.gradient import grad_t_lagrangian, fci_one_rdm, fci_two_rdm, energy
from tests.layout import LayoutMap

TIGHT = dict(r_tol=1e-12, e_tol=1e-14, max_iter=600)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def sym_dirs(n, rng):
    dh = rng.normal(size=(n, n)); dh = dh + dh.T
    dv = rng.normal(size=(n, n, n, n))
    dv = dv + dv.transpose(1, 0, 2, 3); dv = dv + dv.transpose(0, 1, 3, 2)
    dv = dv + dv.transpose(2, 3, 0, 1)
    return dh, dv


def rotate(h, eri, U):
    return U.T @ h @ U, np.einsum('pqrs,pi,qj,rk,sl->ijkl', eri, U, U, U, U, optimize=True)


def sym8(G):
    return (G + G.transpose(1, 0, 2, 3) + G.transpose(0, 1, 3, 2) + G.transpose(1, 0, 3, 2)
            + G.transpose(2, 3, 0, 1) + G.transpose(3, 2, 0, 1) + G.transpose(2, 3, 1, 0)
            + G.transpose(3, 2, 1, 0)) / 8.0


@pytest.mark.parametrize("sites,K_H", [(4, 3), (4, 2), (6, 3)])
def test_lagrangian_gradient_matches_oracle_complex_step(sites, K_H):
    H = build_ppp('polyene', sites)
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=3, K_H=K_H)
    rng = np.random.default_rng(31 + sites + K_H)
    t = rng.uniform(-0.1, 0.1, P.cc.n_amp)
    lam = rng.uniform(-0.1, 0.1, P.cc.n_amp)
    g_ref = grad_t_lagrangian(P, t, lam)
    lm = LayoutMap(P.cc.manifold, H.occ_of_pair, H.vir_of_pair, H.n_orb, ppq.amp_layout(3))
    g, e = ppq.ph_lagrangian_gradient(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri),
                                      dev(lm.to_layout(t)), dev(lm.to_layout(lam)), K_H=K_H)
    gv = g.cpu().numpy()
    assert np.abs(g_ref).max() > 0.05
    assert np.abs(lm.from_layout(gv) - g_ref).max() < 1e-10
    assert lm.mirror_error(gv) == 0.0
    assert abs(e - P.residual(t)[1]) < 1e-11


def _unique_slots(N):
    from tests.test_gpu_ph import _unique_mask
    return _unique_mask(N)


def test_lagrangian_gradient_directional_n7_and_reproducible():
    H = build_ppp('polyene', 14)
    N = H.n_pairs
    L = ppq.amp_count(N, 3)
    uniq = _unique_slots(N)
    rng = np.random.default_rng(7)
    # amplitudes with consistent copies: the residual of zero-copy input fills them
    t0 = np.where(uniq, rng.uniform(-0.05, 0.05, L), 0.0)
    lam = np.where(uniq, rng.uniform(-0.1, 0.1, L), 0.0)
    d = np.where(uniq, rng.normal(size=L), 0.0)
    args = (H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri))
    g1, _ = ppq.ph_lagrangian_gradient(*args, dev(t0), dev(lam))
    g2, _ = ppq.ph_lagrangian_gradient(*args, dev(t0), dev(lam))
    assert torch.equal(g1, g2)
    g = g1.cpu().numpy()

    def lag(tv):
        r, e = ppq.ph_residual(*args, dev(tv))
        return e + float(np.sum(lam[uniq] * r.cpu().numpy()[uniq]))

    eps = 1e-4
    fd = (lag(t0 + eps * d) - lag(t0 - eps * d)) / (2 * eps)
    an = float(np.sum(g[uniq] * d[uniq]))
    assert abs(an) > 1e-2
    assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (fd, an)


def test_ph_gradient_is_fci_density_at_6e6o():
    H = build_ppp('polyene', 6)
    rc, e, dh, dv, dk, info = ppq.ph_gradient(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), H.e_const,
                                              precision=0, **TIGHT)
    assert rc == 0
    g = fci_one_rdm(H.h, H.eri, 3)
    assert np.abs(dh.cpu().numpy() - g).max() < 1e-8
    assert np.abs(dk.cpu().numpy()).max() < 1e-8
    G = sym8(0.5 * fci_two_rdm(H.h, H.eri, 3))
    assert np.abs(dv.cpu().numpy() - G).max() < 1e-8


def test_ph_gradient_octatetraene_against_oracle_energy_differences():
    H = build_ppp('polyene', 8)
    n = H.n_orb
    rc, e, dh, dv, dk, info = ppq.ph_gradient(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), H.e_const,
                                              precision=0, **TIGHT)
    assert rc == 0
    dh, dv, dk = dh.cpu().numpy(), dv.cpu().numpy(), dk.cpu().numpy()
    rng = np.random.default_rng(11)
    Dh, Dv = sym_dirs(n, rng)
    Dh *= 0.1; Dv *= 0.01          # keeps the O(step^2) truncation of the differences below 1e-7
    step = 1e-4

    def E(h, eri):
        return energy(h, eri, H.occ_of_pair, H.vir_of_pair, 3, H.e_const, K_H=3)

    fd = (E(H.h + step * Dh, H.eri + step * Dv) - E(H.h - step * Dh, H.eri - step * Dv)) / (2 * step)
    an = np.sum(dh * Dh) + np.sum(dv * Dv)
    assert abs(fd - an) < 1e-6, (fd, an)
    kap = rng.normal(size=(n, n)); kap = kap - kap.T
    fk = (E(*rotate(H.h, H.eri, expm(step * kap))) - E(*rotate(H.h, H.eri, expm(-step * kap)))) / (2 * step)
    ak = 0.5 * np.sum(dk * kap)
    assert abs(ak) > 1e-4
    assert abs(fk - ak) < 1e-6, (fk, ak)


def test_ph_gradient_naphthalene_against_gpu_energy_differences():
    H = build_ppp('acene', 2)
    n = H.n_orb
    rc, e, dh, dv, dk, info = ppq.ph_gradient(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri), H.e_const,
                                              precision=0, **TIGHT)
    assert rc == 0
    dh, dv = dh.cpu().numpy(), dv.cpu().numpy()
    step = 1e-4

    def E(h, eri):
        rc, et, _, _ = ppq.ph_solve(H.occ_of_pair, H.vir_of_pair, dev(h), dev(eri), H.e_const, precision=0, **TIGHT)
        assert rc == 0
        return et

    rng = np.random.default_rng(12)
    Dh, Dv = sym_dirs(n, rng)
    Dh *= 0.1; Dv *= 0.01
    fd = (E(H.h + step * Dh, H.eri + step * Dv) - E(H.h - step * Dh, H.eri - step * Dv)) / (2 * step)
    assert abs(fd - (np.sum(dh * Dh) + np.sum(dv * Dv))) < 1e-6
    # single symmetric elements: h_oo, h_ov, and (pq|rs) classes over one to four labels
    occ, vir = H.occ_of_pair, H.vir_of_pair
    for (p, q) in [(occ[0], occ[0]), (occ[1], vir[3]), (vir[2], vir[4])]:
        D = np.zeros((n, n)); D[p, q] += 1.0; D[q, p] += 1.0
        fd = (E(H.h + step * D, H.eri) - E(H.h - step * D, H.eri)) / (2 * step)
        assert abs(fd - np.sum(dh * D)) < 1e-6, (p, q, fd, np.sum(dh * D))
    for (p, q, r, s) in [(occ[0], vir[0], occ[0], vir[0]), (occ[1], occ[1], vir[2], vir[2]),
                         (occ[0], vir[1], occ[2], vir[3]), (occ[0], vir[1], occ[1], vir[2])]:
        D = np.zeros((n,) * 4)
        for a, b, c, d in {(p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
                           (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)}:
            D[a, b, c, d] = 1.0
        fd = (E(H.h, H.eri + step * D) - E(H.h, H.eri - step * D)) / (2 * step)
        assert abs(fd - np.sum(dv * D)) < 1e-6, ((p, q, r, s), fd, np.sum(dv * D))


def test_ph_energy_autograd_naphthalene():
    H = build_ppp('acene', 2)
    h, eri = dev(H.h), dev(H.eri)
    rc, e, dh, dv, dk, info = ppq.ph_gradient(H.occ_of_pair, H.vir_of_pair, h, eri, H.e_const, precision=0,
                                              **TIGHT)
    assert rc == 0
    h2 = h.clone().requires_grad_(True); v2 = eri.clone().requires_grad_(True)
    kap = torch.zeros_like(h, requires_grad=True)
    E = ppq.ph_energy(h2, v2, H.occ_of_pair, H.vir_of_pair, H.e_const, kappa=kap, precision=0, **TIGHT)
    E.backward()
    assert abs(float(E.detach()) - e) < 1e-10
    # at kappa = 0 the rotation is the identity: h and (pq|rs) receive dE/dh, dE/d(pq|rs)
    assert float((h2.grad - dh).abs().max()) < 1e-9
    assert float((v2.grad - dv).abs().max()) < 1e-9
    assert float((kap.grad - dk).abs().max()) < 1e-9
