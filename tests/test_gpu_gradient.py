"""Energy gradients through the Lambda equations (pq_gradient) against
facts the paper and mathematics fix:

* 4 electrons in 4 orbitals: PQ is FCI (Abstract), so by Hellmann-Feynman
  dE/dh is the FCI one-particle density matrix, dE/d(pq|rs) half the FCI
  two-particle one (both symmetrised) and dE/dkappa vanishes (FCI is
  invariant to orbital rotations);
* central finite differences (step 1e-4) of converged oracle energies along
  random symmetric directions in h and (pq|rs), and along a random orbital
  rotation, for 6 and 8 orbitals; tolerance 1e-6;
* the same against GPU energies for 16 orbitals;
* the torch.autograd function returns the same gradients, and with an
  orbital rotation kappa the same dE/dkappa.
"""
import numpy as np
import pytest
from scipy.linalg import expm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1609_00077_gb300 as ppq
from workloads import build_ppp, build_hchain
from oracle.gradient import fci_one_rdm, fci_two_rdm, energy

TIGHT = dict(r_tol=1e-12, e_tol=1e-14, max_iter=600)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def sym_dirs(n, rng):
    dh = rng.normal(size=(n, n)); dh = dh + dh.T
    dv = rng.normal(size=(n, n, n, n))
    dv = (dv + dv.transpose(1, 0, 2, 3)); dv = dv + dv.transpose(0, 1, 3, 2)
    dv = dv + dv.transpose(2, 3, 0, 1)
    return dh, dv


def rotate(h, eri, U):
    return U.T @ h @ U, np.einsum('pqrs,pi,qj,rk,sl->ijkl', eri, U, U, U, U, optimize=True)


@pytest.mark.parametrize("which", ["butadiene", "H4"])
def test_fci_hellmann_feynman_at_4e4o(which):
    H = build_ppp('polyene', 4) if which == "butadiene" else build_hchain(4, 1.6)
    rc, e, dh, dv, dk, info = ppq.pq_gradient(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri),
                                              H.e_const, **TIGHT)
    assert rc == 0
    g = fci_one_rdm(H.h, H.eri, 2)
    assert np.abs(dh.cpu().numpy() - g).max() < 1e-8
    assert np.abs(dk.cpu().numpy()).max() < 1e-8
    # dE/d(pq|rs), averaged over the 8 index permutations, is half the FCI
    # two-body density averaged the same way
    G = 0.5 * fci_two_rdm(H.h, H.eri, 2)
    G8 = (G + G.transpose(1, 0, 2, 3) + G.transpose(0, 1, 3, 2) + G.transpose(1, 0, 3, 2)
          + G.transpose(2, 3, 0, 1) + G.transpose(3, 2, 0, 1) + G.transpose(2, 3, 1, 0)
          + G.transpose(3, 2, 1, 0)) / 8.0
    assert np.abs(dv.cpu().numpy() - G8).max() < 1e-8


@pytest.mark.parametrize("which", ["C6H8", "H8"])
def test_integral_and_orbital_gradients_vs_oracle_fd(which):
    H = build_ppp('polyene', 6) if which == "C6H8" else build_hchain(8, 1.4)
    n = H.n_orb
    rc, e, dh, dv, dk, info = ppq.pq_gradient(H.occ_of_pair, H.vir_of_pair, dev(H.h), dev(H.eri),
                                              H.e_const, **TIGHT)
    assert rc == 0
    dh, dv, dk = dh.cpu().numpy(), dv.cpu().numpy(), dk.cpu().numpy()
    rng = np.random.default_rng(7)
    eps = 1e-4
    ddh, ddv = sym_dirs(n, rng)
    ddh *= 0.1; ddv *= 0.01
    E = lambda hh, vv: energy(hh, vv, H.occ_of_pair, H.vir_of_pair, 2, H.e_const)
    fd = (E(H.h + eps * ddh, H.eri + eps * ddv) - E(H.h - eps * ddh, H.eri - eps * ddv)) / (2 * eps)
    an = np.sum(dh * ddh) + np.sum(dv * ddv)
    assert abs(fd - an) < 1e-6, (fd, an)
    # orbital rotation C -> C exp(eps kappa)
    K = rng.normal(size=(n, n)); K = K - K.T
    Ep = E(*rotate(H.h, H.eri, expm(eps * K)))
    Em = E(*rotate(H.h, H.eri, expm(-eps * K)))
    fdk = (Ep - Em) / (2 * eps)
    ank = sum(dk[p, q] * K[p, q] for p in range(n) for q in range(p + 1, n))
    assert abs(fdk - ank) < 1e-6, (fdk, ank)


def test_gradient_vs_gpu_fd_h16_and_autograd():
    H = build_hchain(16, 1.3)
    h, eri = dev(H.h), dev(H.eri)
    rc, e, dh, dv, dk, info = ppq.pq_gradient(H.occ_of_pair, H.vir_of_pair, h, eri, H.e_const, **TIGHT)
    assert rc == 0
    rng = np.random.default_rng(11)
    ddh, ddv = sym_dirs(H.n_orb, rng)
    ddh *= 0.1; ddv *= 0.01
    eps = 1e-4

    def E(hh, vv):
        r, ee, _, _ = ppq.pq_solve(H.occ_of_pair, H.vir_of_pair, dev(hh), dev(vv), H.e_const, **TIGHT)
        assert r == 0
        return ee
    fd = (E(H.h + eps * ddh, H.eri + eps * ddv) - E(H.h - eps * ddh, H.eri - eps * ddv)) / (2 * eps)
    an = float((dh.cpu() * torch.from_numpy(ddh)).sum() + (dv.cpu() * torch.from_numpy(ddv)).sum())
    assert abs(fd - an) < 1e-6, (fd, an)
    # torch.autograd
    h2 = h.clone().requires_grad_(True); v2 = eri.clone().requires_grad_(True)
    E2 = ppq.pq_energy(h2, v2, H.occ_of_pair, H.vir_of_pair, H.e_const, **TIGHT)
    E2.backward()
    assert abs(float(E2.detach()) - e) < 1e-10
    assert float((h2.grad - dh).abs().max()) < 1e-10
    assert float((v2.grad - dv).abs().max()) < 1e-10
    # the orbital-rotation gradient through autograd: E(U^T h U, U^4 eri),
    # U = exp(kappa - kappa^T), at kappa = 0
    kap = torch.zeros_like(h, requires_grad=True)
    E3 = ppq.pq_energy(h, eri, H.occ_of_pair, H.vir_of_pair, H.e_const, kappa=kap, **TIGHT)
    E3.backward()
    assert abs(float(E3.detach()) - e) < 1e-10
    assert float((kap.grad - dk).abs().max()) < 1e-9


def test_h50_asymmetric_gradient_vs_central_differences():
    """The gradient configuration: H50 as 25 H2 units (R = 1.4 bohr, unit gap
    1.8 A, Boys-localised pairs).  Central differences (step 1e-4) of GPU
    energies along a random symmetric (h, (pq|rs)) direction and a random
    orbital rotation agree with pq_gradient to 1e-6."""
    from workloads.hchain_torch import build_hchain_torch
    H = build_hchain_torch(50, 1.8, device="cuda", orbitals="local", bond_bohr=1.4)
    n = H.n_orb
    rc, e, dh, dv, dk, info = ppq.pq_gradient(H.occ_of_pair, H.vir_of_pair, H.h, H.eri, H.e_const,
                                              **TIGHT)
    assert rc == 0
    g = torch.Generator(device="cuda").manual_seed(1234)
    ddh = torch.randn((n, n), generator=g, device="cuda", dtype=torch.float64)
    ddh = 0.1 * (ddh + ddh.T)
    ddv = torch.randn((n, n, n, n), generator=g, device="cuda", dtype=torch.float64)
    ddv = ddv + ddv.permute(1, 0, 2, 3); ddv = ddv + ddv.permute(0, 1, 3, 2)
    ddv = 0.01 * (ddv + ddv.permute(2, 3, 0, 1))
    eps = 1e-4

    def E(hh, vv):
        r, ee, _, _ = ppq.pq_solve(H.occ_of_pair, H.vir_of_pair, hh.contiguous(), vv.contiguous(),
                                   H.e_const, **TIGHT)
        assert r == 0
        return ee
    fd = (E(H.h + eps * ddh, H.eri + eps * ddv) - E(H.h - eps * ddh, H.eri - eps * ddv)) / (2 * eps)
    an = float((dh * ddh).sum() + (dv * ddv).sum())
    assert abs(fd - an) < 1e-6, (fd, an)
    K = torch.randn((n, n), generator=g, device="cuda", dtype=torch.float64)
    K = 0.1 * (K - K.T)

    def rotated(sign):
        U = torch.linalg.matrix_exp(sign * eps * K)
        hh = U.T @ H.h @ U
        vv = torch.einsum('pqrs,pi->iqrs', H.eri, U)
        vv = torch.einsum('iqrs,qj->ijrs', vv, U)
        vv = torch.einsum('ijrs,rk->ijks', vv, U)
        return hh, torch.einsum('ijks,sl->ijkl', vv, U)
    fdk = (E(*rotated(1.0)) - E(*rotated(-1.0))) / (2 * eps)
    iu = torch.triu_indices(n, n, 1, device="cuda")
    ank = float((dk[iu[0], iu[1]] * K[iu[0], iu[1]]).sum())
    assert abs(fdk - ank) < 1e-6, (fdk, ank)
