"""Energy gradients element by element against central differences (step
1e-4) of converged energies: the gradient recipe of the H50 configuration.

For each checked element the Hamiltonian is perturbed along one symmetric
class -- all copies of one (pq|rs) under the 8-fold symmetry, one symmetric
pair (h_pq, h_qp), or one orbital rotation C -> C exp(eps (E_pq - E_qp)) --
and (E(+eps) - E(-eps)) / (2 eps) is compared with the gradient summed over
the same copies (dE = sum_pqrs G_pqrs d(pq|rs) for symmetric changes).
Energies are GPU solves converged to ||R|| <= 1e-12 (their agreement with the
oracle is checked elsewhere); tolerance 1e-6.

* H10 (canonical orbitals, 1.4 A): every h class, 200 (pq|rs) classes chosen
  with seed 7, every occupied-virtual rotation and 50 occupied-occupied or
  virtual-virtual rotations;
* H50 (25 H2 units, R = 1.4 bohr, 1.8 A apart, localised pairs): 100 (pq|rs)
  classes, 50 occupied-virtual and 30 other rotations, seed 7.
"""
import itertools

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1609_00077_gb300 as ppq
from workloads import build_hchain

TIGHT = dict(r_tol=1e-12, e_tol=1e-14, max_iter=600)
EPS = 1e-4


def _copies(p, q, r, s):
    return sorted({(p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
                   (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)})


def _classes(n, count, rng):
    """count distinct symmetry classes of (pq|rs), drawn uniformly over index
    quadruples (seeded), each named by its smallest copy."""
    out = []
    seen = set()
    while len(out) < count:
        c = _copies(*(int(x) for x in rng.integers(0, n, size=4)))[0]
        if c not in seen:
            seen.add(c)
            out.append(c)
    return out


def _rot(h, eri, p, q, eps):
    n = h.shape[0]
    K = torch.zeros((n, n), dtype=torch.float64, device=h.device)
    K[p, q] = eps
    K[q, p] = -eps
    U = torch.linalg.matrix_exp(K)
    hh = U.T @ h @ U
    vv = torch.einsum('pqrs,pi->iqrs', eri, U)
    vv = torch.einsum('iqrs,qj->ijrs', vv, U)
    vv = torch.einsum('ijrs,rk->ijks', vv, U)
    return hh, torch.einsum('ijks,sl->ijkl', vv, U).contiguous()


def _check(H, h, eri, n_eri, n_ov, n_other, all_h):
    rng = np.random.default_rng(7)
    n = H.n_orb
    rc, e0, dh, dv, dk, _ = ppq.pq_gradient(H.occ_of_pair, H.vir_of_pair, h, eri, H.e_const, **TIGHT)
    assert rc == 0
    dh, dv, dk = dh.cpu().numpy(), dv.cpu().numpy(), dk.cpu().numpy()

    def E(hh, vv):
        r, ee, _, _ = ppq.pq_solve(H.occ_of_pair, H.vir_of_pair, hh, vv, H.e_const, **TIGHT)
        assert r == 0
        return ee
    worst = 0.0
    # (pq|rs) classes
    for cls in _classes(n, n_eri, rng):
        cp = _copies(*cls)
        idx = tuple(torch.tensor(x, device=eri.device) for x in zip(*cp))
        vp, vm = eri.clone(), eri.clone()
        vp[idx] += EPS
        vm[idx] -= EPS
        fd = (E(h, vp) - E(h, vm)) / (2 * EPS)
        an = sum(dv[c] for c in cp)
        worst = max(worst, abs(fd - an))
        assert abs(fd - an) < 1e-6, ("eri", cls, fd, an)
    # h classes
    hcls = [(p, q) for p in range(n) for q in range(p, n)]
    if not all_h:
        hcls = [hcls[i] for i in sorted(rng.choice(len(hcls), size=40, replace=False))]
    for p, q in hcls:
        hp, hm = h.clone(), h.clone()
        for a, b in {(p, q), (q, p)}:
            hp[a, b] += EPS
            hm[a, b] -= EPS
        fd = (E(hp, eri) - E(hm, eri)) / (2 * EPS)
        an = dh[p, q] + (dh[q, p] if p != q else 0.0)
        worst = max(worst, abs(fd - an))
        assert abs(fd - an) < 1e-6, ("h", p, q, fd, an)
    # orbital rotations
    occ, vir = list(H.occ_of_pair), list(H.vir_of_pair)
    ov = [(min(i, a), max(i, a)) for i in occ for a in vir]
    other = [(min(x), max(x)) for x in itertools.chain(itertools.combinations(occ, 2), itertools.combinations(vir, 2))]
    if n_ov < len(ov):
        ov = [ov[i] for i in sorted(rng.choice(len(ov), size=n_ov, replace=False))]
    other = [other[i] for i in sorted(rng.choice(len(other), size=min(n_other, len(other)), replace=False))]
    for p, q in ov + other:
        fd = (E(*_rot(h, eri, p, q, EPS)) - E(*_rot(h, eri, p, q, -EPS))) / (2 * EPS)
        worst = max(worst, abs(fd - dk[p, q]))
        assert abs(fd - dk[p, q]) < 1e-6, ("kappa", p, q, fd, dk[p, q])
    return worst


def test_elementwise_gradient_h10():
    H = build_hchain(10, 1.4)
    h = torch.from_numpy(H.h).cuda(); eri = torch.from_numpy(H.eri).cuda()
    _check(H, h, eri, n_eri=200, n_ov=10 ** 9, n_other=50, all_h=True)


def test_elementwise_gradient_h50():
    from workloads.hchain_torch import build_hchain_torch
    H = build_hchain_torch(50, 1.8, device="cuda", orbitals="local", bond_bohr=1.4)
    _check(H, H.h.contiguous(), H.eri.contiguous(), n_eri=100, n_ov=50, n_other=30, all_h=False)
