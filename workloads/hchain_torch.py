"""The H-chain workload of workloads.hchain built with torch on any device
(same closed-form s-Gaussian integrals, same RHF and pairing), for batches
of chains too large to generate with NumPy on the host."""
import math

import numpy as np

from .hchain import BOHR_PER_ANGSTROM, STO3G_EXPONENTS, STO3G_COEFFS, chain_positions
from .scf import Hamiltonian, pair_orbitals


def _boys0(t, torch):
    st = torch.sqrt(torch.clamp(t, min=1e-30))
    big = 0.5 * math.sqrt(math.pi) * torch.erf(st) / st
    return torch.where(t > 1e-12, big, 1.0 - t / 3.0)


def hchain_integrals_torch(n_atoms, spacing_angstrom, device="cuda", bond_bohr=None):
    import torch
    dt = torch.float64
    z = torch.tensor(chain_positions(n_atoms, spacing_angstrom, bond_bohr), dtype=dt, device=device)
    a = torch.tensor(STO3G_EXPONENTS, dtype=dt, device=device)
    c = torch.tensor(STO3G_COEFFS, dtype=dt, device=device) * (2.0 * a / math.pi) ** 0.75
    pab = a[:, None] + a[None, :]
    c = c / torch.sqrt((c[:, None] * c[None, :] * (math.pi / pab) ** 1.5).sum())
    A = z[:, None, None, None]; B = z[None, :, None, None]
    al = a[None, None, :, None]; be = a[None, None, None, :]
    p = al + be
    P = (al * A + be * B) / p
    kab = torch.exp(-al * be / p * (A - B) ** 2)
    cc = c[None, None, :, None] * c[None, None, None, :]
    S = (cc * (math.pi / p) ** 1.5 * kab).sum(dim=(2, 3))
    T = (cc * al * be / p * (3.0 - 2.0 * al * be / p * (A - B) ** 2) * (math.pi / p) ** 1.5 * kab).sum(dim=(2, 3))
    V = torch.zeros_like(S)
    for C in z:
        V = V - (cc * 2.0 * math.pi / p * kab * _boys0(p * (P - C) ** 2, torch)).sum(dim=(2, 3))
    n, k = n_atoms, len(STO3G_EXPONENTS)
    pf = (cc * kab).reshape(n, n, k * k)
    pp = p.expand(n, n, k, k).reshape(n, n, k * k)
    PP = P.reshape(n, n, k * k)
    eri = torch.zeros((n, n, n, n), dtype=dt, device=device)
    for u in range(k * k):
        p1 = pp[:, :, u][:, :, None, None]; P1 = PP[:, :, u][:, :, None, None]
        f1 = pf[:, :, u][:, :, None, None]
        for v in range(k * k):
            q1 = pp[:, :, v][None, None]; Q1 = PP[:, :, v][None, None]
            pre = 2.0 * math.pi ** 2.5 / (p1 * q1 * torch.sqrt(p1 + q1))
            eri += f1 * pf[:, :, v][None, None] * pre * _boys0(p1 * q1 / (p1 + q1) * (P1 - Q1) ** 2, torch)
    r = torch.abs(z[:, None] - z[None, :])
    iu = torch.triu_indices(n, n, 1, device=device)
    e_nuc = float((1.0 / r[iu[0], iu[1]]).sum())
    return S, T + V, eri, e_nuc


def build_hchain_torch(n_atoms, spacing_angstrom, device="cuda", max_iter=500, tol=1e-11, with_host=False,
                       orbitals="canonical", bond_bohr=None):
    """RHF + MO integrals on `device`.  Returns a Hamiltonian whose h / eri are
    torch tensors on the device (numpy copies when with_host)."""
    import torch
    S, h, eri, e_nuc = hchain_integrals_torch(n_atoms, spacing_angstrom, device, bond_bohr)
    n = n_atoms
    nocc = n // 2
    s, U = torch.linalg.eigh(S)
    X = U @ torch.diag(s ** -0.5) @ U.T
    Vm = eri.reshape(n * n, n * n)
    e, Cp = torch.linalg.eigh(X.T @ h @ X)
    C = X @ Cp
    fs, es = [], []
    e_old = 0.0
    for it in range(max_iter):
        Co = C[:, :nocc]
        Pm = 2.0 * Co @ Co.T
        J = (Vm @ Pm.reshape(-1)).reshape(n, n)
        K = (eri.permute(0, 2, 1, 3).reshape(n * n, n * n) @ Pm.reshape(-1)).reshape(n, n)
        F = h + J - 0.5 * K
        e_el = float(0.5 * (Pm * (h + F)).sum())
        err = X.T @ (F @ Pm @ S - S @ Pm @ F) @ X
        fs.append(F); es.append(err)
        fs, es = fs[-8:], es[-8:]
        if len(fs) > 1:
            m = len(fs)
            Bm = -torch.ones((m + 1, m + 1), dtype=h.dtype, device=device); Bm[m, m] = 0.0
            for i in range(m):
                for j in range(m):
                    Bm[i, j] = (es[i] * es[j]).sum()
            rhs = torch.zeros(m + 1, dtype=h.dtype, device=device); rhs[m] = -1.0
            coef = torch.linalg.lstsq(Bm.cpu(), rhs.cpu()).solution[:m].to(device)
            F = sum(cf * f for cf, f in zip(coef, fs))
        e, Cp = torch.linalg.eigh(X.T @ F @ X)
        C = X @ Cp
        if float(err.abs().max()) < tol and abs(e_el - e_old) < tol:
            break
        e_old = e_el
    Co = C[:, :nocc]
    Pm = 2.0 * Co @ Co.T
    J = (Vm @ Pm.reshape(-1)).reshape(n, n)
    K = (eri.permute(0, 2, 1, 3).reshape(n * n, n * n) @ Pm.reshape(-1)).reshape(n, n)
    F = h + J - 0.5 * K
    e, Cp = torch.linalg.eigh(X.T @ F @ X)
    C = X @ Cp
    # deterministic phase: largest component positive
    idx = torch.argmax(torch.abs(C) + 1e-9 * torch.arange(n, 0, -1, device=device, dtype=C.dtype)[:, None], dim=0)
    sgn = torch.sign(C[idx, torch.arange(n, device=device)])
    C = C * sgn[None, :]
    e_el = float(0.5 * (Pm * (h + F)).sum())
    occ, vir = pair_orbitals(nocc)
    name = f"H{n_atoms} d={spacing_angstrom:.3f}A" + (f" (H2 units, R={bond_bohr} bohr)" if bond_bohr else "")
    if orbitals == "local":
        from .localize import localized_pairs_general
        from .hchain import hchain_dipole_z
        Cn, occ, vir = localized_pairs_general(C.cpu().numpy(),
                                               [hchain_dipole_z(n_atoms, spacing_angstrom, bond_bohr)], nocc)
        C = torch.from_numpy(Cn).to(device)
        e = torch.diagonal(C.T @ F @ C)
        name += " (Boys-localised pairs)"
    h_mo = C.T @ h @ C
    eri_mo = torch.einsum('pqrs,pi->iqrs', eri, C)
    eri_mo = torch.einsum('iqrs,qj->ijrs', eri_mo, C)
    eri_mo = torch.einsum('ijrs,rk->ijks', eri_mo, C)
    eri_mo = torch.einsum('ijks,sl->ijkl', eri_mo, C).contiguous()
    Hm = Hamiltonian(name, h_mo, eri_mo, e_nuc, occ, vir, e.cpu().numpy(), e_el + e_nuc)
    if with_host:
        Hm.h_host = h_mo.cpu().numpy(); Hm.eri_host = eri_mo.cpu().numpy()
    return Hm
