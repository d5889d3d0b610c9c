"""Pariser-Parr-Pople pi-space models shaped like the paper's polyene and
polyacene cases (Results, Tables VI and VII).

Conventions (not fixed by the paper; they define the synthetic workloads):
zero-differential-overlap site basis, (ii|jj) = gamma_ij with gamma_ii = U,
Ohno gamma_ij = U / sqrt(1 + (U r_ij / 14.397)^2) eV (r in Angstrom),
h_ij = beta on bonded sites, h_ii = -sum_{j != i} gamma_ij (one neutral core
per site), core-core repulsion e_const = sum_{i<j} gamma_ij.  Energies are
returned in Hartree.
"""
import numpy as np

EV_PER_HARTREE = 27.211386245988
OHNO_EV_ANGSTROM = 14.397


def polyene_geometry(n_sites, short=1.35, long=1.46):
    """All-trans zigzag chain, 120 degree angles, bonds alternating short/long
    starting with a short bond at the chain end.  Returns (xyz[n,2], bonds)."""
    xyz = np.zeros((n_sites, 2))
    bonds = []
    for k in range(n_sites - 1):
        theta = np.deg2rad(30.0 if k % 2 == 0 else -30.0)
        b = short if k % 2 == 0 else long
        xyz[k + 1] = xyz[k] + b * np.array([np.cos(theta), np.sin(theta)])
        bonds.append((k, k + 1))
    return xyz, bonds


def acene_geometry(n_rings, cc=1.40):
    """Linear acene of n_rings fused hexagons (4 n_rings + 2 sites), C-C = cc.
    Sites are ordered by x then y so the numbering is deterministic."""
    pts = []
    for k in range(n_rings):
        cx = k * np.sqrt(3.0) * cc
        for j in range(6):
            ang = np.deg2rad(30.0 + 60.0 * j)
            pts.append((cx + cc * np.cos(ang), cc * np.sin(ang)))
    pts = np.round(np.array(pts), 6)
    uniq = []
    for p in pts:
        if not any(np.linalg.norm(p - q) < 1e-4 for q in uniq):
            uniq.append(p)
    uniq = sorted(uniq, key=lambda p: (round(p[0], 4), round(p[1], 4)))
    xyz = np.array(uniq)
    n = len(xyz)
    bonds = [(i, j) for i in range(n) for j in range(i + 1, n)
             if abs(np.linalg.norm(xyz[i] - xyz[j]) - cc) < 1e-3]
    assert n == 4 * n_rings + 2, n
    return xyz, bonds


def ppp_site_hamiltonian(xyz, bonds, beta_ev=-2.4, u_ev=11.26):
    """Site-basis PPP Hamiltonian in Hartree: (h[n,n], gamma[n,n], e_const)."""
    n = len(xyz)
    r = np.linalg.norm(xyz[:, None, :] - xyz[None, :, :], axis=-1)
    gamma = u_ev / np.sqrt(1.0 + (u_ev * r / OHNO_EV_ANGSTROM) ** 2)
    h = np.zeros((n, n))
    for i, j in bonds:
        h[i, j] = h[j, i] = beta_ev
    off = gamma - np.diag(np.diag(gamma))
    h[np.diag_indices(n)] = -off.sum(axis=1)
    e_const = 0.5 * off.sum()
    return h / EV_PER_HARTREE, gamma / EV_PER_HARTREE, e_const / EV_PER_HARTREE
