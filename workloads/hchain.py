"""Linear hydrogen chains in an STO-3G-shaped s-Gaussian basis, shaped like the
paper's H50 case (Results).  Closed-form s-type integrals with the Boys F0
function; coordinates in bohr; returns AO (S, T+V, ERI, E_nuc)."""
import numpy as np
from scipy.special import erf

BOHR_PER_ANGSTROM = 1.8897261246
STO3G_EXPONENTS = np.array([3.42525, 0.62391, 0.16886])
STO3G_COEFFS = np.array([0.15433, 0.53533, 0.44463])


def _boys0(t):
    t = np.asarray(t, dtype=float)
    out = np.ones_like(t)
    big = t > 1e-12
    st = np.sqrt(t[big])
    out[big] = 0.5 * np.sqrt(np.pi) * erf(st) / st
    small = ~big
    out[small] = 1.0 - t[small] / 3.0
    return out


def chain_positions(n_atoms, spacing_angstrom, bond_bohr=None):
    """z coordinates (bohr).  Equidistant chain, or with bond_bohr the
    asymmetric chain of n/2 H2 units (bond bond_bohr, unit-to-unit gap
    spacing_angstrom) of the paper's asymmetric H50 dissociation."""
    d = spacing_angstrom * BOHR_PER_ANGSTROM
    if bond_bohr is None:
        return np.arange(n_atoms) * d
    k = np.arange(n_atoms) // 2
    return k * (bond_bohr + d) + (np.arange(n_atoms) % 2) * bond_bohr


def hchain_ao_integrals(n_atoms, spacing_angstrom, bond_bohr=None):
    return ao_integrals_at(chain_positions(n_atoms, spacing_angstrom, bond_bohr))


def ao_integrals_at(z):
    """(S, T+V, ERI, E_nuc) for hydrogen atoms at the z coordinates z (bohr)
    on one line, one contracted s function each."""
    z = np.asarray(z, dtype=float)
    a = STO3G_EXPONENTS
    c = STO3G_COEFFS * (2.0 * a / np.pi) ** 0.75
    # renormalise the contraction exactly
    pab = a[:, None] + a[None, :]
    s_self = (c[:, None] * c[None, :] * (np.pi / pab) ** 1.5).sum()
    c = c / np.sqrt(s_self)
    n, k = len(z), len(a)
    # primitive pair quantities for every AO pair (mu, nu) and primitives (i, j)
    A = z[:, None, None, None]; B = z[None, :, None, None]
    al = a[None, None, :, None]; be = a[None, None, None, :]
    p = al + be
    P = (al * A + be * B) / p
    kab = np.exp(-al * be / p * (A - B) ** 2)
    cc = c[None, None, :, None] * c[None, None, None, :]
    S = (cc * (np.pi / p) ** 1.5 * kab).sum(axis=(2, 3))
    T = (cc * al * be / p * (3.0 - 2.0 * al * be / p * (A - B) ** 2)
         * (np.pi / p) ** 1.5 * kab).sum(axis=(2, 3))
    V = np.zeros((n, n))
    for C in z:
        V -= (cc * 2.0 * np.pi / p * kab * _boys0(p * (P - C) ** 2)).sum(axis=(2, 3))
    # ERI over AO quadruples, summed over primitive quadruples
    pf = (cc * kab).reshape(n, n, k * k)
    pp = p.reshape(1, 1, k * k) * np.ones((n, n, 1))
    PP = P.reshape(n, n, k * k)
    eri = np.zeros((n, n, n, n))
    for u in range(k * k):
        for v in range(k * k):
            p1 = pp[:, :, u][:, :, None, None]; q1 = pp[:, :, v][None, None, :, :]
            P1 = PP[:, :, u][:, :, None, None]; Q1 = PP[:, :, v][None, None, :, :]
            pre = 2.0 * np.pi ** 2.5 / (p1 * q1 * np.sqrt(p1 + q1))
            eri += (pf[:, :, u][:, :, None, None] * pf[:, :, v][None, None, :, :]
                    * pre * _boys0(p1 * q1 / (p1 + q1) * (P1 - Q1) ** 2))
    r = np.abs(z[:, None] - z[None, :])
    e_nuc = sum(1.0 / r[i, j] for i in range(n) for j in range(i + 1, n))
    return S, T + V, eri, e_nuc


def hchain_dipole_z(n_atoms, spacing_angstrom, bond_bohr=None):
    """AO matrix of the z coordinate, <mu| z |nu> (s functions: the product
    centre times the primitive overlap)."""
    z = chain_positions(n_atoms, spacing_angstrom, bond_bohr)
    a = STO3G_EXPONENTS
    c = STO3G_COEFFS * (2.0 * a / np.pi) ** 0.75
    pab = a[:, None] + a[None, :]
    c = c / np.sqrt((c[:, None] * c[None, :] * (np.pi / pab) ** 1.5).sum())
    A = z[:, None, None, None]; B = z[None, :, None, None]
    al = a[None, None, :, None]; be = a[None, None, None, :]
    p = al + be
    P = (al * A + be * B) / p
    kab = np.exp(-al * be / p * (A - B) ** 2)
    cc = c[None, None, :, None] * c[None, None, None, :]
    return (cc * (np.pi / p) ** 1.5 * kab * P).sum(axis=(2, 3))
