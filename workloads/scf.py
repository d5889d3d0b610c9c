"""Closed-shell RHF, MO transform and occupied/virtual pairing.

The paper takes its orbitals and integrals from external programs (Implementation
section); this module is the synthetic stand-in: canonical RHF orbitals with a
deterministic phase, dense chemists'-notation MO integrals (pq|rs), and the
pairing of Fig. 1 -- the k-th highest occupied orbital with the k-th lowest
virtual (hole indices reversed).
"""
from dataclasses import dataclass, field
import numpy as np

from .ppp import polyene_geometry, acene_geometry, ppp_site_hamiltonian
from .hchain import hchain_ao_integrals


@dataclass
class Hamiltonian:
    """One active-space Hamiltonian in the MO basis (Hartree, chemists' notation)."""
    name: str
    h: np.ndarray            # [n, n] one-electron integrals
    eri: np.ndarray          # [n, n, n, n] (pq|rs)
    e_const: float           # constant energy (core-core / nuclear repulsion)
    occ_of_pair: np.ndarray  # [N] MO index of the occupied orbital of each pair
    vir_of_pair: np.ndarray  # [N] MO index of the virtual orbital of each pair
    mo_energy: np.ndarray = field(default=None)
    e_rhf: float = 0.0

    @property
    def n_orb(self):
        return self.h.shape[0]

    @property
    def n_pairs(self):
        return len(self.occ_of_pair)

    def min_orbital_gap(self):
        e = np.sort(self.mo_energy)
        return float(np.min(np.diff(e))) if len(e) > 1 else 0.0


def _fix_phase(C):
    C = C.copy()
    for k in range(C.shape[1]):
        i = int(np.argmax(np.abs(C[:, k]) + 1e-9 * np.arange(C.shape[0])[::-1]))
        if C[i, k] < 0:
            C[:, k] = -C[:, k]
    return C


def rhf(S, h, n_occ, jk, max_iter=500, tol=1e-11, diis_dim=8):
    """Closed-shell RHF with Pulay DIIS.  jk(P) returns (J, K) for the AO
    density P = 2 C_occ C_occ^T.  Returns (mo_energy, C, e_elec)."""
    s, U = np.linalg.eigh(S)
    X = U @ np.diag(s ** -0.5) @ U.T
    e, Cp = np.linalg.eigh(X.T @ h @ X)
    C = X @ Cp
    fs, es = [], []
    e_old = 0.0
    for it in range(max_iter):
        Co = C[:, :n_occ]
        P = 2.0 * Co @ Co.T
        J, K = jk(P)
        F = h + J - 0.5 * K
        e_elec = 0.5 * np.sum(P * (h + F))
        err = X.T @ (F @ P @ S - S @ P @ F) @ X
        fs.append(F); es.append(err)
        fs, es = fs[-diis_dim:], es[-diis_dim:]
        if len(fs) > 1:
            m = len(fs)
            B = -np.ones((m + 1, m + 1)); B[m, m] = 0.0
            for i in range(m):
                for j in range(m):
                    B[i, j] = np.sum(es[i] * es[j])
            rhs = np.zeros(m + 1); rhs[m] = -1.0
            coef = np.linalg.lstsq(B, rhs, rcond=None)[0][:m]
            F = sum(c * f for c, f in zip(coef, fs))
        e, Cp = np.linalg.eigh(X.T @ F @ X)
        C = X @ Cp
        if np.max(np.abs(err)) < tol and abs(e_elec - e_old) < tol:
            break
        e_old = e_elec
    Co = C[:, :n_occ]
    P = 2.0 * Co @ Co.T
    J, K = jk(P)
    F = h + J - 0.5 * K
    e, Cp = np.linalg.eigh(X.T @ F @ X)
    C = _fix_phase(X @ Cp)
    e_elec = 0.5 * np.sum(P * (h + F))
    return e, C, e_elec


def mo_integrals(C, h_ao, eri_ao=None, gamma_zdo=None):
    """(h_mo, eri_mo).  Either a dense AO ERI or a ZDO gamma matrix."""
    h_mo = C.T @ h_ao @ C
    if gamma_zdo is not None:
        n = C.shape[1]
        D = (C[:, :, None] * C[:, None, :]).reshape(C.shape[0], n * n)
        eri = (D.T @ gamma_zdo @ D).reshape(n, n, n, n)
    else:
        n = C.shape[1]
        t = np.tensordot(eri_ao, C, axes=([0], [0]))          # qrs i
        t = np.tensordot(t, C, axes=([0], [0]))               # rs i j
        t = np.tensordot(t, C, axes=([0], [0]))               # s i j k
        eri = np.tensordot(t, C, axes=([0], [0]))             # i j k l
    return h_mo, eri


def pair_orbitals(n_occ, n_pairs=None):
    """Fig. 1 pairing on energy-ordered MOs: pair k couples occupied orbital
    n_occ-1-k (k-th highest) with virtual n_occ+k (k-th lowest)."""
    N = n_occ if n_pairs is None else n_pairs
    occ = np.array([n_occ - 1 - k for k in range(N)], dtype=np.int32)
    vir = np.array([n_occ + k for k in range(N)], dtype=np.int32)
    return occ, vir


def build_ppp(kind, size, beta_ev=-2.4, u_ev=11.26, with_eri=True, orbitals="canonical"):
    """kind 'polyene' (size = number of sites) or 'acene' (size = rings).
    orbitals: 'canonical' (RHF, Fig. 1 energy pairing) or 'local' (Boys
    localised occupied and virtual orbitals, nearest-centroid pairing)."""
    if kind == 'polyene':
        xyz, bonds = polyene_geometry(size)
        name = f"PPP C{size}H{size + 2}"
    elif kind == 'acene':
        xyz, bonds = acene_geometry(size)
        name = f"PPP {size}-acene"
    else:
        raise ValueError(kind)
    h, gamma, e_const = ppp_site_hamiltonian(xyz, bonds, beta_ev, u_ev)
    n = h.shape[0]
    assert n % 2 == 0
    nocc = n // 2

    def jk(P):
        J = np.diag(gamma @ np.diag(P))
        K = P * gamma
        return J, K
    e, C, e_elec = rhf(np.eye(n), h, nocc, jk)
    occ, vir = pair_orbitals(nocc)
    if orbitals == "local":
        from .localize import localized_pairs
        C, occ, vir = localized_pairs(C, np.asarray(xyz), nocc)
        name += " (Boys-localised pairs)"
        P = 2.0 * C[:, occ] @ C[:, occ].T
        J, K = jk(P)
        e = np.diag(C.T @ (h + J - 0.5 * K) @ C)
    elif orbitals != "canonical":
        raise ValueError(orbitals)
    if with_eri:
        h_mo, eri = mo_integrals(C, h, gamma_zdo=gamma)
    else:
        h_mo, eri = C.T @ h @ C, None
    H = Hamiltonian(name, h_mo, eri, e_const, occ, vir, e, e_elec + e_const)
    H.C = C
    H.gamma_site = gamma
    return H


def ppp_cholesky_vectors(H):
    """Three-index factors B[Q, p, q] of a PPP workload with (pq|rs) =
    sum_Q B[Q,p,q] B[Q,r,s]: the site matrix gamma (zero differential overlap,
    positive definite for the Ohno form at these geometries) factored as
    gamma = L L^T, B[Q] = C^T diag(L[:, Q]) C -- one vector per site, exact."""
    L = np.linalg.cholesky(H.gamma_site)
    return np.ascontiguousarray(np.einsum('aq,ap,ar->qpr', L, H.C, H.C))


def cholesky_vectors(eri, tol=1e-12):
    """Pivoted (incomplete) Cholesky factors of the (pq),(rs) supermatrix of a
    real 8-fold symmetric (pq|rs): B[Q, p, q] with |(pq|rs) - sum_Q B B| <= tol
    on the diagonal, stopping once the largest remaining diagonal is below tol."""
    n = eri.shape[0]
    M = eri.reshape(n * n, n * n)
    d = np.diag(M).copy()
    vecs = []
    while True:
        k = int(np.argmax(d))
        if d[k] <= tol:
            break
        v = M[:, k].copy()
        for u in vecs:
            v -= u * u[k]
        v /= np.sqrt(d[k])
        vecs.append(v)
        d -= v * v
        d[k] = 0.0
    return np.ascontiguousarray(np.array(vecs).reshape(len(vecs), n, n))


def build_hchain(n_atoms, spacing_angstrom, orbitals="canonical", bond_bohr=None):
    """orbitals: 'canonical' (Fig. 1 energy pairing) or 'local' (Boys-localised
    occupied and virtual orbitals paired by nearest centroid, the stand-in
    for the paper's perfect-pairing orbitals of H50)."""
    S, h, eri, e_nuc = hchain_ao_integrals(n_atoms, spacing_angstrom, bond_bohr)
    nocc = n_atoms // 2

    def jk(P):
        n = P.shape[0]
        J = (eri.reshape(n * n, n * n) @ P.ravel()).reshape(n, n)
        K = (eri.transpose(0, 2, 1, 3).reshape(n * n, n * n) @ P.ravel()).reshape(n, n)
        return J, K
    e, C, e_elec = rhf(S, h, nocc, jk)
    occ, vir = pair_orbitals(nocc)
    name = f"H{n_atoms} d={spacing_angstrom:.3f}A" + (f" (H2 units, R={bond_bohr} bohr)" if bond_bohr else "")
    if orbitals == "local":
        from .localize import localized_pairs_general
        from .hchain import hchain_dipole_z
        C, occ, vir = localized_pairs_general(C, [hchain_dipole_z(n_atoms, spacing_angstrom, bond_bohr)], nocc)
        P = 2.0 * C[:, occ] @ C[:, occ].T
        J, K = jk(P)
        e = np.diag(C.T @ (h + J - 0.5 * K) @ C)
        name += " (Boys-localised pairs)"
    elif orbitals != "canonical":
        raise ValueError(orbitals)
    h_mo, eri_mo = mo_integrals(C, h, eri_ao=eri)
    return Hamiltonian(name, h_mo, eri_mo, e_nuc, occ, vir, e, e_elec + e_nuc)


def ppp_eri_device(H, torch):
    """MO two-electron integrals of a PPP workload (built with with_eri=False)
    on the current CUDA device: (pq|rs) = sum_{AB} D[A,pq] gamma[A,B] D[B,rs]
    with D[A,pq] = C[A,p] C[A,q] (zero differential overlap), as a contiguous
    float64 tensor of shape (n, n, n, n).  Keeps the n^4 array off the host."""
    C = torch.from_numpy(H.C).cuda()
    g = torch.from_numpy(H.gamma_site).cuda()
    n = C.shape[1]
    D = (C[:, :, None] * C[:, None, :]).reshape(C.shape[0], n * n)
    eri = (D.T @ g @ D).reshape(n, n, n, n).contiguous()
    del D
    return eri
