"""Localised orbitals with matching virtuals, the stand-in for the paper's
Pipek-Mezey occupied orbitals paired with Sano virtuals (Implementation
section; Table VI caption).

Foster-Boys localisation (maximise sum_i |<i|r|i>|^2) by Jacobi sweeps, done
separately in the occupied and the virtual space of an orthonormal site basis
with site positions r_s (ZDO: <s|r|t> = delta_st r_s).  Each localised
occupied orbital is paired with the localised virtual whose centroid is
nearest (optimal assignment), and pairs are ordered along the molecule.
"""
import numpy as np
from scipy.optimize import linear_sum_assignment


def boys(C, pos, sweeps=200, tol=1e-12):
    """Rotate the columns of C (sites x orbitals) to maximise the Boys
    functional for site positions pos (sites x dim)."""
    C = C.copy()
    m = C.shape[1]
    dim = pos.shape[1]
    for _ in range(sweeps):
        change = 0.0
        for i in range(m):
            for j in range(i + 1, m):
                ci, cj = C[:, i], C[:, j]
                rii = (ci * ci) @ pos; rjj = (cj * cj) @ pos; rij = (ci * cj) @ pos
                A = rij @ rij - 0.25 * (rii - rjj) @ (rii - rjj)
                B = rij @ (rii - rjj)
                if abs(A) < 1e-14 and abs(B) < 1e-14:
                    continue
                theta = 0.25 * np.arctan2(B, -A)
                if abs(theta) < tol:
                    continue
                c, s = np.cos(theta), np.sin(theta)
                C[:, i], C[:, j] = c * ci + s * cj, -s * ci + c * cj
                change = max(change, abs(theta))
        if change < 1e-10:
            break
    return C


def localized_pairs(C, pos, n_occ):
    """(C_new, occ_of_pair, vir_of_pair): Boys-localised occupied and virtual
    orbitals, each occupied paired with the nearest virtual."""
    Co = boys(C[:, :n_occ], pos)
    Cv = boys(C[:, n_occ:], pos)
    ro = np.array([(Co[:, i] ** 2) @ pos for i in range(Co.shape[1])])
    rv = np.array([(Cv[:, a] ** 2) @ pos for a in range(Cv.shape[1])])
    cost = np.linalg.norm(ro[:, None, :] - rv[None, :, :], axis=-1)
    oi, vi = linear_sum_assignment(cost)
    order = np.lexsort(tuple(ro[oi, d] for d in reversed(range(pos.shape[1]))))
    oi, vi = oi[order], vi[order]
    Cn = np.concatenate([Co[:, oi], Cv[:, vi]], axis=1)
    for k in range(Cn.shape[1]):
        j = int(np.argmax(np.abs(Cn[:, k])))
        if Cn[j, k] < 0:
            Cn[:, k] = -Cn[:, k]
    N = len(oi)
    occ = np.arange(N, dtype=np.int32)
    vir = np.arange(N, 2 * N, dtype=np.int32)
    return Cn, occ, vir


def boys_general(C, Zs, sweeps=300):
    """Boys localisation for a general (non-diagonal) position operator.
    C: AO coefficients (ao x m); Zs: list of AO matrices of the Cartesian
    position components.  Returns (C_rotated, centroids[m, dim])."""
    C = C.copy()
    m = C.shape[1]
    R = [C.T @ Z @ C for Z in Zs]
    for _ in range(sweeps):
        change = 0.0
        for i in range(m):
            for j in range(i + 1, m):
                A = sum(r[i, j] ** 2 - 0.25 * (r[i, i] - r[j, j]) ** 2 for r in R)
                B = sum(r[i, j] * (r[i, i] - r[j, j]) for r in R)
                if abs(A) < 1e-14 and abs(B) < 1e-14:
                    continue
                th = 0.25 * np.arctan2(B, -A)
                if abs(th) < 1e-13:
                    continue
                c, s = np.cos(th), np.sin(th)
                ci, cj = C[:, i].copy(), C[:, j].copy()
                C[:, i], C[:, j] = c * ci + s * cj, -s * ci + c * cj
                for r in R:
                    ri, rj = r[i, :].copy(), r[j, :].copy()
                    r[i, :], r[j, :] = c * ri + s * rj, -s * ri + c * rj
                    ci_, cj_ = r[:, i].copy(), r[:, j].copy()
                    r[:, i], r[:, j] = c * ci_ + s * cj_, -s * ci_ + c * cj_
                change = max(change, abs(th))
        if change < 1e-10:
            break
    cent = np.array([[r[k, k] for r in R] for k in range(m)])
    return C, cent


def localized_pairs_general(C, Zs, n_occ):
    """Boys-localised occupied and virtual orbitals (general position
    operator), each occupied paired with the nearest virtual centroid, pairs
    ordered along the first coordinate.  Returns (C_new, occ, vir)."""
    Co, ro = boys_general(C[:, :n_occ], Zs)
    Cv, rv = boys_general(C[:, n_occ:], Zs)
    cost = np.linalg.norm(ro[:, None, :] - rv[None, :, :], axis=-1)
    oi, vi = linear_sum_assignment(cost)
    order = np.lexsort(tuple(ro[oi, d] for d in reversed(range(ro.shape[1]))))
    oi, vi = oi[order], vi[order]
    Cn = np.concatenate([Co[:, oi], Cv[:, vi]], axis=1)
    for k in range(Cn.shape[1]):
        j = int(np.argmax(np.abs(Cn[:, k])))
        if Cn[j, k] < 0:
            Cn[:, k] = -Cn[:, k]
    N = len(oi)
    return Cn, np.arange(N, dtype=np.int32), np.arange(N, 2 * N, dtype=np.int32)
