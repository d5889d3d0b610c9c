"""O-det: the PQ / PH amplitude equations evaluated exactly in the full
determinant space (test infrastructure only; see the package header).

Method (Theory section): the amplitudes are those CC excitations whose holes
and particles carry at most K distinct pairing labels (K = 2 for PQ, the
CCSDTQ truncation to two pairs; K = 3 for PH, CCSDTQ56 truncated to three
pairs), labels assigned by the pairing of Fig. 1.  The two-electron integrals
are truncated to at most K_H labels (Table I; Implementation section, where the
integral truncation is controlled separately from the amplitudes); the Fock
operator is the full one.  The projected equations are

    R_mu = <mu| exp(-T) (F_N + W_N^(K_H)) exp(T) |Phi> = 0,   mu in M_K,

evaluated with no truncation of intermediates, and the correlation energy is
<Phi| exp(-T) H_N exp(T) |Phi> (Eq. Ec for its doubles part).  The normal-ordered
Hamiltonian is rebuilt in bare form, h' = f - sum_i [2 v'(pq|ii) - v'(pi|iq)]
with v' the truncated integrals, so that normal ordering h', v' gives back the
full Fock matrix and the truncated W_N.

Amplitude convention: t_D multiplies the excitation operator tau_D that maps the
reference to +|D> in the determinant basis of ``fci.Strings``.
"""
from itertools import combinations
import numpy as np

from .fci import Strings, sigma


def label_of_orbital(n_orb, occ_of_pair, vir_of_pair):
    lab = -np.ones(n_orb, dtype=np.int64)
    for k, (i, a) in enumerate(zip(occ_of_pair, vir_of_pair)):
        lab[i] = k
        lab[a] = k
    if np.any(lab < 0):
        raise ValueError("every active orbital must belong to a pair")
    return lab


def truncated_hamiltonian(h, eri, occ_of_pair, vir_of_pair, K_H):
    """Bare (h', v') whose normal-ordered form is F_N + W_N^(K_H), plus the
    full Fock matrix f and the reference energy without constant.

    K_H = -1 keeps every integral.  f_pq = h_pq + sum_i [2(pq|ii) - (pi|iq)]."""
    n = h.shape[0]
    lab = label_of_orbital(n, occ_of_pair, vir_of_pair)
    occ = np.asarray(occ_of_pair)
    if K_H < 0:
        vt = eri.copy()
    else:
        # number of distinct labels of each index quadruple (p, q, r, s)
        La = lab[:, None, None, None]; Lb = lab[None, :, None, None]
        Lc = lab[None, None, :, None]; Ld = lab[None, None, None, :]
        nl = (1 + (Lb != La).astype(np.int8) + ((Lc != La) & (Lc != Lb)).astype(np.int8)
              + ((Ld != La) & (Ld != Lb) & (Ld != Lc)).astype(np.int8))
        vt = np.where(nl <= K_H, eri, 0.0)
        del nl
    f = h + 2.0 * eri[:, :, occ, occ].sum(-1) - eri[:, occ, occ, :].sum(1)
    hp = f - 2.0 * vt[:, :, occ, occ].sum(-1) + vt[:, occ, occ, :].sum(1)
    e_ref = float(np.sum(h[occ, occ]) + np.sum(f[occ, occ]))
    return hp, vt, f, e_ref


def enumerate_manifold(occ_of_pair, vir_of_pair, K, max_rank=0):
    """All M_s-conserving excitations whose orbitals span 1..K pair labels.
    Each is (a_holes, a_parts, b_holes, b_parts) as sorted spatial indices.
    max_rank > 0 keeps only excitations of at most that many electrons (the
    Conclusions section: higher excitations disabled, e.g. PH with singles and
    doubles only)."""
    N = len(occ_of_pair)
    out = []
    for m in range(1, min(K, N) + 1):
        for Lset in combinations(range(N), m):
            occL = sorted(int(occ_of_pair[k]) for k in Lset)
            virL = sorted(int(vir_of_pair[k]) for k in Lset)
            lab = {int(occ_of_pair[k]): k for k in Lset}
            lab.update({int(vir_of_pair[k]): k for k in Lset})
            sides = []
            for r in range(m + 1):
                for hs in combinations(occL, r):
                    for ps in combinations(virL, r):
                        sides.append((hs, ps))
            for ah, ap in sides:
                for bh, bp in sides:
                    if not (ah or bh):
                        continue
                    if max_rank and len(ah) + len(bh) > max_rank:
                        continue
                    labs = {lab[x] for x in ah + ap + bh + bp}
                    if len(labs) == m:
                        out.append((ah, ap, bh, bp))
    return out


def _side_ops(holes, parts):
    """a+_{p1} ... a+_{pk} a_{hk} ... a_{h1} as an ops list (applied right to left)."""
    return [(p, 1) for p in parts] + [(h, 0) for h in reversed(holes)]


class DetCC:
    """Determinant-space evaluator of the truncated-CC residual for one system."""

    def __init__(self, n_orb, occ_of_pair, vir_of_pair, K, manifold=None):
        self.n_orb = n_orb
        self.occ = np.asarray(occ_of_pair)
        self.vir = np.asarray(vir_of_pair)
        self.N = len(self.occ)
        self.K = K
        self.S = Strings(n_orb, self.N)
        self.ref = sum(1 << int(i) for i in self.occ)
        self.iref = self.S.index[self.ref]
        self.manifold = enumerate_manifold(self.occ, self.vir, K) if manifold is None else manifold
        self.index = {d: k for k, d in enumerate(self.manifold)}
        cache = {}

        def side(holes, parts):
            key = (holes, parts)
            if key not in cache:
                ops = _side_ops(holes, parts)
                t, g = Strings.apply(self.ref, ops)
                src, dst, sg = self.S.op_map(ops)
                cache[key] = (src, dst, sg * g, self.S.index[t])
            return cache[key]
        self.ops = []
        for (ah, ap, bh, bp) in self.manifold:
            self.ops.append((side(ah, ap), side(bh, bp)))
        self.det_alpha = np.array([o[0][3] for o in self.ops], dtype=np.int64)
        self.det_beta = np.array([o[1][3] for o in self.ops], dtype=np.int64)

    @property
    def n_amp(self):
        return len(self.manifold)

    def apply_T(self, t, v):
        out = np.zeros(v.shape, dtype=np.result_type(v, np.asarray(t)))
        for tk, ((sa, da, ga, _), (sb, db, gb, _)) in zip(t, self.ops):
            if tk == 0.0 or len(sa) == 0 or len(sb) == 0:
                continue
            out[np.ix_(da, db)] += tk * (ga[:, None] * gb[None, :]) * v[np.ix_(sa, sb)]
        return out

    def exp_T(self, t, v):
        out = v.astype(np.result_type(v, np.asarray(t)))
        term = v
        for k in range(1, 4 * self.N + 2):
            term = self.apply_T(t, term) / k
            if not np.any(term):
                break
            out += term
        return out

    def ref_vector(self, dtype=float):
        v = np.zeros((self.S.n, self.S.n), dtype=dtype)
        v[self.iref, self.iref] = 1.0
        return v

    def transformed(self, t, h1, v2):
        """exp(-T) H exp(T) |Phi> as a determinant-space vector (bare H = h1, v2).
        Complex amplitudes are allowed (complex-step derivatives)."""
        t = np.asarray(t)
        psi = self.exp_T(t, self.ref_vector(t.dtype if np.iscomplexobj(t) else float))
        phi = sigma(self.S, h1, v2, psi)
        return self.exp_T(-np.asarray(t), phi)

    def residual(self, t, h1, v2):
        """(R over the manifold, <Phi|exp(-T) H exp(T)|Phi>) for the bare H."""
        chi = self.transformed(t, h1, v2)
        e = chi[self.iref, self.iref]
        return chi[self.det_alpha, self.det_beta].copy(), (e if np.iscomplexobj(chi) else float(e))

    def reference_energy(self, h1, v2):
        return self.residual(np.zeros(self.n_amp), h1, v2)[1]

    def denominators(self, f, level_shift=0.0):
        """D_mu = sum of hole Fock diagonals - sum of particle Fock diagonals."""
        d = np.empty(self.n_amp)
        fd = np.diag(f)
        for k, (ah, ap, bh, bp) in enumerate(self.manifold):
            d[k] = sum(fd[list(ah + bh)]) - sum(fd[list(ap + bp)]) - level_shift
        return d


class Problem:
    """A PQ/PH problem: Hamiltonian + pairing + truncation, with residual,
    energy and the Jacobi/DIIS solver of the amplitude equations."""

    def __init__(self, h, eri, occ_of_pair, vir_of_pair, K, K_H=0, e_const=0.0, max_rank=0):
        self.K = K
        self.K_H = K if K_H == 0 else K_H
        self.hp, self.vt, self.f, e_ref = truncated_hamiltonian(
            h, eri, occ_of_pair, vir_of_pair, self.K_H)
        self.e_ref = e_ref + e_const
        man = enumerate_manifold(occ_of_pair, vir_of_pair, K, max_rank) if max_rank else None
        self.cc = DetCC(h.shape[0], occ_of_pair, vir_of_pair, K, manifold=man)
        self.e_ref_bare = self.cc.reference_energy(self.hp, self.vt)

    def residual(self, t):
        """(R, E_c) at amplitudes t."""
        R, e = self.cc.residual(t, self.hp, self.vt)
        return R, e - self.e_ref_bare

    def solve(self, **kw):
        return jacobi_diis(self.residual, self.cc.denominators(self.f, kw.pop('level_shift', 0.0)),
                           self.cc.n_amp, **kw)


def jacobi_diis(residual, denom, n_amp, t0=None, r_tol=1e-10, e_tol=1e-12,
                max_iter=200, diis_dim=8, diis_start=3):
    """Jacobi update t <- t + R/D with Pulay DIIS on the update vectors
    (Implementation section: denominators and DIIS; subspace size, start and
    error vector are not given in the paper and take the values above).

    Returns dict(t, e_corr, res_norm, iters, converged, history)."""
    t = np.zeros(n_amp) if t0 is None else np.array(t0, dtype=float)
    ts, es = [], []
    e_old = None
    hist = []
    for it in range(1, max_iter + 1):
        R, e = residual(t)
        rn = float(np.linalg.norm(R))
        hist.append((e, rn))
        if e_old is not None and rn <= r_tol and abs(e - e_old) <= e_tol:
            return dict(t=t, e_corr=e, res_norm=rn, iters=it, converged=True, history=hist)
        if not np.isfinite(rn) or rn > 1e6:
            return dict(t=t, e_corr=e, res_norm=rn, iters=it, converged=False, history=hist)
        e_old = e
        t_new = t + R / denom
        ts.append(t_new); es.append(t_new - t)
        ts, es = ts[-diis_dim:], es[-diis_dim:]
        if it >= diis_start and len(ts) > 1:
            t_new = diis_extrapolate(ts, es)
        t = t_new
    R, e = residual(t)
    return dict(t=t, e_corr=e, res_norm=float(np.linalg.norm(R)), iters=max_iter,
                converged=False, history=hist)


def diis_extrapolate(ts, es):
    """Pulay extrapolation: minimise |sum c_i e_i| subject to sum c_i = 1."""
    m = len(ts)
    B = np.empty((m + 1, m + 1))
    for i in range(m):
        for j in range(m):
            B[i, j] = np.dot(es[i], es[j])
    # scaling the error block leaves c unchanged (the multiplier absorbs it)
    # but keeps lstsq from treating a block of tiny dot products as zero
    sc = np.max(np.abs(np.diag(B[:m, :m])))
    if sc > 0.0:
        B[:m, :m] /= sc
    B[m, :] = -1.0; B[:, m] = -1.0; B[m, m] = 0.0
    rhs = np.zeros(m + 1); rhs[m] = -1.0
    c = np.linalg.lstsq(B, rhs, rcond=None)[0][:m]
    return sum(ci * ti for ci, ti in zip(c, ts))
