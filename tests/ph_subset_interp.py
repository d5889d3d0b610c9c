"""CPU interpreter of the label-subset expansion tables (test infrastructure).

The PH kernels evaluate the residual from structure tables that the library
generates natively (``ph_tables_counts`` / ``ph_tables_copy``): per subset
size k, the zero-charge sector of k sites, the recursion of exp(T)|ref>, the
Hamiltonian rows of the outputs and the back-substitution with exp(-T).  This
module reads those tables through the C ABI and interprets them with numpy the
way the kernels use them:

    psi(s)    = sum_e sign_e t[slot_e] psi(sub_e)              (levels in order)
    phi(o)    = sum_e c_e v[key_e] psi(s_e) + (D_o - E_0) psi(state(o)),
                D_o = <o|H|o> and E_0 = <ref|H|ref> of the local problem
    R_loc(mu) = sum_e sign_e psi_minus(w_e) phi(kappa_e)
    R_mu      = sum over subsets L containing labels(mu), |L| <= K + K_H, of
                c_|L| R_loc^(L)(mu),  c_k = sum_j (-1)^j C(N - k, j), j <= K + K_H - k
    E_c       = sum over |L| <= K_H of c^E_|L| phi^(L)(ref)

so that a test can hold the generated tables against the oracle on the CPU,
before and independently of the GPU kernels.  The integrals are gathered here
from their definitions (the site, pair and triple keys of ``tables``).
"""
import ctypes
import itertools
from math import comb

import numpy as np

import paper_1609_00077_gb300 as ppq
from paper_1609_00077_gb300 import tables as T
from tests.ph_decomposition import bare_truncated_hamiltonian

NAMES = ["code", "lvl_ptr", "ent_ptr", "ent_sub", "ent_slot", "slot_desc", "out_state", "out_desc",
         "olvl_ptr", "olvl_order", "oent_ptr", "oent_sub", "oent_slot", "key_desc", "h_ptr", "h_s",
         "h_key", "h_c", "e0_key", "e0_c", "b_ptr", "b_k", "b_w", "d_ptr", "d_key", "d_c",
         "bs_ptr", "bs_ent", "bl_ptr", "bl_ent", "obs_ptr", "obs_ent", "obl_ptr", "obl_ent", "hs_ptr", "hs_ent",
         "hk_ptr", "hk_ent", "dk_ptr", "dk_out", "dk_c", "e0_by_key", "bk_ptr", "bk_ent", "bw_ptr", "bw_ent",
         "out_of_state"]
DTYPES = {"code": np.uint32, "ent_slot": np.int16, "oent_slot": np.int16, "h_key": np.int16,
          "e0_key": np.int16, "h_c": np.float64, "e0_c": np.float64, "d_key": np.int16, "d_c": np.float64,
          "bs_ent": np.uint64, "bl_ent": np.uint64, "obs_ent": np.uint64, "obl_ent": np.uint64,
          "hs_ent": np.uint32, "hk_ent": np.uint64, "dk_c": np.float64, "e0_by_key": np.float64,
          "bk_ent": np.uint32, "bw_ent": np.uint32}

_CACHE = {}


def tables(k, K, K_H):
    key = (k, K, K_H)
    if key not in _CACHE:
        L = ppq.lib()
        L.ph_tables_counts.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p]
        L.ph_tables_copy.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p]
        cnt = np.zeros(48, dtype=np.int64)
        rc = L.ph_tables_counts(k, K, K_H, cnt.ctypes.data)
        if rc != 0:
            raise ppq.PPQError(ppq.lib().ppq_last_error().decode())
        out = {}
        for i, name in enumerate(NAMES):
            a = np.zeros(int(cnt[i]), dtype=DTYPES.get(name, np.int32))
            if len(a):
                assert L.ph_tables_copy(k, K, K_H, i, a.ctypes.data) == 0
            out[name] = a
        _CACHE[key] = out
    return _CACHE[key]


def unpack(d):
    m = d & 15
    pos = [(d >> (4 + 4 * i)) & 15 for i in range(m)]
    return m, pos, d >> 20


def moebius(N, k, kmax):
    return sum((-1) ** j * comb(N - k, j) for j in range(0, kmax - k + 1))


class SubsetInterp:
    """Residual of the K-pair model (K = 2 or 3) with integrals truncated to
    K_H labels (K_H = 4: untruncated), from the generated tables."""

    def __init__(self, h, eri, occ, vir, K, K_H):
        self.occ = [int(i) for i in occ]
        self.vir = [int(a) for a in vir]
        self.N = N = len(self.occ)
        self.K, self.K_H = K, K_H
        hp, v, _ = bare_truncated_hamiltonian(h, eri, np.array(self.occ), np.array(self.vir), K_H)
        self.keys = {1: T.site_integral_keys(), 2: T.pair_integral_keys(), 3: T.triple_integral_keys(),
                     4: T.quad_integral_keys()}
        self.nch = {1: 3, 2: 29, 3: 303}
        self.hp, self.v = hp, v

    def integral(self, labels, j):
        orbs = []
        for X in labels:
            orbs += [self.occ[X], self.vir[X]]
        key = self.keys[len(labels)][j]
        if key[0] == "h":
            return self.hp[orbs[key[1]], orbs[key[2]]]
        return self.v[orbs[key[1]], orbs[key[2]], orbs[key[3]], orbs[key[4]]]

    def amp(self, t, labels, ch):
        N = self.N
        m = len(labels)
        if m == 1:
            return t[3 * labels[0] + ch]
        if m == 2:
            return t[3 * N + (labels[0] * N + labels[1]) * 29 + ch]
        return t[3 * N + 29 * N * N + ((labels[0] * N + labels[1]) * N + labels[2]) * 303 + ch]

    def slot_of(self, labels, ch):
        N = self.N
        m = len(labels)
        if m == 1:
            return 3 * labels[0] + ch
        if m == 2:
            return 3 * N + (labels[0] * N + labels[1]) * 29 + ch
        return 3 * N + 29 * N * N + ((labels[0] * N + labels[1]) * N + labels[2]) * 303 + ch

    def local(self, Tb, Lset, t, sign_flip_control=False):
        """(R over the outputs, phi(ref)) of the problem restricted to Lset."""
        tl = np.array([self.amp(t, [Lset[p] for p in unpack(d)[1]], unpack(d)[2]) for d in Tb["slot_desc"]])
        sg = np.where(Tb["ent_slot"] & 1, -1.0, 1.0)
        if sign_flip_control:
            sg = np.abs(sg)
        slot = Tb["ent_slot"].astype(np.int64) >> 1
        w = sg * tl[slot]
        psi = np.zeros(len(Tb["code"]))
        psi[0] = 1.0
        lp, ep = Tb["lvl_ptr"], Tb["ent_ptr"]
        for lv in range(1, len(lp) - 1):
            s0, s1 = lp[lv], lp[lv + 1]
            e0, e1 = ep[s0], ep[s1]
            contrib = w[e0:e1] * psi[Tb["ent_sub"][e0:e1]]
            owner = np.repeat(np.arange(s0, s1), np.diff(ep[s0:s1 + 1]))
            psi[s0:s1] = np.bincount(owner - s0, weights=contrib, minlength=s1 - s0)
        vl = np.array([self.integral([Lset[p] for p in unpack(d)[1]], unpack(d)[2]) for d in Tb["key_desc"]])
        E0 = float(np.sum(Tb["e0_c"] * vl[Tb["e0_key"]]))
        hp = Tb["h_ptr"]
        owner = np.repeat(np.arange(len(hp) - 1), np.diff(hp))
        phi = np.bincount(owner, weights=Tb["h_c"] * vl[Tb["h_key"]] * psi[Tb["h_s"]], minlength=len(hp) - 1)
        dp = Tb["d_ptr"]
        downer = np.repeat(np.arange(len(dp) - 1), np.diff(dp))
        diag = np.bincount(downer, weights=Tb["d_c"] * vl[Tb["d_key"]], minlength=len(dp) - 1)
        phi += (diag - E0) * psi[Tb["out_state"]]
        # exp(-T) on the outputs
        nout = len(Tb["out_state"])
        pm = np.zeros(nout)
        pm[0] = 1.0
        osg = np.where(Tb["oent_slot"] & 1, -1.0, 1.0) * -tl[Tb["oent_slot"].astype(np.int64) >> 1]
        order, olp, oep = Tb["olvl_order"], Tb["olvl_ptr"], Tb["oent_ptr"]
        for lv in range(1, len(olp) - 1):
            for i in range(olp[lv], olp[lv + 1]):
                e0, e1 = oep[i], oep[i + 1]
                pm[order[i]] = np.sum(osg[e0:e1] * pm[Tb["oent_sub"][e0:e1]])
        bp = Tb["b_ptr"]
        owner = np.repeat(np.arange(nout), np.diff(bp))
        bsg = np.where(Tb["b_w"] & 1, -1.0, 1.0)
        R = np.bincount(owner, weights=bsg * pm[Tb["b_w"] >> 1] * phi[Tb["b_k"]], minlength=nout)
        return R, phi[0]

    def residual(self, t, kmax=None, **kw):
        """(R in the K = 3 (or 2) layout, sorted-label slots only; E_c)."""
        N, K, K_H = self.N, self.K, self.K_H
        kfull = K + K_H
        kmax = min(kfull, N) if kmax is None else kmax
        R = np.zeros_like(t)
        e = 0.0
        for k in range(1, kmax + 1):
            c = moebius(N, k, kfull)
            ce = moebius(N, k, K_H) if k <= K_H else 0
            if c == 0 and ce == 0:
                continue
            Tb = tables(k, K, K_H)
            descs = [unpack(d) for d in Tb["out_desc"]]
            for Lset in itertools.combinations(range(N), k):
                Rl, e0 = self.local(Tb, Lset, t, **kw)
                e += ce * e0
                if c == 0:
                    continue
                for o in range(1, len(descs)):
                    m, pos, ch = descs[o]
                    R[self.slot_of([Lset[p] for p in pos], ch)] += c * Rl[o]
        return R, e

    def fill_copies(self, v, lm):
        """The other stored orders of every two- and three-pair entry, from
        the sorted-label slots (the layout's copy rule)."""
        N = self.N
        out = v.copy()
        t2 = out[3 * N:3 * N + 29 * N * N].reshape(N, N, 29)
        for P in range(N):
            for Q in range(P + 1, N):
                for k in range(29):
                    k2, sg = lm.swap[k]
                    t2[Q, P, k2] = sg * t2[P, Q, k]
        if lm.A3:
            t3 = out[3 * N + 29 * N * N:].reshape(N, N, N, len(lm.A3))
            for P, Q, R in itertools.combinations(range(N), 3):
                for k in range(len(lm.A3)):
                    for lbl, c, sg in lm._copies3((P, Q, R), k):
                        t3[lbl + (c,)] = sg * t3[P, Q, R, k]
        return out


def _rows(ptr):
    return np.repeat(np.arange(len(ptr) - 1), np.diff(ptr))


class SubsetAdjoint(SubsetInterp):
    """Reverse pass of the label-subset residual: the gradient of the
    Lagrangian L = E_c + sum over unique slots of lam R with respect to the
    amplitudes and to the integral keys, from the transposed tables (the
    algorithm of the adjoint kernels, interpreted with numpy)."""

    def local_adjoint(self, Tb, Lset, t, w):
        """(tbar[slot], vlbar[key]) of the local Lagrangian sum_o w[o] R_o
        (R_0 = phi'(ref))."""
        sd = [unpack(d) for d in Tb["slot_desc"]]
        tl = np.array([self.amp(t, [Lset[p] for p in pos], ch) for _, pos, ch in sd])
        kd = [unpack(d) for d in Tb["key_desc"]]
        vl = np.array([self.integral([Lset[p] for p in pos], j) for _, pos, j in kd])
        # forward
        sg = np.where(Tb["ent_slot"] & 1, -1.0, 1.0)
        slot = Tb["ent_slot"].astype(np.int64) >> 1
        psi = np.zeros(len(Tb["code"])); psi[0] = 1.0
        lp, ep = Tb["lvl_ptr"], Tb["ent_ptr"]
        for lv in range(1, len(lp) - 1):
            s0, s1 = lp[lv], lp[lv + 1]
            e0, e1 = ep[s0], ep[s1]
            owner = np.repeat(np.arange(s0, s1), np.diff(ep[s0:s1 + 1]))
            psi[s0:s1] = np.bincount(owner - s0, weights=sg[e0:e1] * tl[slot[e0:e1]] * psi[Tb["ent_sub"][e0:e1]],
                                     minlength=s1 - s0)
        E0 = float(np.sum(Tb["e0_c"] * vl[Tb["e0_key"]]))
        hp = Tb["h_ptr"]
        nout = len(Tb["out_state"])
        phi = np.bincount(_rows(hp), weights=Tb["h_c"] * vl[Tb["h_key"]] * psi[Tb["h_s"]], minlength=nout)
        D = np.bincount(_rows(Tb["d_ptr"]), weights=Tb["d_c"] * vl[Tb["d_key"]], minlength=nout) - E0
        phi += D * psi[Tb["out_state"]]
        pm = np.zeros(nout); pm[0] = 1.0
        order, olp, oep = Tb["olvl_order"], Tb["olvl_ptr"], Tb["oent_ptr"]
        osg = np.where(Tb["oent_slot"] & 1, -1.0, 1.0)
        oslot = Tb["oent_slot"].astype(np.int64) >> 1
        for lv in range(1, len(olp) - 1):
            for i in range(olp[lv], olp[lv + 1]):
                e0, e1 = oep[i], oep[i + 1]
                pm[order[i]] = -np.sum(osg[e0:e1] * tl[oslot[e0:e1]] * pm[Tb["oent_sub"][e0:e1]])
        # reverse
        M13 = (1 << 13) - 1
        w0, w = w[0], w.copy()
        w[0] = 0.0                      # output 0 enters as phi'(ref) itself, not through R_0
        bk = Tb["bk_ent"].astype(np.int64)
        o, om, bsg = bk & M13, (bk >> 13) & M13, np.where((bk >> 26) & 1, -1.0, 1.0)
        phibar = np.bincount(_rows(Tb["bk_ptr"]), weights=bsg * w[o] * pm[om], minlength=nout)
        phibar[0] += w0
        bw = Tb["bw_ent"].astype(np.int64)
        o2, kk, bsg2 = bw & M13, (bw >> 13) & M13, np.where((bw >> 26) & 1, -1.0, 1.0)
        pmbar = np.bincount(_rows(Tb["bw_ptr"]), weights=bsg2 * w[o2] * phi[kk], minlength=nout)
        obs = Tb["obs_ent"].astype(np.int64)
        obs_s, obs_sl = obs & 0xFFFFFFFF, obs >> 32
        obsp = Tb["obs_ptr"]
        for lv in range(len(olp) - 2, 0, -1):
            for i in range(olp[lv], olp[lv + 1]):
                u = order[i]
                e0, e1 = obsp[i], obsp[i + 1]
                if e1 > e0:
                    sl2 = obs_sl[e0:e1]
                    pmbar[u] += np.sum(-np.where(sl2 & 1, -1.0, 1.0) * tl[sl2 >> 1] * pmbar[obs_s[e0:e1]])
        nslot = len(Tb["slot_desc"])
        obl = Tb["obl_ent"].astype(np.int64)
        s_, sub_, sgn_ = obl & 0xFFFFF, (obl >> 20) & 0xFFFFF, np.where((obl >> 40) & 1, -1.0, 1.0)
        tbar = np.bincount(_rows(Tb["obl_ptr"]), weights=-sgn_ * pm[sub_] * pmbar[s_], minlength=nslot)
        hs = Tb["hs_ent"].astype(np.int64)
        kap, key = hs & M13, (hs >> 13) & 0x7FFF
        coef = np.where((hs >> 29) & 1, 0.5, 1.0) * np.where((hs >> 28) & 1, -1.0, 1.0)
        ns = len(Tb["code"])
        psibar = np.bincount(_rows(Tb["hs_ptr"]), weights=coef * vl[key] * phibar[kap], minlength=ns)
        oos = Tb["out_of_state"]
        isout = oos >= 0
        psibar[isout] += D[oos[isout]] * phibar[oos[isout]]
        bs = Tb["bs_ent"].astype(np.int64)
        bs_s, bs_sl = bs & 0xFFFFFFFF, bs >> 32
        bsp = Tb["bs_ptr"]
        for lv in range(len(lp) - 2, 0, -1):
            s0, s1 = lp[lv], lp[lv + 1]
            e0, e1 = bsp[s0], bsp[s1]
            if e1 > e0:
                owner = np.repeat(np.arange(s0, s1), np.diff(bsp[s0:s1 + 1]))
                sl2 = bs_sl[e0:e1]
                psibar[s0:s1] += np.bincount(owner - s0, weights=np.where(sl2 & 1, -1.0, 1.0) * tl[sl2 >> 1]
                                             * psibar[bs_s[e0:e1]], minlength=s1 - s0)
        bl = Tb["bl_ent"].astype(np.int64)
        s_, sub_, sgn_ = bl & 0xFFFFF, (bl >> 20) & 0xFFFFF, np.where((bl >> 40) & 1, -1.0, 1.0)
        tbar += np.bincount(_rows(Tb["bl_ptr"]), weights=sgn_ * psi[sub_] * psibar[s_], minlength=nslot)
        hk = Tb["hk_ent"].astype(np.int64)
        kap, st = hk & M13, (hk >> 13) & 0xFFFFF
        coef = np.where((hk >> 34) & 1, 0.5, 1.0) * np.where((hk >> 33) & 1, -1.0, 1.0)
        nkey = len(Tb["key_desc"])
        vlbar = np.bincount(_rows(Tb["hk_ptr"]), weights=coef * psi[st] * phibar[kap], minlength=nkey)
        dko = Tb["dk_out"]
        vlbar += np.bincount(_rows(Tb["dk_ptr"]), weights=Tb["dk_c"] * psi[Tb["out_state"][dko]] * phibar[dko],
                             minlength=nkey)
        vlbar -= Tb["e0_by_key"] * float(np.sum(psi[Tb["out_state"]] * phibar))
        return tbar, vlbar, (sd, kd)

    def lagrangian_gradient(self, t, lam, kmax=None):
        """(grad_t L in the layout (sorted-label slots), dict key -> dL/dvalue
        over the global integral keys (labels tuple, key index))."""
        N, K, K_H = self.N, self.K, self.K_H
        kfull = K + K_H
        kmax = min(kfull, N) if kmax is None else kmax
        g = np.zeros_like(t)
        gv = {}
        for k in range(1, kmax + 1):
            c = moebius(N, k, kfull)
            ce = moebius(N, k, K_H) if k <= K_H else 0
            if c == 0 and ce == 0:
                continue
            Tb = tables(k, K, K_H)
            descs = [unpack(d) for d in Tb["out_desc"]]
            for Lset in itertools.combinations(range(N), k):
                w = np.zeros(len(descs))
                w[0] = ce
                for o in range(1, len(descs)):
                    m, pos, ch = descs[o]
                    w[o] = c * lam[self.slot_of([Lset[p] for p in pos], ch)]
                tbar, vlbar, (sd, kd) = self.local_adjoint(Tb, Lset, t, w)
                for (m, pos, ch), tb in zip(sd, tbar):
                    g[self.slot_of([Lset[p] for p in pos], ch)] += tb
                for (m, pos, j), vb in zip(kd, vlbar):
                    key = (tuple(Lset[p] for p in pos), j)
                    gv[key] = gv.get(key, 0.0) + vb
        return g, gv
