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
         "h_key", "h_c", "e0_key", "e0_c", "b_ptr", "b_k", "b_w", "d_ptr", "d_key", "d_c"]
DTYPES = {"code": np.uint32, "ent_slot": np.int16, "oent_slot": np.int16, "h_key": np.int16,
          "e0_key": np.int16, "h_c": np.float64, "e0_c": np.float64, "d_key": np.int16, "d_c": np.float64}

_CACHE = {}


def tables(k, K, K_H):
    key = (k, K, K_H)
    if key not in _CACHE:
        L = ppq.lib()
        L.ph_tables_counts.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p]
        L.ph_tables_copy.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p]
        cnt = np.zeros(32, dtype=np.int64)
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
