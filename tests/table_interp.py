"""A plain NumPy interpreter of the generated tables (test infrastructure).

It reads the header that the build generates (``tables.emit_header``) and
evaluates the PQ residual and energy the way the device kernels use those
tables: staging (Fock, truncated one-body h', gathers), link coefficients,
site and pair closures by operator-by-operator sweeps, the topologies T1-T9,
the exp(-T_YZ) transform and the assembly.  It shares no code with the CUDA
path (it only reads the same tables) and none with the oracle; comparing it
with the oracle on the CPU pins the table generator without a GPU.
"""
import os
import re
import tempfile

import numpy as np

from paper_1609_00077_gb300 import tables as T


class Header:
    """Arrays and #defines of a generated header."""

    def __init__(self, path=None):
        if path is None:
            fd, path = tempfile.mkstemp(suffix=".h")
            os.close(fd)
            try:
                T.emit_header(path)
                text = open(path).read()
            finally:
                os.remove(path)
        else:
            text = open(path).read()
        self.defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define (\w+) (-?\d+)", text)}
        self.arr = {}
        for m in re.finditer(r"\b(?:static\s+)?(?:__device__\s+)?const\s+\w+\s+(\w+)\[\d*\]\s*=\s*\{([^}]*)\}",
                             text):
            vals = [v.strip().rstrip("f") for v in m.group(2).split(",") if v.strip()]
            self.arr[m.group(1)] = np.array([float(v) for v in vals])

    def __getitem__(self, name):
        return self.arr[name]

    def i(self, name):
        return self.arr[name].astype(np.int64)

    def f(self, name):
        return self.arr[name].astype(np.float64)


def _unpack(w):
    return w >> 17, (w >> 1) & 0xFFFF, np.where(w & 1, -1.0, 1.0)


def staging(hd, h, eri, occ, vir):
    """Fock f, truncated one-body h' and the per-site / per-pair gathers."""
    n = h.shape[0]
    N = len(occ)
    lab = np.empty(n, dtype=np.int64)
    lab[occ] = np.arange(N)
    lab[vir] = np.arange(N)
    f = h.copy()
    hp = h.copy()
    for p in range(n):
        for q in range(n):
            mf = mfl = 0.0
            for k in range(N):
                i = occ[k]
                v = 2.0 * eri[p, q, i, i] - eri[p, i, i, q]
                mf += v
                if k == lab[p] or k == lab[q]:
                    mfl += v
            f[p, q] = h[p, q] + mf
            hp[p, q] = h[p, q] if lab[p] == lab[q] else h[p, q] + mf - mfl
    g1key = hd.i("ppq_g1key").reshape(-1, 5)
    g2key = hd.i("ppq_g2key").reshape(-1, 5)

    def val(o, k):
        return hp[o[k[1]], o[k[2]]] if k[0] == 0 else eri[o[k[1]], o[k[2]], o[k[3]], o[k[4]]]

    g1 = np.array([[val((occ[X], vir[X]), k) for k in g1key] for X in range(N)])
    g2 = np.zeros((N, N, len(g2key)))
    for X in range(N):
        for W in range(N):
            if X != W:
                o = (occ[X], vir[X], occ[W], vir[W])
                g2[X, W] = [val(o, k) for k in g2key]
    return f, hp, g1, g2


def links(hd, t2):
    """Cl[X,Y][c] = <c| exp(T_XY) |ref> on the 36-state sector."""
    N = t2.shape[0]
    sop, sptr = hd.i("ppq_sop"), hd.i("ppq_sop_ptr")
    cl = np.zeros((N, N, 36))
    for X in range(N):
        for Y in range(N):
            if X == Y:
                continue
            v = np.zeros(36)
            v[0] = 1.0
            for k in range(29):
                for w in sop[sptr[k]:sptr[k + 1]]:
                    tg, s, g = _unpack(w)
                    v[tg] += t2[X, Y, k] * g * v[s]
            cl[X, Y] = v
    return cl


def _sweeps(M, lists, ops, tvals):
    """M <- M prod (1 + t O) (right), then M <- prod (1 - t O) M (left), one
    operator at a time; the entries of one operator act in parallel."""
    (right, rptr), (left, lptr) = lists
    for sgn, lst, ptr in ((1.0, right, rptr), (-1.0, left, lptr)):
        for o in range(ops):
            ent = lst[ptr[o]:ptr[o + 1]]
            if len(ent) == 0:
                continue
            tg, s, g = _unpack(ent)
            upd = sgn * tvals[o] * g * M[s]
            np.add.at(M, tg, upd)
    return M


def site_closure(hd, g1, t1):
    """Ht_X (16x16, flattened) and the site energy pieces."""
    N = g1.shape[0]
    el, ptr, j, c = hd.i("ppq_h1_el"), hd.i("ppq_h1_ptr"), hd.i("ppq_h1_j"), hd.f("ppq_h1_c")
    lists = ((hd.i("ppq_s_right"), hd.i("ppq_s_rptr")), (hd.i("ppq_s_left"), hd.i("ppq_s_lptr")))
    hs = np.zeros((N, 256))
    es = np.zeros(N)
    for X in range(N):
        M = np.zeros(256)
        for e in range(len(el)):
            M[el[e]] = np.dot(c[ptr[e]:ptr[e + 1]], g1[X, j[ptr[e]:ptr[e + 1]]])
        h00 = M[0]
        _sweeps(M, lists, 3, t1[X])
        hs[X] = M
        es[X] = M[0] - h00
    return hs, es


def pair_closure(hd, g2, t1, t2):
    """Outputs of the two-site closures: G row, T7 entries, column 0, energy."""
    N = g2.shape[0]
    el, ptr, j, c = hd.i("ppq_h2_el"), hd.i("ppq_h2_ptr"), hd.i("ppq_h2_j"), hd.f("ppq_h2_c")
    lists = ((hd.i("ppq_p_right"), hd.i("ppq_p_rptr")), (hd.i("ppq_p_left"), hd.i("ppq_p_lptr")))
    g_el, t7_el, c0_el = hd.i("ppq_g_el"), hd.i("ppq_t7_el"), hd.i("ppq_col0_el")
    el00 = hd.defs["PPQ_EL00"]
    blk = hd.defs["PPQ_BLK"]
    pg = np.zeros((N, N, 36))
    pt7 = np.zeros((N, N, len(t7_el)))
    pc0 = np.zeros((N, N, len(c0_el)))
    ep = np.zeros((N, N))
    for X in range(N):
        for W in range(N):
            if X == W:
                continue
            M = np.zeros(blk)
            for e in range(len(el)):
                M[el[e]] = np.dot(c[ptr[e]:ptr[e + 1]], g2[X, W, j[ptr[e]:ptr[e + 1]]])
            h00 = M[el00]
            tops = np.concatenate([t1[X], t1[W], t2[X, W]])
            _sweeps(M, lists, 35, tops)
            pg[X, W], pt7[X, W], pc0[X, W] = M[g_el], M[t7_el], M[c0_el]
            ep[X, W] = M[el00] - h00
    return pg, pt7, pc0, ep


def r1_terms(hd, hs, pc0, cl, pg):
    """r1[Y][k]: T1 (site element), T3, column 0 of the pair closures, T8."""
    N = hs.shape[0]
    A1 = hd.i("ppq_A1")
    t3, t3p = hd.i("ppq_t3").reshape(-1, 3), hd.i("ppq_t3p")
    t8, t8p = hd.i("ppq_t8").reshape(-1, 5), hd.i("ppq_t8p")
    r1 = np.zeros((N, 3))
    for Y in range(N):
        for k in range(3):
            acc = hs[Y, A1[k] * 16]
            for X in range(N):
                if X == Y:
                    continue
                for e in range(t3p[k], t3p[k + 1]):
                    acc += hs[X, t3[e, 1]] * cl[X, Y, t3[e, 0]]
                acc += pc0[Y, X, 29 + k]
                for W in range(N):
                    if W == X or W == Y:
                        continue
                    for e in range(t8p[k], t8p[k + 1]):
                        q = t8[e]
                        acc += 0.5 * q[4] * cl[X, Y, q[0]] * cl[W, Y, q[1]] * pg[X, W, q[2]]
            r1[Y, k] = acc
    return r1


def r2_terms(hd, hs, pc0, pt7, pg, cl, t2):
    """dir (T4 + column 0, Y < Z) and abuf (T2 + T7 through exp(-T_YZ))."""
    N = hs.shape[0]
    t4, t4p = hd.i("ppq_t4").reshape(-1, 5), hd.i("ppq_t4p")
    t2c, t2p = hd.i("ppq_t2").reshape(-1, 4), hd.i("ppq_t2p")
    t7, t7p = hd.i("ppq_t7").reshape(-1, 5), hd.i("ppq_t7p")
    sop, sptr = hd.i("ppq_sop"), hd.i("ppq_sop_ptr")
    dirr = np.zeros((N, N, 29))
    abuf = np.zeros((N, N, 29))
    for Y in range(N):
        for Z in range(N):
            if Y == Z:
                continue
            if Y < Z:
                for o in range(29):
                    acc = pc0[Y, Z, o]
                    for X in range(N):
                        if X == Y or X == Z:
                            continue
                        for e in range(t4p[o], t4p[o + 1]):
                            q = t4[e]
                            acc += q[4] * cl[X, Y, q[0]] * cl[X, Z, q[1]] * hs[X, q[2]]
                    dirr[Y, Z, o] = acc
            U = np.zeros(36)
            for nu in range(36):
                acc = 0.0
                for e in range(t2p[nu], t2p[nu + 1]):
                    q = t2c[e]
                    acc += cl[Y, Z, q[0]] * hs[Y, q[1] * 16 + q[2]]
                # T7: sum_W pt7[Y,W][e] Cl[W,Z][c2] Cl[Y,Z][c1]
                for e in range(t7p[nu], t7p[nu + 1]):
                    c1, c2, el, _, sg = t7[e]
                    acc += sg * cl[Y, Z, c1] * np.dot(pt7[Y, :, el], cl[:, Z, c2])
                U[nu] = acc
            for k in range(29):
                ent = sop[sptr[k]:sptr[k + 1]]
                if len(ent):
                    tg, s, g = _unpack(ent)
                    upd = -t2[Y, Z, k] * g * U[s]
                    np.add.at(U, tg, upd)
            abuf[Y, Z] = U[1:30]
    return dirr, abuf


def t9_term(hd, cl, pg):
    """Quartic topology for Y < Z:
    t9[Y,Z][o] = 1/2 sum_{X != W} sum_ch s Cl[X,Y][c1] Cl[X,Z][c2] G[X,W][g] Cl[W,Y][c3] Cl[W,Z][c4]."""
    N = cl.shape[0]
    p9 = hd.i("ppq_p9").reshape(-1, 2)
    q9 = hd.i("ppq_q9").reshape(-1, 2)
    c9 = hd.i("ppq_c9").reshape(-1, 5)    # (q, c3, c4, out, sign)
    off = ~np.eye(N, dtype=bool)
    t9 = np.zeros((N, N, 29))
    for q, c3, c4, o, sg in c9:
        (c1, c2), g = p9[q9[q, 0]], q9[q, 1]
        G = pg[:, :, g] * off
        for Y in range(N):
            for Z in range(Y + 1, N):
                a = cl[:, Y, c1] * cl[:, Z, c2]
                b = cl[:, Y, c3] * cl[:, Z, c4]
                t9[Y, Z, o] += 0.5 * sg * (a @ G @ b)
    return t9


def residual(hd, h, eri, occ, vir, t):
    """(R in the layout of include/ppq.h, E_c) at amplitudes t (same layout)."""
    occ = np.asarray(occ, dtype=np.int64)
    vir = np.asarray(vir, dtype=np.int64)
    N = len(occ)
    t1 = t[:3 * N].reshape(N, 3)
    t2 = t[3 * N:].reshape(N, N, 29)
    _, _, g1, g2 = staging(hd, h, eri, occ, vir)
    cl = links(hd, t2)
    hs, es = site_closure(hd, g1, t1)
    pg, pt7, pc0, ep = pair_closure(hd, g2, t1, t2)
    r1 = r1_terms(hd, hs, pc0, cl, pg)
    dirr, abuf = r2_terms(hd, hs, pc0, pt7, pg, cl, t2)
    t9 = t9_term(hd, cl, pg)
    swap, swsg = hd.i("ppq_a2_swap"), hd.f("ppq_a2_swsg")
    r2 = np.zeros((N, N, 29))
    for Y in range(N):
        for Z in range(Y + 1, N):
            a = dirr[Y, Z] + t9[Y, Z] + abuf[Y, Z] + swsg * abuf[Z, Y, swap]
            r2[Y, Z] = a
            r2[Z, Y, swap] = swsg * a
    e = es.sum() + 0.5 * ep.sum()
    return np.concatenate([r1.ravel(), r2.ravel()]), e
