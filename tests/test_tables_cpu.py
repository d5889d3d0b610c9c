"""Host-side pins of the generated tables and of the arithmetic the tensor-core
kernels rely on (no GPU needed).

* The pair closure's per-sector sweep lists (groups of four entries of one
  operator, padded with no-op entries, offsets in the padded sector layout)
  reproduce the flat operator-by-operator sweeps exactly, stay inside their
  sector block, and give every thread of a sector a row start in its own
  shared-memory bank.
* The generated straight-line sweeps (ppq_sweep_right / ppq_sweep_left, the
  C++ source the kernel compiles, parsed back here) give the same entries as
  the flat sweeps on every sector, row by row and column by column.
* The pair closure's gather as per-thread term streams (256 coalesced
  streams, zero-padded) writes every Hamiltonian element once, with the same
  terms in the same order as the CSR, at the element's padded offset.
* The exact integer splitting of the FP64 quartic kernel (six 7-bit slices,
  K <= 80): every grouped slice-product sum is an exact FP32 integer below
  2^23, and the recombined product is within 3e-12 of row-max x column-max x K;
  the slicing on bit patterns (integer operations only) rounds to the nearest
  integer, ties away from zero, and its digits recombine exactly.
* The FP64 epilogue groups keep each output of a (c1, c2, g) in one group.
* The generated straight-line T8 code of r1 and T4 code of r2 hold their
  tables' entries in order.
* The FP64 epilogue's double-float W contraction, run in emulated FP32
  operations, stays within 2^-43 of the sum of |terms| of the exact value
  (a variant that kept the lower limbs of D in plain FP32 accumulators, an
  earlier draft, fails it), and the float pair of an integer below 2^58 is
  exact to 2^-48.
* The spin-flip map of the amplitude channels (spin_flip_channels) and its
  signs hold for closed-shell amplitudes of the oracle mapped to the layout.
"""
import numpy as np
import pytest

from paper_1609_00077_gb300 import tables as T


@pytest.fixture(scope="module")
def layout():
    Tb = T.Tables()
    return Tb, T.BlockLayout(Tb)


def test_sector_lists_reproduce_flat_sweeps(layout):
    Tb, L = layout
    pr, prp, pl, plp = T.pair_transform_lists(Tb, L)
    sr, srp, sl, slp = T.pair_sector_lists(Tb, L)
    rng = np.random.default_rng(3)
    M0 = rng.standard_normal(L.size)
    t = rng.standard_normal(35) * 0.3
    # flat lists, operator by operator
    M = M0.copy()
    for o in range(35):
        for w in pr[prp[o]:prp[o + 1]]:
            M[w >> 17] += t[o] * (-1 if w & 1 else 1) * M[(w >> 1) & 0xFFFF]
    for o in range(35):
        for w in pl[plp[o]:plp[o + 1]]:
            M[w >> 17] -= t[o] * (-1 if w & 1 else 1) * M[(w >> 1) & 0xFFFF]
    # per-sector lists in the padded layout (row stride dim + 1)
    pbase, off = [], 0
    for d in L.dim:
        pbase.append(off)
        off += d * (d + 1)
    P = np.zeros(off)
    for q, ss in enumerate(L.sectors):
        for r in ss:
            for c in ss:
                P[pbase[q] + L.pos[r] * (L.dim[q] + 1) + L.pos[c]] = M0[L.elem(r, c)]
    fac = np.zeros(72)
    fac[0:70:2], fac[1:70:2] = t, -t
    for lst, lp, rows, sgn in ((sr, srp, True, 1.0), (sl, slp, False, -1.0)):
        for st in range(256):
            q = L.sec_of[st]
            d, dp = L.dim[q], L.dim[q] + 1
            base = pbase[q] + (L.pos[st] * dp if rows else L.pos[st])
            lo, hi = pbase[q], pbase[q] + d * dp
            for e in range(lp[q], lp[q + 1], 4):
                grp = lst[e:e + 4]
                ti = [base + (w & 0xFFF) for w in grp]
                si = [base + ((w >> 12) & 0xFFF) for w in grp]
                assert all(lo <= x < hi for x in ti + si)
                real = [x for x, w in zip(ti, grp) if (w >> 24) != 70]
                assert len(set(real)) == len(real) and not set(real) & set(si)
                vals = [P[a] + sgn * fac[w >> 24] * P[b] for a, b, w in zip(ti, si, grp)]
                for a, v in zip(ti, vals):
                    P[a] = v
    for q, ss in enumerate(L.sectors):
        for r in ss:
            for c in ss:
                assert P[pbase[q] + L.pos[r] * (L.dim[q] + 1) + L.pos[c]] == M[L.elem(r, c)]
    # row starts of the threads of one sector fall in distinct banks
    for q, ss in enumerate(L.sectors):
        banks = [(pbase[q] + L.pos[r] * (L.dim[q] + 1)) % 32 for r in ss[:32]]
        assert len(set(banks)) == len(banks)


def test_generated_sweep_code_reproduces_flat_sweeps(layout):
    import re
    Tb, L = layout
    code, _ = T.pair_sweep_code(Tb, L)
    pr, prp, pl, plp = T.pair_transform_lists(Tb, L)
    rng = np.random.default_rng(4)
    M0 = rng.standard_normal(L.size)
    t = rng.standard_normal(35) * 0.3
    M = M0.copy()
    for o in range(35):
        for w in pr[prp[o]:prp[o + 1]]:
            M[w >> 17] += t[o] * (-1 if w & 1 else 1) * M[(w >> 1) & 0xFFFF]
    for o in range(35):
        for w in pl[plp[o]:plp[o + 1]]:
            M[w >> 17] -= t[o] * (-1 if w & 1 else 1) * M[(w >> 1) & 0xFFFF]
    fac = np.zeros(72)
    fac[0:70:2], fac[1:70:2] = t, -t
    # parse: side -> sector -> list of (target, source, factor slot, sign)
    prog = {}
    side = q = None
    for line in code.splitlines():
        m = re.match(r".*void ppq_sweep_(right|left)\(", line)
        if m:
            side = m.group(1); prog[side] = {}
            continue
        m = re.match(r"\s*case (\d+): \{", line)
        if m:
            q = int(m.group(1)); prog[side][q] = []
            continue
        m = re.match(r"\s*v\[(\d+)\] ([+-])= f(\d+) \* v\[(\d+)\];", line)
        if m:
            prog[side][q].append((int(m.group(1)), int(m.group(4)), int(m.group(3)),
                                  1.0 if m.group(2) == "+" else -1.0))
    assert set(prog) == {"right", "left"}
    A = np.zeros((256, 256))
    for r in range(256):
        for c in range(256):
            e = L.elem(r, c)
            if e >= 0:
                A[r, c] = M0[e]
    for sname, rows in (("right", True), ("left", False)):
        for qq, ss in enumerate(L.sectors):
            for st in ss:
                v = np.array([A[st, c] if rows else A[c, st] for c in ss])
                for a, b, f, sg in prog[sname].get(qq, []):
                    v[a] = v[a] + sg * fac[f] * v[b]
                for i, c in enumerate(ss):
                    if rows:
                        A[st, c] = v[i]
                    else:
                        A[c, st] = v[i]
    for qq, ss in enumerate(L.sectors):
        for r in ss:
            for c in ss:
                assert A[r, c] == M[L.elem(r, c)]


def test_gather_streams_reproduce_the_csr():
    from tests.table_interp import Header
    hd = Header()
    slen = hd.defs["PPQ_H2_SLEN"]
    st = hd.i("ppq_h2_stream").reshape(slen, 256)
    ptr, cj, elp = hd.i("ppq_h2_ptr"), hd.i("ppq_h2_cj"), hd.i("ppq_h2_elp")
    ng = hd.defs["PPQ_H2_NCODE"] * hd.defs["PPQ_NG2"]
    rng = np.random.default_rng(5)
    gsv = np.concatenate([rng.standard_normal(ng).astype(np.float32), np.zeros(8, np.float32)])
    ref = {}
    for el in range(len(elp)):
        acc = np.float32(0)
        for p in range(ptr[el], ptr[el + 1]):
            acc = np.float32(acc + gsv[cj[p]])
        ref[int(elp[el])] = acc
    got = {}
    for t in range(256):
        acc = np.float32(0)
        for j in range(slen):
            w = int(st[j, t])
            acc = np.float32(acc + gsv[w & 0x7FF])
            if w >> 31:
                off = (w >> 11) & 0x1FFF
                assert off not in got
                got[off] = acc
                acc = np.float32(0)
        assert acc == 0
    assert got.keys() == ref.keys()
    assert all(got[k] == ref[k] for k in ref)
    # balanced: the longest stream is within a few terms of the mean
    assert slen <= np.ceil(ptr[-1] / 256) + 12


def _split(M, bits=7, nsl=6):
    mx = np.abs(M).max(axis=1, keepdims=True)
    e = np.where(mx > 0, np.frexp(mx)[1], 0)
    xi = np.rint(np.ldexp(M, bits * nsl - e)).astype(np.int64)
    out, rem = [], xi
    for i in range(nsl):
        sh = bits * (nsl - 1 - i)
        a = rem >> sh
        rem = rem - (a << sh)
        out.append(a)
    assert (rem == 0).all()
    return out, e


@pytest.mark.parametrize("K", [8, 70, 80])
def test_exact_splitting_is_exact_and_bounded(K):
    rng = np.random.default_rng(K)
    A = rng.standard_normal((128, K)) * np.exp(rng.standard_normal((128, 1)) * 3)
    B = rng.standard_normal((80, K)) * np.exp(rng.standard_normal((80, 1)) * 2)
    As, ea = _split(A)
    Bs, eb = _split(B)
    assert np.abs(As[0]).max() <= 128 and all(0 <= a.min() and a.max() < 128 for a in As[1:])
    Dint = np.zeros((128, 80), dtype=np.int64)
    for g in range(6):
        S = sum(As[i].astype(np.float64) @ Bs[g - i].astype(np.float64).T for i in range(g + 1))
        assert np.abs(S).max() < 2 ** 23
        assert (S.astype(np.float32).astype(np.float64) == S).all()   # exact in the FP32 accumulator
        Dint += S.astype(np.int64) << (7 * (5 - g))
    D = np.ldexp(Dint.astype(np.float64), ea + eb.T - 49)
    scale = np.abs(A).max(1, keepdims=True) * np.abs(B).max(1, keepdims=True).T * K
    assert (np.abs(D - A @ B.T) / scale).max() < 3e-12


def test_three_pair_channels_and_sector(layout):
    # PH groundwork: the 303 three-pair channels, the three-label integral
    # keys, and the zero-charge three-site sector they span with the lower
    # ranks: 1 (reference) + 3 x 3 (one site) + 3 x 29 (two sites) + 303 = 400
    import itertools
    Tb, _ = layout
    A3 = T.amplitude_channels3()
    assert len(A3) == 303 and len(set(A3)) == 303
    assert len(T.triple_integral_keys()) == 576
    zero = sum(1 for st in itertools.product(range(16), repeat=3)
               if all(sum(Tb.qn[m][i] for m in st) == 0 for i in range(len(Tb.qn[0]))))
    assert zero == 1 + 3 * len(Tb.A1) + 3 * len(Tb.A2) + len(A3) == 400


def test_three_pair_channels_match_the_oracle_manifold():
    # the oracle enumerates the K = 3 manifold on its own; its excitations that
    # touch all three labels of N = 3 pairs, written as per-site monomial
    # masks, are exactly the 303 channels
    from oracle.detcc import enumerate_manifold
    occ, vir = [0, 1, 2], [3, 4, 5]
    lab = {0: 0, 1: 1, 2: 2, 3: 0, 4: 1, 5: 2}
    A3 = set(T.amplitude_channels3())
    seen = set()
    for ah, ap, bh, bp in enumerate_manifold(occ, vir, 3):
        mono = [0, 0, 0]
        for x in ah: mono[lab[x]] |= 1
        for x in bh: mono[lab[x]] |= 2
        for x in ap: mono[lab[x]] |= 4
        for x in bp: mono[lab[x]] |= 8
        if all(mono):
            seen.add(tuple(mono))
    assert seen == A3


def _split_bits(v, e):
    """The FP64 kernels' slicing on bit patterns: v 2^(42 - e) rounded to the
    nearest integer (ties away from zero) from the mantissa and exponent
    fields, then six floor digits of 7 bits (the first one signed)."""
    b = v.view(np.int64)
    ev = (b >> 52) & 0x7FF
    m = (b & 0x000FFFFFFFFFFFFF) | 0x0010000000000000
    sh = 1075 - 42 + e - ev
    ok = (ev != 0) & (sh > 0) & (sh < 64)
    shc = np.clip(sh, 1, 63)
    x = np.where(ok, (m + (np.int64(1) << (shc - 1))) >> shc, 0)
    x = np.where(b < 0, -x, x)
    a0 = x >> 35
    r = x - (a0 << 35)
    rh, rl = r >> 14, r & 0x3FFF
    return x, [a0, rh >> 14, (rh >> 7) & 127, rh & 127, rl >> 7, rl & 127]


def test_bit_pattern_split_rounds_to_nearest_and_recombines():
    from fractions import Fraction
    rng = np.random.default_rng(3)
    v = rng.standard_normal(20000) * np.exp(rng.standard_normal(20000) * 8)
    v[:2] = [0.0, -0.0]
    e = np.frexp(np.abs(v).max())[1]
    x, sl = _split_bits(v, e)
    assert np.abs(sl[0]).max() <= 128 and all(0 <= a.min() and a.max() < 128 for a in sl[1:])
    assert (sum(a << (7 * (5 - i)) for i, a in enumerate(sl)) == x).all()
    for vi, xi in zip(v[:2000], x[:2000]):
        q = Fraction(float(vi)) * Fraction(2) ** (42 - int(e))
        n = int(abs(q) + Fraction(1, 2))   # nearest, ties away from zero
        assert xi == (n if q >= 0 else -n)
    # exact ties go away from zero: 2.5 -> 3, -2.5 -> -3, 0.5 -> 1
    xt, _ = _split_bits(np.array([2.5, -2.5, 0.5]) * 2.0 ** -42, 0)
    assert list(xt) == [3, -3, 1]
    # the small slices are exact in FP32 through the 1.5 2^23 magic number
    a = np.arange(-128, 129, dtype=np.int32)
    f = (a + np.int32(0x4B400000)).view(np.float32) - np.float32(12582912.0)
    assert (f == a.astype(np.float32)).all()


def test_fp64_epilogue_groups_keep_outputs_whole_and_balance():
    from tests.table_interp import Header
    hd = Header()
    qp = hd.i("ppq_c9qp")
    c9q = hd.i("ppq_c9q").reshape(-1, 4)
    grp = hd.i("ppq_c9grp")
    assert len(grp) == len(c9q) and grp.min() >= 0 and grp.max() <= 3
    worst, fixed = 0, 0
    for q in range(len(qp) - 1):
        o, g = c9q[qp[q]:qp[q + 1], 2], grp[qp[q]:qp[q + 1]]
        for out in np.unique(o):
            assert len(np.unique(g[o == out])) == 1          # no two groups add into one output
        load = np.bincount(g, minlength=4)
        cnt = np.unique(o, return_counts=True)[1]
        assert load.max() <= max(cnt.max(), int(np.ceil(len(o) / 4)) + cnt.max() - 1)
        worst += load.max()
        fixed += np.bincount(o & 3, minlength=4).max()
    assert worst < 0.85 * fixed          # the busiest group does less than with outputs mod 4


def test_generated_r1_t8_code_reproduces_the_table():
    import re
    t8 = T.t8_channels(T.Tables())
    order = np.argsort(t8[:, 3], kind="stable")
    ref = [tuple(int(x) for x in t8[i]) for i in order]
    import os, tempfile
    fd, path = tempfile.mkstemp(suffix=".h")
    os.close(fd)
    try:
        T.emit_header(path)
        text = open(path).read()
    finally:
        os.remove(path)
    body = text[text.index("void ppq_r1_t8("):]
    body = body[:body.index("\n}")]
    lines = [l for l in body.splitlines() if l.strip().startswith("acc[")]
    pat = re.compile(r"acc\[(\d)\] \+= R\((-?0\.5)\) \* cx\[(\d+)\] \* cw\[(\d+)\] \* g\[(\d+) \* NN\];")
    got = []
    for l in lines:
        m = pat.fullmatch(l.strip())
        assert m, l
        k, h, c1, c2, g = m.groups()
        got.append((int(c1), int(c2), int(g), int(k), 1 if float(h) > 0 else -1))
    assert got == ref


def _generated_function(name):
    import os, re, tempfile
    fd, path = tempfile.mkstemp(suffix=".h")
    os.close(fd)
    try:
        T.emit_header(path)
        text = open(path).read()
    finally:
        os.remove(path)
    body = text[text.index(f"void {name}("):]
    return body[:body.index("\n}")]


def test_generated_link_code_follows_the_operator_table_and_inverts():
    import re
    sop = T.sector_pair_ops(T.Tables())
    rng = np.random.default_rng(2)
    t = rng.uniform(-0.3, 0.3, 29)
    progs = {}
    for name, sgn in (("ppq_link_apply", 1.0), ("ppq_link_unapply", -1.0)):
        body = _generated_function(name)
        k = None
        prog = []
        for l in body.splitlines():
            m = re.fullmatch(r"\s*\{ const R tk = R\(t\[(\d+)\]\);", l)
            if m:
                k = int(m.group(1))
                continue
            m = re.fullmatch(r"\s*v\[(\d+)\] ([+-])= tk \* R\((-?1)\) \* v\[(\d+)\];", l)
            if m:
                d, op, g, src = int(m.group(1)), m.group(2), int(m.group(3)), int(m.group(4))
                assert (op == "+") == (sgn > 0)
                prog.append((k, src, d, g))
        assert prog == [tuple(int(x) for x in r) for r in sop]
        progs[name] = (prog, sgn)

    def run(name, v):
        prog, sgn = progs[name]
        v = v.copy()
        for k, src, d, g in prog:
            v[d] += sgn * t[k] * g * v[src]
        return v

    v0 = np.zeros(36); v0[0] = 1.0
    v1 = run("ppq_link_apply", v0)
    assert np.abs(v1 - v0).max() > 1e-2
    assert np.abs(run("ppq_link_unapply", v1) - v0).max() < 1e-14   # exp(-T) exp(T) |ref> = |ref>


def _fma32(a, b, c):
    """fmaf on float32 values: the product is exact in FP64 (48 bits), the
    sum rounded once to FP64 and then to FP32 (a double rounding that can
    differ from a fused operation in the last bit, which the bound below
    absorbs)."""
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def _dpair(d):
    d2, d1, d0 = d >> 46, (d >> 23) & 0x7FFFFF, d & 0x7FFFFF
    f2 = np.float32(d2) * np.float32(2.0 ** 46)
    f1 = np.float32(d1) * np.float32(2.0 ** 23)
    f0 = np.float32(d0)
    x = np.float32(f2 + f1)
    e1 = np.float32(f1 - np.float32(x - f2))
    dh = np.float32(x + f0)
    e2 = np.float32(f0 - np.float32(dh - x))
    return dh, np.float32(e1 + e2)


def _epilogue_sum(D, A, B):
    """The FP64 quartic epilogue's W contraction as the kernel runs it in
    FP32 operations: float pairs for the link coefficients, a two-product,
    the float pair of the exact integer D, a two-sum accumulator."""
    vh = vl = np.float32(0.0)
    for d, a, b in zip(D, A, B):
        ax, ay = np.float32(a), np.float32(a - np.float64(np.float32(a)))
        bx, by = np.float32(b), np.float32(b - np.float64(np.float32(b)))
        dh, dl = _dpair(int(d))
        p = np.float32(ax * bx)
        pe = _fma32(ax, bx, -p)
        pe = _fma32(ax, by, pe)
        pe = _fma32(ay, bx, pe)
        hp = np.float32(dh * p)
        he = _fma32(dh, p, -hp)
        he = _fma32(dh, pe, he)
        he = _fma32(dl, p, he)
        s = np.float32(vh + hp)
        bb = np.float32(s - vh)
        t = np.float32(np.float32(vh - np.float32(s - bb)) + np.float32(hp - bb))
        vl = np.float32(vl + np.float32(t + he))
        vh = s
    return np.float64(vh) + np.float64(vl)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_double_float_epilogue_is_accurate_to_2e_minus_43(seed):
    from fractions import Fraction
    rng = np.random.default_rng(seed)
    W = 80
    # exact slice combinations of every magnitude below 2^58, both signs
    D = [int(rng.integers(0, 2 ** int(rng.integers(1, 58)))) * (1 if rng.random() < 0.5 else -1) for _ in range(W)]
    A = rng.standard_normal(W) * np.exp(rng.standard_normal(W))
    B = rng.standard_normal(W) * np.exp(rng.standard_normal(W))
    got = _epilogue_sum(D, A, B)
    exact = sum(Fraction(d) * Fraction(float(a)) * Fraction(float(b)) for d, a, b in zip(D, A, B))
    scale = sum(abs(Fraction(d) * Fraction(float(a)) * Fraction(float(b))) for d, a, b in zip(D, A, B))
    assert abs(Fraction(float(got)) - exact) <= Fraction(2) ** -43 * scale
    # the integer split alone is exact to 2^-48
    for d in D:
        dh, dl = _dpair(d)
        assert abs(Fraction(float(dh)) + Fraction(float(dl)) - d) <= Fraction(2) ** -48 * abs(d)


def test_generated_r2_t4_code_reproduces_the_table():
    import re
    t4 = T.t4_channels(T.Tables())
    order = np.argsort(t4[:, 3], kind="stable")
    ref = [tuple(int(x) for x in t4[i]) for i in order]
    hm = {0: 5, 1: 10, 2: 15}
    pat = re.compile(r"acc\[(\d+)\] \+= R\((-?1)\) \* cy\[(\d+)\] \* cz\[(\d+)\] \* hx\[(\d)\];")
    got = []
    for half, o0 in ((0, 0), (1, 15)):
        body = _generated_function(f"ppq_r2_t4_{half}")
        for l in body.splitlines():
            if not l.strip().startswith("acc["):
                continue
            m = pat.fullmatch(l.strip())
            assert m, l
            k, sg, c1, c2, j = (int(x) for x in m.groups())
            assert 0 <= k < (15 if half == 0 else 14)
            got.append((c1, c2, hm[j], o0 + k, sg))
    assert got == ref


@pytest.mark.parametrize("sites", [6, 8])
def test_spin_flip_channel_map_matches_the_oracle(sites):
    """Closed-shell amplitudes in the oracle's convention (equal on the
    alpha <-> beta exchange of every excitation, the symmetry the oracle pin
    test_residual_is_spin_flip_symmetric_for_closed_shell_hamiltonians
    fixes) satisfy t[flip(k)] = sigma(k) t[k] per pair and per ordered pair
    in the C-ABI layout, with the flip and signs of spin_flip_channels."""
    import paper_1609_00077_gb300 as ppq
    from workloads import build_ppp
    from oracle.detcc import enumerate_manifold
    from tests.layout import LayoutMap
    H = build_ppp('polyene', sites)
    N = H.n_pairs
    man = enumerate_manifold(H.occ_of_pair, H.vir_of_pair, 2)
    idx = {m: i for i, m in enumerate(man)}
    flip = np.array([idx[(bh, bp, ah, ap)] for ah, ap, bh, bp in man])
    t = np.random.default_rng(sites).uniform(-0.1, 0.1, len(man))
    t = 0.5 * (t + t[flip])
    lm = LayoutMap(man, H.occ_of_pair, H.vir_of_pair, H.n_orb, ppq.amp_layout(2))
    v = lm.to_layout(t)
    f1, s1, f2, s2 = T.spin_flip_channels(T.Tables())
    t1 = v[:3 * N].reshape(N, 3)
    t2 = v[3 * N:].reshape(N, N, 29)
    assert np.abs(t1).max() > 1e-3 and np.abs(t2).max() > 1e-3
    assert np.abs(t1[:, f1] - s1 * t1).max() < 1e-15
    assert np.abs(t2[:, :, f2] - s2 * t2).max() < 1e-15
    # and the map is an involution with consistent signs
    assert (f1[f1] == np.arange(3)).all() and (f2[f2] == np.arange(29)).all()
    assert (s2[f2] == s2).all() and (s1[f1] == s1).all()
