"""C-ABI checks that need no GPU: the library loads, exports every function of
include/ppq.h, describes its layout, and rejects bad arguments before any
device work."""
import os
import re

import numpy as np
import pytest

import paper_1609_00077_gb300 as ppq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ppq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ppq_\w+|pq_\w+|ph_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = ppq.lib()
    names = _declared()
    assert {"pq_solve", "ph_solve", "pq_residual", "ppq_amp_count", "ppq_amp_layout"} <= set(names)
    for name in names:
        assert hasattr(L, name), name


def test_amp_count_and_layout():
    for N in (2, 5, 70):
        assert ppq.amp_count(N) == 3 * N + 29 * N * N
    d = ppq.amp_layout()
    assert (d[:3, 0] == 1).all() and (d[3:, 0] == 2).all()
    # every channel conserves charge and S_z (Eq. decompose: excitations only)
    def qn(m):
        dn = bin(m & 12).count("1") - bin(m & 3).count("1")
        ds = ((m >> 2) & 1) - ((m >> 3) & 1) - ((m & 1) - ((m >> 1) & 1))
        return dn, ds
    for kind, a, b in d:
        qa, qb = qn(a), qn(b)
        assert qa[0] + qb[0] == 0 and qa[1] + qb[1] == 0
    assert len({(a, b) for k, a, b in d if k == 2}) == 29


def test_bad_pairing_rejected_without_gpu():
    n = 4
    h = np.zeros((n, n)); eri = np.zeros((n,) * 4)
    with pytest.raises(ppq.PPQError, match="twice"):
        ppq.pq_solve([0, 0], [2, 3], h, eri)
    with pytest.raises(ppq.PPQError, match="range"):
        ppq.pq_solve([0, 1], [2, 9], h, eri)
    with pytest.raises(ppq.PPQError, match="n_pairs"):
        ppq.pq_solve([0], [1], np.zeros((2, 2)), np.zeros((2,) * 4))


def test_ph_entry_points_reject_bad_arguments_without_gpu():
    # argument errors come back before any device work, with their own codes
    n = 6
    h = np.zeros((n, n)); eri = np.zeros((n,) * 4)
    with pytest.raises(ppq.PPQError, match=r"ph_solve failed \(-4\).*K_H"):
        ppq.ph_solve([2, 1, 0], [3, 4, 5], h, eri, K_H=4)
    with pytest.raises(ppq.PPQError, match="twice"):
        ppq.ph_solve([2, 2, 0], [3, 4, 5], h, eri)
    with pytest.raises(ppq.PPQError, match=r"pq_solve failed \(-4\).*max_rank"):
        ppq.pq_solve([2, 1, 0], [3, 4, 5], h, eri, max_rank=2)
    with pytest.raises(ppq.PPQError, match=r"pq_solve failed \(-4\).*switch_tol"):
        ppq.pq_solve([2, 1, 0], [3, 4, 5], h, eri, switch_tol=-1e-5)
    with pytest.raises(ppq.PPQError, match=r"ph_solve failed \(-4\).*max_rank"):
        ppq.ph_solve([2, 1, 0], [3, 4, 5], h, eri, max_rank=7)
    t = np.zeros(ppq.amp_count(3, 3))
    with pytest.raises(ppq.PPQError, match=r"ph_residual failed \(-4\).*K_H"):
        ppq.ph_residual([2, 1, 0], [3, 4, 5], h, eri, t, K_H=1)


def test_amp_count_three_pair():
    for N in (2, 3, 15):
        assert ppq.amp_count(N, 3) == 3 * N + 29 * N * N + 303 * N ** 3


def test_binding_checks_buffers_before_any_launch():
    # a short, mistyped or non-contiguous buffer is refused in the binding,
    # before the library could read or write past it
    N, n = 3, 6
    h = np.zeros((n, n)); eri = np.zeros((n,) * 4)
    L = ppq.amp_count(N)
    occ, vir = [2, 1, 0], [3, 4, 5]
    with pytest.raises(ppq.PPQError, match="t holds"):
        ppq.pq_residual(occ, vir, h, eri, np.zeros(L - 1))
    with pytest.raises(ppq.PPQError, match="float64"):
        ppq.pq_residual(occ, vir, h, eri, np.zeros(L, dtype=np.float32))
    with pytest.raises(ppq.PPQError, match="eri holds"):
        ppq.pq_residual(occ, vir, h, eri[:5], np.zeros(L))
    with pytest.raises(ppq.PPQError, match="float64"):
        ppq.pq_residual(occ, vir, h, eri, np.zeros((L, 2))[:, 0])
    with pytest.raises(ppq.PPQError, match="r holds"):
        ppq.pq_residual(occ, vir, h, eri, np.zeros(L), np.zeros(3))
    with pytest.raises(ppq.PPQError, match="device pointers"):
        ppq.pq_residual_static(occ, vir, h, eri, np.zeros(L), np.zeros(L))
    with pytest.raises(ppq.PPQError, match="t_out holds"):
        ppq.ph_solve(occ, vir, h, eri, t_out=np.zeros(ppq.amp_count(N, 3) - 1))
    with pytest.raises(ppq.PPQError, match="t holds"):
        ppq.ph_residual(occ, vir, h, eri, np.zeros(ppq.amp_count(N)))


def test_layout_map_round_trip():
    from oracle.detcc import enumerate_manifold
    from tests.layout import LayoutMap
    occ, vir = np.array([2, 0, 1]), np.array([3, 5, 4])
    man = enumerate_manifold(occ, vir, 2)
    lm = LayoutMap(man, occ, vir, 6, ppq.amp_layout())
    t = np.random.default_rng(3).normal(size=len(man))
    v = lm.to_layout(t)
    assert np.allclose(lm.from_layout(v), t)
    assert lm.mirror_error(v) == 0.0
