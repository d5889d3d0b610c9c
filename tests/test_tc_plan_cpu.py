"""Host-side work list of the tensor-core quartic kernel (no GPU needed).

For every size the kernel takes (1..80 pairs) the plan must cover each
(c1, c2, g) combination of the quartic topology exactly once with the right
link pair and Hamiltonian component, respect the tensor-memory limits
(n_cols = n_g * 16 ceil(N / 16) <= 256, a multiple of 16), and split the chunk
list of every 128-row tile into CTA ranges that partition it."""
import numpy as np
import pytest

import paper_1609_00077_gb300 as ppq
from paper_1609_00077_gb300 import tables as T


@pytest.fixture(scope="module")
def combos():
    t9 = T.t9_channels(T.Tables())
    p9 = sorted(set((int(a), int(b)) for a, b in t9[:, [0, 1]]))
    pi = {p: i for i, p in enumerate(p9)}
    q9 = sorted(set((pi[(int(a), int(b))], int(g)) for a, b, g in t9[:, [0, 1, 4]]))
    return p9, q9


@pytest.mark.parametrize("N", list(range(1, 81)))
def test_plan_covers_every_combination_once(N, combos):
    p9, q9 = combos
    ch, ct = ppq.tc_plan(N)
    npad = (N + 15) // 16 * 16
    seen = np.zeros(len(q9), dtype=int)
    for rec in ch:
        c1, c2, ng, ncols = (int(x) for x in rec[:4])
        assert 1 <= ng <= 4 and ncols == ng * npad and ncols <= 256 and ncols % 16 == 0
        for j in range(ng):
            g, q = int(rec[4 + j]), int(rec[8 + j])
            assert q9[q][1] == g and p9[q9[q][0]] == (c1, c2)
            seen[q] += 1
        assert not rec[4 + ng:8].any() and not rec[8 + ng:12].any()
    assert (seen == 1).all()
    P = N * (N - 1) // 2
    ntiles = (P + 127) // 128
    assert len(ct) <= 152 + ntiles
    for t in range(ntiles):
        rng = sorted((int(a), int(b)) for tt, a, b in ct if tt == t)
        assert rng[0][0] == 0 and rng[-1][1] == len(ch)
        assert all(b0 == a1 for (_, b0), (a1, _) in zip(rng, rng[1:]))
        assert all(a < b for a, b in rng)
    assert set(int(x) for x in ct[:, 0]) == set(range(ntiles))


def test_plan_rejects_sizes_out_of_range():
    for N in (0, 81, 200):
        with pytest.raises(ppq.PPQError):
            ppq.tc_plan(N)
