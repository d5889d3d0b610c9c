"""The generated tables, interpreted on the CPU, against the oracle.

`tests/table_interp.py` evaluates the residual and energy the way the device
kernels use the tables of `tables.emit_header` (staging, links, site and
pair closures, topologies T1-T9, the exp(-T_YZ) transform, the assembly).
At random amplitudes (uniform +-0.1, zero diagonal, consistent pair copies)
its residual must equal the oracle's determinant-space residual element by
element and its energy the oracle's energy, to FP64 rounding (1e-12).  N = 4
is the smallest size where every topology, the quartic one included, is
non-zero.  This pins the table generator without a GPU.
"""
import numpy as np
import pytest

from workloads import build_ppp, build_hchain, random_pair_amplitude_seed
from oracle.detcc import Problem
import paper_1609_00077_gb300 as ppq
from tests.layout import LayoutMap
from tests.table_interp import Header, residual

SYSTEMS = {
    "H4": lambda: build_hchain(4, 1.5),
    "C6H8": lambda: build_ppp('polyene', 6),
    "C8H10": lambda: build_ppp('polyene', 8),
}


@pytest.fixture(scope="module")
def header():
    return Header()


def _layout_desc(hd):
    return hd.i("ppq_layout_desc").reshape(-1, 3)


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_interpreted_tables_match_oracle(name, header):
    H = SYSTEMS[name]()
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=2)
    man = P.cc.manifold
    lm = LayoutMap(man, H.occ_of_pair, H.vir_of_pair, H.n_orb, _layout_desc(header))
    rng = np.random.default_rng(random_pair_amplitude_seed(H.n_pairs, 11))
    t = rng.uniform(-0.1, 0.1, len(man))
    R_ref, e_ref = P.residual(t)
    r, e = residual(header, H.h, H.eri, H.occ_of_pair, H.vir_of_pair, lm.to_layout(t))
    assert lm.mirror_error(r) < 1e-14
    assert np.abs(lm.from_layout(r) - R_ref).max() < 1e-12
    assert abs(e - e_ref) < 1e-12


def test_layout_descriptor_matches_the_library(header):
    # the interpreter and the C ABI describe the same 32 channels
    try:
        desc = ppq.amp_layout()
    except ppq.PPQError:
        pytest.skip("libppq.so not built")
    assert (desc == _layout_desc(header)).all()
