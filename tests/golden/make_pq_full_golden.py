"""Write tests/golden/pq_full_c14h16.npz: the PQ residual with untruncated
two-electron integrals (K = 2, K_H = FULL) of PPP C14H16 (7 pairs) at seeded
random amplitudes, from the oracle's full determinant-space evaluation
(O-det, 11.8 M determinants) alone.

With untruncated integrals a linked term carries up to K + 4 = 6 labels, so
at 7 pairs every subset size of the label-subset expansion enters; these
values pin that expansion (and the oracle's own local assembly) where O-det is
the only other exact evaluator.  Stored: h, eri, e_const, the pairing, the
amplitudes over the oracle's K = 2 manifold, R and E_c.

    python -m tests.golden.make_pq_full_golden
"""
import os
import time

import numpy as np

from workloads import build_ppp
from oracle.detcc import Problem

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pq_full_c14h16.npz")
SEED = 1609004


def main():
    H = build_ppp('polyene', 14)
    t0 = time.time()
    P = Problem(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, K=2, K_H=-1)
    t = np.random.default_rng(SEED).uniform(-0.1, 0.1, P.cc.n_amp)
    R, e = P.residual(t)
    np.savez_compressed(OUT, h=H.h, eri=H.eri, e_const=H.e_const, occ=H.occ_of_pair, vir=H.vir_of_pair,
                        t=t, R=R, e_corr=e, seed=SEED)
    print(f"wrote {OUT}: {len(R)} elements, max |R| {np.abs(R).max():.3e}, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
