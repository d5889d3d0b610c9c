"""Write tests/golden/ph_c14h16_triple.npz: exact PH residual elements of one
label triple of PPP C14H16 (7 pairs, integrals truncated to three labels) at
seeded random amplitudes, from the oracle's local assembly (O-loc) alone.

At 7 pairs every coefficient of the label-subset inclusion-exclusion is
nonzero (K + K_H = 6 < 7), so these elements check the assembly of the
three-pair residual from local problems, not just one whole-system problem.
The elements with labels exactly M = {2, 3, 4} need the local problems of the
15 label sets L containing M with |L| <= 6; they are computed in parallel
processes.  Stored: the Hamiltonian (h, eri, e_const, pairing), the
amplitudes over the oracle's K = 3 manifold, and (manifold index, R) of every
element whose labels are M.

    python -m tests.golden.make_ph_triple_golden [--workers 8]
"""
import argparse
import itertools
import multiprocessing as mp
import os
import time

import numpy as np

from workloads import build_ppp
from oracle.detcc import truncated_hamiltonian, enumerate_manifold
from oracle.loccc import LocalAssembly

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ph_c14h16_triple.npz")
M = (2, 3, 4)
SEED = 1609003

_S = {}


def _one(sub):
    H, trunc, t = _S["H"], _S["trunc"], _S["t"]
    LA = LocalAssembly(None, None, H.occ_of_pair, H.vir_of_pair, K=3, K_H=3, subsets=[sub], truncated=trunc)
    R, _ = LA.residual(t)
    return R


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count())
    args = ap.parse_args()
    H = build_ppp('polyene', 14)
    N = H.n_pairs
    trunc = truncated_hamiltonian(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, 3)
    man = enumerate_manifold(H.occ_of_pair, H.vir_of_pair, 3)
    t = np.random.default_rng(SEED).uniform(-0.1, 0.1, len(man))
    others = [k for k in range(N) if k not in M]
    subs = [tuple(sorted(M + e)) for j in range(0, 4) for e in itertools.combinations(others, j)]
    assert len(subs) == 15
    _S.update(H=H, trunc=trunc, t=t)
    t0 = time.time()
    with mp.get_context("fork").Pool(min(args.workers, len(subs))) as pool:
        parts = pool.map(_one, sorted(subs, key=len, reverse=True))
    R = np.sum(parts, axis=0)
    lab = {}
    for k in range(N):
        lab[int(H.occ_of_pair[k])] = k
        lab[int(H.vir_of_pair[k])] = k
    idx = np.array([i for i, d in enumerate(man)
                    if {lab[x] for part in d for x in part} == set(M)], dtype=np.int64)
    np.savez_compressed(OUT, h=H.h, eri=H.eri, e_const=H.e_const, occ=H.occ_of_pair, vir=H.vir_of_pair,
                        t=t, idx=idx, R=R[idx], labels=np.array(M), seed=SEED)
    print(f"wrote {OUT}: {len(idx)} elements, max |R| {np.abs(R[idx]).max():.3e}, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
