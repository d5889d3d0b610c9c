"""Exact residual elements of a few pairs at large N from the oracle's local
assembly, spread over processes (test infrastructure).

The elements of the pair (Y, Z) need the local problems of every label set
L containing Y and Z with |L| <= K + K_H (PQ: 1 + (N-2) + C(N-2, 2) of them,
2347 at N = 70).  They are independent, so a fork pool shares them out; the
truncated integrals are computed once before the fork and shared copy-on-write.
A fork is only safe in a process that has not initialised CUDA, so GPU tests
run this module as a command in a fresh process:

    python -m tests.oloc_sampled --kind polyene --size 140 --orbitals local \\
        --pairs 33,34 68,69 --tag 0 --workers 16 --out sampled.npz

The amplitudes are uniform(-0.1, 0.1) over the oracle's manifold from
random_pair_amplitude_seed(N, tag), so the caller can draw the same ones, or
are read from --t-in.  The output holds the manifold indices of the sampled
pairs' elements and their exact residual values, the reference energy and
constant and, with --energy, the correlation energy at those amplitudes.
"""
import argparse
import multiprocessing as mp
import os
from itertools import combinations

import numpy as np

from workloads import (build_ppp, build_hchain, random_pair_amplitude_seed, polyene_geometry,
                       acene_geometry, ppp_site_hamiltonian, mo_integrals, Hamiltonian)
from oracle.detcc import truncated_hamiltonian, enumerate_manifold
from oracle.loccc import LocalAssembly

_SHARED = {}


def pair_subsets(N, pairs, kmax):
    """Every label set containing one of the pairs, with at most kmax labels."""
    subs = set()
    for Y, Z in pairs:
        others = [k for k in range(N) if k not in (Y, Z)]
        for m in range(0, kmax - 1):
            for extra in combinations(others, m):
                subs.add(tuple(sorted((Y, Z) + extra)))
    return sorted(subs)


def _chunk_residual(subsets):
    d = _SHARED
    L = LocalAssembly(None, None, d["occ"], d["vir"], d["K"], d["K_H"], subsets=subsets,
                      truncated=d["truncated"])
    return L.residual(d["t"])


def sampled_residual(h, eri, occ, vir, pairs, t, K=2, K_H=2, workers=2, energy=False):
    """(indices, values, e_c, e_ref): the oracle's residual elements of the
    given pairs at amplitudes t (over the oracle's manifold), exact; with
    energy=True also the correlation energy at t (every label set of at most
    K_H labels is added), else None; e_ref is the reference energy without
    the constant.  Uses a fork pool."""
    occ = np.asarray(occ)
    vir = np.asarray(vir)
    truncated = truncated_hamiltonian(h, eri, occ, vir, K_H)
    subsets = set(pair_subsets(len(occ), pairs, K + K_H))
    if energy:
        for m in range(1, K_H + 1):
            subsets.update(combinations(range(len(occ)), m))
    subsets = sorted(subsets)
    _SHARED.update(occ=occ, vir=vir, K=K, K_H=K_H, truncated=truncated, t=np.asarray(t, float))
    chunks = [subsets[i::workers] for i in range(workers)]
    try:
        with mp.get_context("fork").Pool(workers) as pool:
            parts = pool.map(_chunk_residual, [c for c in chunks if c])
    finally:
        _SHARED.clear()
    R = sum(p[0] for p in parts)
    e_c = sum(p[1] for p in parts) if energy else None
    probe = LocalAssembly(None, None, occ, vir, K, K_H, subsets=[], truncated=truncated)
    want = [set(p) for p in pairs]
    idx = np.array([k for k, d in enumerate(probe.manifold) if probe._labels(d) in want], dtype=np.int64)
    return idx, R[idx], e_c, truncated[3]


def workload(kind, size, orbitals, orbitals_from=None):
    """The Hamiltonian; with orbitals_from (an .npz of C, occ_of_pair,
    vir_of_pair written by the caller) a PPP model is transformed with the
    caller's own orbitals instead of re-running RHF and the localisation: a
    phase chosen by argmax can differ between processes when two coefficients
    of an orbital agree to ~1e-11, and that would flip the sign convention of
    the amplitudes."""
    if orbitals_from is not None:
        if kind not in ("polyene", "acene"):
            raise ValueError("orbitals_from needs a PPP model")
        xyz, bonds = polyene_geometry(size) if kind == "polyene" else acene_geometry(size)
        h_site, gamma, e_const = ppp_site_hamiltonian(xyz, bonds)
        d = np.load(orbitals_from)
        h, eri = mo_integrals(d["C"], h_site, gamma_zdo=gamma)
        return Hamiltonian(f"PPP {kind} {size} (given orbitals)", h, eri, e_const,
                           d["occ_of_pair"], d["vir_of_pair"])
    if kind == "hchain":
        return build_hchain(size, 1.5, orbitals=orbitals)
    return build_ppp(kind, size, orbitals=orbitals)


def save_orbitals(path, H):
    """Write H's orbitals and pairing for workload(..., orbitals_from=path)."""
    np.savez(path, C=H.C, occ_of_pair=H.occ_of_pair, vir_of_pair=H.vir_of_pair)


def amplitudes(n_amp, N, tag):
    return np.random.default_rng(random_pair_amplitude_seed(N, tag)).uniform(-0.1, 0.1, n_amp)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--kind", default="polyene")
    ap.add_argument("--size", type=int, required=True)
    ap.add_argument("--orbitals", default="canonical")
    ap.add_argument("--pairs", nargs="+", required=True, help="Y,Z label pairs")
    ap.add_argument("--tag", type=int, default=0)
    ap.add_argument("--K", type=int, default=2)
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--orbitals-from", default=None, help="C and pairing of the caller (.npz)")
    ap.add_argument("--t-in", default=None, help="amplitudes over the oracle's manifold (.npy)")
    ap.add_argument("--energy", action="store_true", help="also the correlation energy at t")
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)
    H = workload(a.kind, a.size, a.orbitals, a.orbitals_from)
    pairs = [tuple(int(x) for x in p.split(",")) for p in a.pairs]
    if a.t_in:
        t = np.load(a.t_in)
    else:
        t = amplitudes(len(enumerate_manifold(H.occ_of_pair, H.vir_of_pair, a.K)), H.n_pairs, a.tag)
    idx, vals, e_c, e_ref = sampled_residual(H.h, H.eri, H.occ_of_pair, H.vir_of_pair, pairs, t,
                                             K=a.K, K_H=a.K, workers=a.workers, energy=a.energy)
    np.savez(a.out, idx=idx, vals=vals, e_c=np.nan if e_c is None else e_c, e_ref=e_ref,
             e_const=H.e_const)


if __name__ == "__main__":
    main()
