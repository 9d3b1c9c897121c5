"""Shared test helpers: oracle systems built from lattices, and cut-out neighbourhoods."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_1310_6143_gb300.lattice import SpinLattice


def oracle_system(lat: SpinLattice, alpha=0.1, dt=1e-16, H=(0.0, 0.0, 0.0), seed=1, sys_id=0, ids=None,
                  gamma=1.76e11) -> O.OracleSystem:
    return O.OracleSystem(lat.row_ptr, lat.col, lat.J, lat.mu_s, lat.k_u, lat.easy_axis, lat.K_neel,
                          alpha=alpha, dt=dt, gamma=gamma, H_app=tuple(H), seed=seed, sys_id=sys_id, ids=ids)


def neighbourhood(lat: SpinLattice, centres: np.ndarray, hops: int):
    """Sites within `hops` bonds of `centres`, and the induced sub-lattice on them.

    Returns (sites, sub) with sub a SpinLattice whose site k is lat's site sites[k]; rows
    of sites at distance < hops are complete, so a one-step Heun update of the centres
    (which needs their neighbours' predictor values) is exact when hops >= 2.
    """
    sites = set(int(c) for c in centres)
    frontier = set(sites)
    rp, col = lat.row_ptr, lat.col
    for _ in range(hops):
        nxt = set()
        for i in frontier:
            nxt.update(int(j) for j in col[rp[i]:rp[i + 1]])
        nxt -= sites
        sites |= nxt
        frontier = nxt
    sites = np.array(sorted(sites), dtype=np.int64)
    local = {int(g): k for k, g in enumerate(sites)}
    row_ptr = [0]
    cols, Js = [], []
    for g in sites:
        for k in range(rp[g], rp[g + 1]):
            j = int(col[k])
            if j in local:
                cols.append(local[j])
                Js.append(lat.J[k])
        row_ptr.append(len(cols))
    sub = SpinLattice(np.array(row_ptr, dtype=np.int64), np.array(cols, dtype=np.int32), np.array(Js),
                      lat.mu_s[sites], lat.k_u[sites], lat.easy_axis[sites],
                      None if lat.K_neel is None else lat.K_neel[sites])
    return sites, sub
