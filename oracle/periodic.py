"""Oracle for the lattice sums of the exchange matrix (paper Sec. 2, Eq. vx), by their
definition on an explicit cluster of images.  TEST INFRASTRUCTURE ONLY (like the rest of
oracle/): nothing in the CUDA library uses it.

Eq. vx (without its -1/2):  K^G_{mu lambda} = sum_{nu sigma} sum_{N,H} P^{H-N}_{nu sigma}
(mu^0 nu^N | lambda^G sigma^H), mu and lambda in the home cell, nu^N in cell N, sigma^H in
cell H.  With the orbital cutoff only finitely many cells N, H contribute to a given G, so
the sum is the molecular exchange matrix of the finite cluster of those cells, with the
block-Toeplitz density P_cl[(nu,N),(sigma,H)] = P^{H-N}_{nu sigma}: K^G is the cluster
K's block (home cell, cell G).  The molecular oracle (Screen.build_K) is pinned elsewhere;
the screening is the same (pair Q and Q_max are translation invariant)."""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import Basis, Screen


def cells_within(r: int):
    return [c for c in itertools.product(range(-r, r + 1), repeat=3)]


def contributing_range(ps, g_max: int) -> int:
    """Cells (in every direction) needed for K^G with |G_i| <= g_max: pairs reach at most
    2 r_c plus a cell diagonal beyond the cell of their first function."""
    c = ps.cell
    edge = float(np.min(np.diag(ps.lattice)))
    reach = 2.0 * c.rcut + np.linalg.norm(np.ptp(c.xyz, axis=0))
    return g_max + int(math.ceil(reach / edge))


def cluster_K(ps, P_R: dict, r_cluster: int):
    """Molecular K of the image cluster with cells |n_i| <= r_cluster; returns (cells,
    K_cl, n_bf of the home cell).  Density blocks missing from P_R are zero."""
    from paper_2009_03559_gb300 import inputs
    cells = cells_within(r_cluster)
    sysc = inputs.image_system(ps, cells)
    nb = ps.cell.n_bf
    Pcl = np.zeros((nb * len(cells), nb * len(cells)))
    for a, N in enumerate(cells):
        for b, H in enumerate(cells):
            R = tuple(h - n for h, n in zip(H, N))
            if R in P_R:
                Pcl[a * nb:(a + 1) * nb, b * nb:(b + 1) * nb] = P_R[R]
    S = Screen(Basis(sysc))
    K, _ = S.build_K(Pcl, "sym")
    return cells, K, nb


def periodic_K(ps, P_R: dict, G_list, r_cluster: int | None = None) -> dict:
    """K^G (n_bf x n_bf) for every cell G in G_list."""
    g_max = max(max(abs(x) for x in G) for G in G_list)
    r = contributing_range(ps, g_max) if r_cluster is None else r_cluster
    cells, K, nb = cluster_K(ps, P_R, r)
    i0 = cells.index((0, 0, 0))
    out = {}
    for G in G_list:
        j = cells.index(tuple(G))
        out[tuple(G)] = K[i0 * nb:(i0 + 1) * nb, j * nb:(j + 1) * nb].copy()
    return out
