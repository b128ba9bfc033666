"""The lattice-sum oracle (Eq. vx with images) on explicit image clusters.  Pins: with the
images out of the orbital-cutoff range, K^0 is the home cell's molecular K and every other
K^G vanishes; a larger cluster leaves K^G unchanged (the contributing cells are all in);
K^G and K^{-G} are transposes of each other (the exchange operator is symmetric); and
the cluster K is translation invariant between interior cells."""
import numpy as np
import pytest

import oracle
import oracle.periodic as op
from paper_2009_03559_gb300 import inputs

G_LIST = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (1, 1, 0)]


@pytest.fixture(scope="module")
def crystal():
    ps = inputs.periodic_sc()
    P_R = inputs.periodic_density(ps, r_cells=2, seed=77, truncate_bohr=10.0)
    return ps, P_R


def test_density_blocks_are_symmetric(crystal):
    ps, P_R = crystal
    for R, blk in P_R.items():
        mR = tuple(-x for x in R)
        assert np.array_equal(blk, P_R[mR].T)


def test_isolated_images_give_the_molecular_K():
    ps = inputs.periodic_sc(spacing=40.0)
    P_R = inputs.periodic_density(ps, r_cells=1, seed=78)
    K = op.periodic_K(ps, P_R, G_LIST, r_cluster=1)
    Kmol, _ = oracle.Screen(oracle.Basis(ps.cell)).build_K(P_R[(0, 0, 0)], "sym")
    assert np.abs(K[(0, 0, 0)] - Kmol).max() <= 1e-13
    for G in G_LIST[1:]:
        assert np.abs(K[G]).max() == 0.0


def test_cluster_covers_every_contribution(crystal):
    ps, P_R = crystal
    r = op.contributing_range(ps, 1)
    K1 = op.periodic_K(ps, P_R, G_LIST, r_cluster=r)
    K2 = op.periodic_K(ps, P_R, G_LIST, r_cluster=r + 1)
    for G in G_LIST:
        assert np.abs(K1[G] - K2[G]).max() <= 1e-12
    assert np.abs(K1[(1, 0, 0)]).max() > 1e-6  # neighbouring cells do couple


def test_opposite_cells_are_transposes(crystal):
    ps, P_R = crystal
    K = op.periodic_K(ps, P_R, G_LIST)
    assert np.abs(K[(1, 0, 0)] - K[(-1, 0, 0)].T).max() <= 1e-12
    assert np.abs(K[(0, 0, 0)] - K[(0, 0, 0)].T).max() <= 1e-12


def test_translation_invariance_of_the_cluster(crystal):
    ps, P_R = crystal
    r = op.contributing_range(ps, 1) + 1
    cells, Kc, nb = op.cluster_K(ps, P_R, r)
    i0, j0 = cells.index((0, 0, 0)), cells.index((1, 0, 0))
    i1, j1 = cells.index((0, 1, 0)), cells.index((1, 1, 0))   # the same pair shifted by (0,1,0)
    b0 = Kc[i0 * nb:(i0 + 1) * nb, j0 * nb:(j0 + 1) * nb]
    b1 = Kc[i1 * nb:(i1 + 1) * nb, j1 * nb:(j1 + 1) * nb]
    assert np.abs(b0 - b1).max() <= 1e-12
