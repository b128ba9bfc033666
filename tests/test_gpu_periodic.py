"""GPU lattice sums of the exchange matrix (Eq. vx with images, list-IJ in the home cell,
Sec. 3.1) against the image-cluster oracle: K^G for several cells G, element by element at
1e-10, on simple-cubic crystals with s and p shells and with the s, s, p, p, d shell set
(every quartet class)."""
import numpy as np
import pytest
import torch

import oracle.periodic as op
from paper_2009_03559_gb300 import inputs

pytestmark = pytest.mark.gpu

G_LIST = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (1, 1, 0), (0, 0, -1)]


@pytest.fixture(scope="module")
def hfx_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_03559_gb300 import hfx
    return hfx


def check(hfx_mod, ps, P_R, G_list, tol=1e-10):
    Kref = op.periodic_K(ps, P_R, G_list)
    h = hfx_mod.Periodic(ps).build_pairs()
    K = h.build_K(P_R, G_list)
    worst = 0.0
    for G in G_list:
        d = np.abs(K[tuple(G)].cpu().numpy() - Kref[tuple(G)]).max()
        worst = max(worst, d)
        assert d <= tol, (G, d)
    assert max(np.abs(Kref[tuple(G)]).max() for G in G_list[1:]) > 1e-6  # images do couple
    h.close()
    return worst


def test_simple_cubic(hfx_mod):
    ps = inputs.periodic_sc()
    P_R = inputs.periodic_density(ps, r_cells=2, seed=77, truncate_bohr=10.0)
    check(hfx_mod, ps, P_R, G_LIST)


def test_d_shells(hfx_mod):
    """One atom per cell with the diamond workload's shell set s, s, p, p, d: every quartet
    class, in both the forward and the translated (lower bra class) launches."""
    ps = inputs.periodic_sc(shells=(0, 0, 1, 1, 2), a=7.0, rcut=3.0, tau=1e-10)
    P_R = inputs.periodic_density(ps, r_cells=1, seed=79, truncate_bohr=8.0)
    check(hfx_mod, ps, P_R, [(0, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 1)])


def test_isolated_images_give_the_molecular_K(hfx_mod):
    """With the images beyond the cutoff, K^0 is the home cell's molecular K (the molecular
    GPU path) and K^G = 0 for G != 0."""
    ps = inputs.periodic_sc(spacing=40.0)
    P_R = inputs.periodic_density(ps, r_cells=1, seed=78)
    h = hfx_mod.Periodic(ps).build_pairs()
    K = h.build_K(P_R, [(0, 0, 0), (1, 0, 0)])
    m = hfx_mod.HFX(ps.cell).build_pairs()
    Km = m.build_K(torch.from_numpy(P_R[(0, 0, 0)]).cuda())
    assert torch.abs(K[(0, 0, 0)] - Km).max().item() <= 1e-13
    assert torch.abs(K[(1, 0, 0)]).max().item() == 0.0


def test_missing_density_blocks_contribute_nothing(hfx_mod):
    """Only the density blocks given enter: dropping P^R for |R| = 2 changes K^G exactly as the
    oracle with the same reduced set."""
    ps = inputs.periodic_sc()
    P_R = inputs.periodic_density(ps, r_cells=2, seed=80, truncate_bohr=10.0)
    P_R = {R: v for R, v in P_R.items() if max(abs(x) for x in R) <= 1}
    check(hfx_mod, ps, P_R, [(0, 0, 0), (1, 0, 0)])
