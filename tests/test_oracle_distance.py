"""Pins of the distance-aware screening rule (hfx_oracle.c, ora_dist_estimate / ora_build_K_dist):
with the threshold 0 it is the unscreened build; the plain and the symmetric loops agree under
it; on two groups of atoms far apart the estimate Q_IJ Q_KL exp(-kappa rho R^2) is above the
true largest |(mu nu|lambda sigma)| of every cross quartet; and so the change of K it causes is
bounded by the estimates of the quartets it drops."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2009_03559_gb300 import inputs


def two_groups(gap=18.0):
    """Two copies of a 3-atom diamond piece (s, s, p, p, d shells), the second shifted by
    `gap` bohr along x: every pair within a group, every cross quartet far apart."""
    s = inputs.diamond_system(3, seed=31, tau=1e-12, rcut=0.0)
    n = s.n_atoms
    xyz = np.concatenate([s.xyz, s.xyz + np.array([gap, 0.0, 0.0])])
    sys2 = inputs.System("two3", xyz, np.concatenate([s.shell_atom, s.shell_atom + n]).astype(np.int32),
                         np.tile(s.shell_l, 2), np.tile(s.shell_nprim, 2), np.tile(s.alpha, 2), np.tile(s.coef, 2),
                         omega=s.omega, tau=1e-12, rcut=0.0, seed=s.seed, kind="diamond")
    return sys2, s.n_shells


@pytest.fixture(scope="module")
def setup():
    s, ns1 = two_groups()
    B = oracle.Basis(s)
    S = oracle.Screen(B, tau=1e-12, rcut=0.0)
    P = inputs.density_matrix(s, seed=5)
    return s, ns1, B, S, P


def test_zero_threshold_is_the_plain_build(setup):
    s, ns1, B, S, P = setup
    K0, e0 = S.build_K(P, "sym")
    K1, e1 = S.build_K_dist(P, 0.0, "sym")
    # the same quartets; only the order of the threads' partial sums may differ
    assert np.abs(K0 - K1).max() <= 1e-14 and abs(e0 - e1) <= 1e-13


def test_plain_and_symmetric_loops_agree(setup):
    s, ns1, B, S, P = setup
    Kp, _ = S.build_K_dist(P, 1e-6, "plain")
    Ks, _ = S.build_K_dist(P, 1e-6, "sym")
    assert np.abs(Kp - Ks).max() <= 1e-13


def test_estimate_bounds_every_cross_quartet(setup):
    """Every (IJ|KL) with both shells of IJ in one group and both of KL in the other."""
    s, ns1, B, S, P = setup
    n = s.n_shells
    worst, n_below_schwarz = 0.0, 0
    Q = S.export()[0]
    for I, J in itertools.combinations_with_replacement(range(ns1), 2):
        for K, L in itertools.combinations_with_replacement(range(ns1, n), 2):
            v = np.abs(B.quartet(J, I, L, K)).max()
            est = S.dist_estimate(J, I, L, K)
            worst = max(worst, v / est)
            n_below_schwarz += est < 0.5 * Q[I, J] * Q[K, L]
    assert worst <= 1.0, worst
    assert n_below_schwarz > 100  # the decay factor does bite at this distance


def test_dropped_quartets_bound_the_change(setup):
    """|K_tau - K_0| <= sum over dropped quartets of 2 * (largest block) * estimate * max|P|,
    the same argument as for the Schwarz drop bound with the estimate in place of Q Q."""
    s, ns1, B, S, P = setup
    tau = 1e-7
    K0, _ = S.build_K(P, "sym")
    Kt, _ = S.build_K_dist(P, tau, "sym")
    n = s.n_shells
    # all estimates at once from the exported pair data (the formula of ora_dist_estimate),
    # checked against the oracle's own value on a few quartets
    Q = S.export()[0]
    pst, pexp = S.export_dist()
    iu = np.tril_indices(n)
    c, sp, pe, q = pst[iu][:, :3], pst[iu][:, 3], pexp[iu], Q[iu]
    r = np.linalg.norm(c[:, None, :] - c[None, :, :], axis=-1) - sp[:, None] - sp[None, :]
    r = np.maximum(r, 0.0)
    rho = pe[:, None] * pe[None, :] / (pe[:, None] + pe[None, :])
    om2 = s.omega ** 2
    est = q[:, None] * q[None, :] * np.exp(-om2 * rho / (om2 + rho) * r * r)
    for a, b in ((0, 5), (17, 200), (300, 31)):
        ref = S.dist_estimate(iu[0][a], iu[1][a], iu[0][b], iu[1][b])
        assert abs(est[a, b] - ref) <= 1e-14 * ref
    tri = np.tril(np.ones(est.shape, dtype=bool))   # canonical pair-of-pairs order
    bound = 25.0 * est[(est < tau) & tri].sum()
    dk = np.abs(Kt - K0).max()
    assert 0.0 < dk <= 8 * bound * np.abs(P).max()
