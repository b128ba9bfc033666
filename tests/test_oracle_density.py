"""Density-weighted screening in the oracle (a next step beyond the exact-zero skip):
a canonical quartet is kept only if also Q_IJ Q_KL Pmax >= dens_tau, Pmax the largest |P|
over the density blocks its K updates multiply.  Pins: the plain four-fold loop and the
symmetric loop apply the rule identically; dens_tau = 0 is the unscreened build; the change
of K is bounded by the dropped quartets' Schwarz-times-density bounds."""
import numpy as np
import pytest

import oracle
from paper_2009_03559_gb300 import inputs


def dropped_bound(S, pm, dens_tau):
    """sum over dropped canonical quartets of 2 * n_b * n_d * Q_IJ Q_KL Pmax: each dropped
    quartet changes any element of K = A + A^T by at most that much."""
    Q, cut, kept, qmax = S.export()
    l = S.basis.shell_l
    nsph = np.array([2 * int(x) + 1 for x in l])
    I, J = np.nonzero(np.tril(kept))
    total = 0.0
    n_drop = 0
    for p in range(len(I)):
        a, b = I[p], J[p]
        K, L = I[: p + 1], J[: p + 1]
        qq = Q[a, b] * Q[K, L]
        ok = qq >= S.tau
        pmx = np.maximum.reduce([pm[b, L], pm[b, K], pm[a, L], pm[a, K]])
        drop = ok & (qq * pmx < dens_tau)
        n_drop += int(drop.sum())
        width = np.maximum(nsph[b] * nsph[L], nsph[a] * nsph[K])
        total += float((2 * width * qq * pmx)[drop].sum())
    return total, n_drop


@pytest.fixture(scope="module")
def case():
    s, P = inputs.config1(4)
    S = oracle.Screen(oracle.Basis(s))
    return s, P, S


def test_zero_threshold_is_the_plain_build(case):
    s, P, S = case
    K0, e0 = S.build_K(P, "sym")
    K1, e1, pm = S.build_K_dens(P, 0.0, "sym")
    # same quartets; the OpenMP threads' shares (and so the summation order) may differ
    assert np.abs(K0 - K1).max() <= 1e-13 and abs(e0 - e1) <= 1e-12
    # block maxima
    off = np.concatenate([[0], np.cumsum(s.shell_nbf)])
    I, J = 3, 7
    assert pm[I, J] == np.abs(P[off[I]:off[I + 1], off[J]:off[J + 1]]).max()


def test_plain_and_symmetric_loops_agree(case):
    s, P, S = case
    Kp, ep, _ = S.build_K_dens(P, 1e-4, "plain")
    Ks, es, _ = S.build_K_dens(P, 1e-4, "sym")
    assert np.abs(Kp - Ks).max() <= 1e-12
    assert abs(ep - es) <= 1e-10


@pytest.mark.parametrize("dens_tau", [1e-8, 1e-5, 1e-3])
def test_change_within_dropped_bound(case, dens_tau):
    s, P, S = case
    K0, e0 = S.build_K(P, "sym")
    K1, e1, pm = S.build_K_dens(P, dens_tau, "sym")
    bound, n_drop = dropped_bound(S, pm, dens_tau)
    dk = np.abs(K1 - K0).max()
    assert dk <= bound + 1e-13
    if dens_tau >= 1e-5:
        assert n_drop > 0 and dk > 0.0
    assert np.array_equal(K1, K1.T)
