"""Pins of the oracle's exchange matrix (paper Eq. vx, one cell, no images, no -1/2).

* the plain four-fold loop (the definition) and the symmetric canonical loop (eight-fold
  symmetry with degeneracy factors, then K + K^T) agree;
* K is symmetric; for an untruncated P = C C^T, K is positive semi-definite and
  E_K = tr(PK) >= 0 (K = sum_i Gram matrix of mu*phi_i under a positive-definite kernel);
* dropping quartets by Schwarz changes K by no more than the sum of their bounds;
* the quartet counts equal a direct count from the exported screening data;
* the compensated trace equals math.fsum of the products;
* sampled K blocks equal the full build.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2009_03559_gb300 import inputs


@pytest.fixture(scope="module")
def cfg0():
    s, P = inputs.config0()
    B = oracle.Basis(s)
    S = oracle.Screen(B)
    K, ek = S.build_K(P, "sym")
    return s, P, B, S, K, ek


def test_plain_equals_symmetric_cluster(cfg0):
    s, P, B, S, K, ek = cfg0
    K2, ek2 = S.build_K(P, "plain")
    assert np.abs(K - K2).max() <= 1e-13
    assert ek == pytest.approx(ek2, abs=1e-12)


def test_plain_equals_symmetric_diamond():
    s, P = inputs.config1(n_atoms=4)
    B = oracle.Basis(s)
    S = oracle.Screen(B)
    K1, e1 = S.build_K(P, "plain")
    K2, e2 = S.build_K(P, "sym")
    assert np.abs(K1 - K2).max() <= 1e-13
    assert e1 == pytest.approx(e2, abs=1e-12)


def test_symmetric_and_psd(cfg0):
    s, P, B, S, K, ek = cfg0
    assert np.array_equal(K, K.T)
    assert np.linalg.eigvalsh(K).min() > -1e-12
    assert ek > 0


def test_trace_compensated(cfg0):
    s, P, B, S, K, ek = cfg0
    assert ek == pytest.approx(math.fsum((P * K).ravel()), rel=1e-15)
    assert oracle.trace_PK(P, K) == ek


def test_counts_match_screening_data(cfg0):
    s, P, B, S, K, ek = cfg0
    Q, cut, kept, qmax = S.export()
    n = s.n_shells
    pairs = [(I, J) for I in range(n) for J in range(I + 1) if kept[I, J]]
    qv = np.array([Q[I, J] for I, J in pairs])
    idx = {p: i for i, p in enumerate(pairs)}
    cnt = 0
    for a, (I, J) in enumerate(pairs):
        ij = I * (I + 1) // 2 + J
        for b, (Kk, L) in enumerate(pairs):
            kl = Kk * (Kk + 1) // 2 + L
            if kl <= ij and qv[a] * qv[b] >= S.tau:
                cnt += 1
    assert cnt == S.count_quartets()[21]
    assert S.count_quartets()[:21].sum() == cnt


def test_pair_screen_rule():
    """Pair kept iff cutoff passes and Q_IJ * Q_max >= tau; cutoff = 2 r_c between atoms."""
    s = inputs.diamond_system(16, seed=1001, tau=1e-8, rcut=6.0)
    B = oracle.Basis(s)
    S = oracle.Screen(B)
    Q, cut, kept, qmax = S.export()
    d = np.linalg.norm(s.xyz[:, None] - s.xyz[None], axis=-1)
    sa = s.shell_atom
    dd = d[sa][:, sa]
    assert np.array_equal(cut, (dd < 12.0) | (sa[:, None] == sa[None, :]))
    assert np.array_equal(kept, cut & (Q * qmax >= 1e-8))
    assert qmax == pytest.approx(Q[cut].max())


def test_schwarz_drop_bound():
    s, P = inputs.config1(n_atoms=8)
    B = oracle.Basis(s)
    S0 = oracle.Screen(B, tau=0.0)
    St = oracle.Screen(B, tau=1e-4)
    K0, _ = S0.build_K(P, "sym")
    Kt, _ = St.build_K(P, "sym")
    Q, cut, kept, qmax = S0.export()
    _, _, kept_t, _ = St.export()
    n = s.n_shells
    # each dropped ordered quartet moves any K element by at most Q_IJ Q_KL max|P|
    dropped = 0.0
    for I in range(n):
        for J in range(n):
            if not cut[I, J]:
                continue
            for K_ in range(n):
                for L in range(n):
                    if not cut[K_, L]:
                        continue
                    keep = kept_t[I, J] and kept_t[K_, L] and Q[I, J] * Q[K_, L] >= 1e-4
                    if not keep:
                        dropped += Q[I, J] * Q[K_, L]
    diff = np.abs(K0 - Kt).max()
    assert diff > 0
    assert diff <= dropped * np.abs(P).max()


def test_K_blocks_match_full(cfg0):
    s, P, B, S, K, ek = cfg0
    off = s.shell_offset
    nb = s.shell_nbf
    rng = np.random.default_rng(3)
    for _ in range(12):
        I, Kk = rng.integers(0, s.n_shells, 2)
        blk = S.K_block(P, I, Kk)
        ref = K[off[I]:off[I] + nb[I], off[Kk]:off[Kk] + nb[Kk]]
        assert np.abs(blk - ref).max() <= 1e-13


def test_psd_for_diamond_untruncated():
    s = inputs.diamond_system(6, seed=55)
    P = inputs.density_matrix(s)
    S = oracle.Screen(oracle.Basis(s), tau=0.0)
    K, ek = S.build_K(P, "sym")
    assert np.linalg.eigvalsh(K).min() > -1e-12 * np.abs(K).max()
    assert ek > 0
