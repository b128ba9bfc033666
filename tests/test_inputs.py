"""Seeded input generators: shapes of the paper's Si64 benchmark systems."""
import json
import os

import numpy as np
import pytest

from paper_2009_03559_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "si64_shell_counts.json")


def test_si64_shell_and_function_counts():
    """Paper Sec. 4: Si64 SZ = 128 shells / 256 functions, DZP = 320 / 832."""
    g = json.load(open(GOLD))
    sz = inputs.cluster_system(64, seed=1)
    assert sz.n_atoms == g["SZ"]["atoms"]
    assert sz.n_shells == g["SZ"]["shells"]
    assert sz.n_bf == g["SZ"]["functions"]
    dzp = inputs.diamond_system(64, seed=1)
    assert dzp.n_shells == g["DZP"]["shells"]
    assert dzp.n_bf == g["DZP"]["functions"]


def test_config_sizes():
    s0, p0 = inputs.config0()
    assert (s0.n_atoms, s0.n_shells, s0.n_bf) == (16, 32, 64)
    assert p0.shape == (64, 64)
    s1, p1 = inputs.config1()
    assert (s1.n_atoms, s1.n_shells, s1.n_bf) == (64, 320, 832)
    s3 = inputs.diamond_system(216, seed=3000)
    assert (s3.n_shells, s3.n_bf) == (1080, 2808)


def test_diamond_geometry():
    s = inputs.diamond_system(64, seed=5, jitter=0.0)
    d = np.linalg.norm(s.xyz[:, None] - s.xyz[None], axis=-1)
    d[np.diag_indices(64)] = np.inf
    assert np.isclose(d.min(), 10.26 * np.sqrt(3) / 4)  # nearest neighbour a*sqrt(3)/4
    # 2x2x2 conventional cells: extent a*(2 - 1/4) along each axis
    assert np.allclose(s.xyz.max(0) - s.xyz.min(0), 10.26 * 1.75)


def test_cluster_geometry_and_jitter():
    s = inputs.cluster_system(16, seed=0, jitter=0.0)
    assert np.allclose(s.xyz[:3], [[0, 0, 0], [0, 0, 2.5], [0, 0, 5.0]])
    sj = inputs.cluster_system(16, seed=0)
    assert np.abs(sj.xyz - s.xyz).max() <= 0.3


def test_exponents_and_weights():
    s = inputs.diamond_system(8, seed=3)
    a = s.alpha.reshape(-1, 3)
    assert np.all(np.diff(a, axis=1) <= 0)  # sorted descending within a shell
    assert a.min() >= 0.08 and a.max() <= 8.0
    assert s.coef.min() >= 0.1 and s.coef.max() < 1.0
    c = inputs.cluster_system(8, seed=3)
    assert c.alpha.min() >= 0.1 and c.alpha.max() <= 20.0


def test_density_matrix_projector():
    s, p = inputs.config0()
    assert np.allclose(p, p.T)
    assert np.allclose(p @ p, p, atol=1e-12)          # P = C C^T with orthonormal C
    assert np.isclose(np.trace(p), 32.0)


def test_density_truncation():
    s, p = inputs.config1(n_atoms=16)
    ba = s.bf_atom
    d = np.linalg.norm(s.xyz[:, None] - s.xyz[None], axis=-1)[ba][:, ba]
    assert np.all(p[d > 10.0] == 0.0)
    assert np.any(p[d <= 10.0] != 0.0)
    assert np.array_equal(p, p.T)


def test_determinism():
    a, pa = inputs.config0()
    b, pb = inputs.config0()
    assert np.array_equal(a.xyz, b.xyz) and np.array_equal(a.alpha, b.alpha)
    assert np.array_equal(pa, pb)


def test_batch_and_requests():
    sys_ = inputs.config2_systems(n_systems=4)
    assert len(sys_) == 4
    for s, p in sys_:
        assert 8 <= s.n_atoms <= 128 and p.shape == (s.n_bf, s.n_bf)
    systems, reqs = inputs.config4_requests(n_requests=50)
    assert len(systems) == 64 and len(reqs) == 50
    times = [r[0] for r in reqs]
    assert all(np.diff(times) > 0)
    assert all(16 <= n <= 512 for _, n, _ in systems)


def test_request_stream_statistics():
    """Poisson arrivals at 50/s: mean gap 1/50 s (2000 gaps: within 10 %); pool sizes are
    log-uniform in [16, 512] (median near sqrt(16*512) = 90.5); both generators occur."""
    systems, reqs = inputs.config4_requests()
    gaps = np.diff([0.0] + [t for t, _, _ in reqs])
    assert abs(gaps.mean() - 1 / 50) < 0.1 / 50
    assert 0.8 < gaps.std() / gaps.mean() < 1.2           # exponential: cv = 1
    sizes = np.array([n for _, n, _ in systems])
    assert 45 < np.median(sizes) < 180
    assert {k for k, _, _ in systems} == {"cluster", "diamond"}
    assert all(0 <= w < 64 for _, w, _ in reqs)
    assert len({sd for _, _, sd in reqs}) == len(reqs)     # a fresh P seed per request


def test_scaled_serving_pool_stays_in_range():
    systems, reqs = inputs.config4_requests(n_requests=64, n_hi=64)
    assert all(16 <= n <= 64 for _, n, _ in systems)
    assert len(reqs) == 64


def test_batch_of_32_matches_recipe():
    """32 systems, atom counts in 8..128, kind by coin; seeds 2000 + i; P per kind."""
    sys_ = inputs.config2_systems()
    assert len(sys_) == 32
    kinds = {s.kind for s, _ in sys_}
    assert kinds == {"cluster", "diamond"}
    for i, (s, p) in enumerate(sys_):
        assert s.seed == 2000 + i and 8 <= s.n_atoms <= 128
        assert np.allclose(p, p.T)
        if s.kind == "diamond":
            assert s.rcut == 6.0 and s.tau == 1e-8
        else:
            assert s.rcut == 0.0 and s.tau == 1e-10


def test_nao_set_shape_confinement_normalisation():
    """Synthetic radial functions: 2s 2p 1d per element, zero at and beyond the confining
    radius, value and slope going to zero there, unit norm on the grid, seeded."""
    rs = inputs.nao_set(3, seed=11)
    assert rs.phi.shape == (15, 512)
    assert list(rs.l) == [0, 0, 1, 1, 2] * 3
    r = rs.h * np.arange(1, 513)
    assert r[-1] == pytest.approx(rs.r_cut)
    assert np.all(rs.phi[:, -1] == 0.0)
    assert np.allclose((rs.phi ** 2 * r ** 2).sum(axis=1) * rs.h, 1.0)
    # near r_c the function vanishes quadratically (value and slope zero at the radius)
    tail = np.abs(rs.phi[:, -5:-1]).max(axis=1) / np.abs(rs.phi).max(axis=1)
    assert np.all(tail < 1e-3)
    again = inputs.nao_set(3, seed=11)
    assert np.array_equal(again.phi, rs.phi)
    assert not np.array_equal(inputs.nao_set(3, seed=12).phi, rs.phi)
