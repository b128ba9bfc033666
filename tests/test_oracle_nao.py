"""Pins of the NAO2GTO oracle (oracle/nao2gto.py; paper Sec. "NAO2GTO scheme" and Algorithm 1)
against things other than itself: published SplitMix64 outputs, the residual written out by
hand, the closed-form one-Gaussian least-squares fit, the least-squares optimality of the
projected coefficients, central finite differences of the residual (Jacobian), exact recovery of
a target that is itself a sum of Gaussians, the Karush-Kuhn-Tucker condition at an active bound,
stationarity of a converged fit, and the bookkeeping of Algorithm 1."""
import json
import math
import os

import numpy as np
import pytest

from oracle import nao2gto as N
from paper_2009_03559_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_outputs():
    g = json.load(open(os.path.join(GOLD, "splitmix64.json")))
    for case in g["cases"]:
        want = case.get("outputs") or [int(x, 16) for x in case["outputs_hex"]]
        got = [N.splitmix64(case["seed"], c) for c in range(len(want))]
        assert got == want


def test_uniform_is_top_53_bits():
    u = N.uniform(0, 0)
    assert u == (0xE220A8397B1DCDAF >> 11) / 2.0 ** 53
    us = [N.uniform(99, c) for c in range(2000)]
    assert min(us) >= 0.0 and max(us) < 1.0
    assert abs(np.mean(us) - 0.5) < 0.03


def test_err_written_out():
    rs = inputs.nao_set(1, n_r=64)
    phi, l, h = rs.phi[2], int(rs.l[2]), rs.h
    alpha, D = [0.4, 2.0, 11.0], [0.3, -0.2, 0.9]
    tot = 0.0
    for i in range(1, 65):
        r = i * h
        chi = sum(D[m] * r ** l * math.exp(-alpha[m] * r * r) for m in range(3))
        tot += (chi / r ** l - phi[i - 1] / r ** l) ** 2
    y = N.targets(phi, l, h)
    assert N.err(alpha, D, y, N.grid(64, h)) == pytest.approx(tot, rel=1e-13)


def test_project_one_gaussian_closed_form():
    r = N.grid(200, 0.03)
    y = np.cos(r) * np.exp(-0.2 * r)
    a = 0.7
    e = np.exp(-a * r * r)
    D, f = N.project(np.array([a]), y, r)
    # one-column least squares: D = <e, y> / <e, e>, with the relative ridge on the diagonal
    assert D[0] == pytest.approx(float(e @ y) / (float(e @ e) * (1 + N.RIDGE)), rel=1e-14)
    assert f == pytest.approx(float(((D[0] * e - y) ** 2).sum()), rel=1e-14)


def test_project_is_least_squares_minimum():
    rs = inputs.nao_set(1, n_r=256)
    y = N.targets(rs.phi[0], 0, rs.h)
    r = N.grid(256, rs.h)
    alpha = np.array([0.5, 3.0, 30.0])
    D, f = N.project(alpha, y, r)
    rng = np.random.default_rng(1)
    for _ in range(20):
        v = rng.standard_normal(3)
        for eps in (1e-3, 1e-5):
            assert N.err(alpha, D + eps * v, y, r) >= f * (1 - 1e-12)


def test_jacobian_central_differences():
    r = N.grid(128, 0.04)
    alpha = np.array([0.3, 1.9, 8.0])
    D = np.array([0.7, -0.4, 1.1])
    J = N.jacobian(alpha, D, r)
    x = np.concatenate([alpha, D])

    def res(x):
        return N.gaussians(x[:3], r) @ x[3:]

    for k in range(6):
        hstep = 1e-5 * max(1.0, abs(x[k]))
        xp, xm = x.copy(), x.copy()
        xp[k] += hstep
        xm[k] -= hstep
        fd = (res(xp) - res(xm)) / (2 * hstep)
        assert np.allclose(J[:, k], fd, rtol=1e-7, atol=1e-9)


def test_exact_recovery_of_a_gaussian_sum():
    n_r, h = 512, 6.0 / 512
    r = N.grid(n_r, h)
    a_true, d_true = np.array([0.3, 1.7, 9.0]), np.array([0.5, -0.8, 1.2])
    y = N.gaussians(a_true, r) @ d_true
    out = N.fit(y, 0, h, M=3, N=3, P=32, G=20, max_iter=200, seed=3)
    b = out["best"]
    assert b["err"] <= 1e-24 * float(y @ y)
    assert np.allclose(b["alpha"], a_true, rtol=1e-6)
    assert np.allclose(b["D"], d_true, rtol=1e-6)


def test_active_bound_kkt():
    """A target decaying slower than the bound allows: the one-Gaussian fit sits on
    alpha_min, D is the projected one there, and err grows into the feasible set."""
    n_r, h = 512, 6.0 / 512
    r = N.grid(n_r, h)
    y = np.exp(-0.03 * r * r)
    out = N.fit(y, 0, h, M=1, N=2, P=16, G=8, max_iter=100, seed=5)
    b = out["best"]
    assert b["alpha"][0] == 0.1
    D0, f0 = N.project(np.array([0.1]), y, r)
    assert b["err"] == pytest.approx(f0, rel=1e-12)
    assert b["D"][0] == pytest.approx(D0[0], rel=1e-5)  # err is flat to second order in D
    assert N.project(np.array([0.1 * (1 + 1e-4)]), y, r)[1] > f0


@pytest.fixture(scope="module")
def nao_fit():
    rs = inputs.nao_set(1)
    f = 2
    out = N.fit(rs.phi[f], int(rs.l[f]), rs.h, M=4, N=4, P=24, G=12, max_iter=150, seed=11, fun=f)
    return rs, f, out


def test_converged_fit_is_stationary(nao_fit):
    rs, f, out = nao_fit
    y = N.targets(rs.phi[f], int(rs.l[f]), rs.h)
    r = N.grid(len(y), rs.h)
    for p in out["restarts"]:
        a, d = p["alpha"], p["D"]
        assert np.all(a >= 0.1)
        assert p["err"] == pytest.approx(N.err(a, d, y, r), rel=1e-12)
        if p["steps"] >= 150:
            continue
        J = N.jacobian(a, d, r)
        res = N.gaussians(a, r) @ d - y
        g = J.T @ res
        scale = np.linalg.norm(J, axis=0) * np.linalg.norm(res)
        free = np.concatenate([a > 0.1, np.ones(len(d), bool)])
        assert np.all(np.abs(g[free]) <= 1e-3 * scale[free])
        assert np.all(g[~free] >= 0)


def test_local_search_never_worsens(nao_fit):
    rs, f, out = nao_fit
    y = N.targets(rs.phi[f], int(rs.l[f]), rs.h)
    r = N.grid(len(y), rs.h)
    for p in out["restarts"]:
        assert p["err"] <= N.err(p["ga_alpha"], p["ga_D"], y, r)


def test_algorithm1_keeps_the_first_smallest(nao_fit):
    _, _, out = nao_fit
    errs = [p["err"] for p in out["restarts"]]
    k = out["best"]["iter"]
    assert out["best"]["err"] == min(errs)
    assert all(e > errs[k] for e in errs[:k])


def test_genetic_elitism_and_box():
    rs = inputs.nao_set(1, n_r=256)
    y = N.targets(rs.phi[1], 0, rs.h)
    r = N.grid(256, rs.h)
    hist = []
    a, d, fbest = N.genetic(3, y, r, M=3, P=16, G=10, alpha_min=0.1, alpha_max=1000.0, seed=2,
                            history=hist)
    assert len(hist) == 11
    assert all(hist[i + 1]["best"] <= hist[i]["best"] for i in range(10))
    for h_ in hist:
        u = h_["genes"]
        assert np.all(u >= math.log(0.1)) and np.all(u <= math.log(1000.0))
        assert np.all(np.diff(u, axis=1) >= 0)
    assert fbest == pytest.approx(N.project(a, y, r)[1], rel=1e-14)


def test_more_gaussians_fit_better():
    rs = inputs.nao_set(1, n_r=256)
    f = 0
    errs = []
    for M in (2, 3, 4):
        out = N.fit(rs.phi[f], 0, rs.h, M=M, N=3, P=24, G=10, max_iter=150, seed=4)
        errs.append(out["best"]["err"])
    assert errs[0] > errs[1] > errs[2]
