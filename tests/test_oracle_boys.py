"""Pins of the oracle's Boys function F_m(T) and its erfc-attenuated form G_m(T).

F_m(T) = int_0^1 u^{2m} exp(-T u^2) du; G_m(T) = F_m(T) - kappa^{m+1/2} F_m(kappa T)
= int_{sqrt(kappa)}^1 u^{2m} exp(-T u^2) du.  Checked against: the exact values at
T = 0, the closed form of F_0 through erf, composite Gauss-Legendre quadrature of the
defining integral, and the large-T asymptote.
"""
import math

import numpy as np
import pytest

import oracle


def quad_u(m, T, lo=0.0, hi=1.0, panels=64, npts=20):
    """Composite Gauss-Legendre of int_lo^hi u^{2m} exp(-T u^2) du."""
    x, w = np.polynomial.legendre.leggauss(npts)
    edges = np.linspace(lo, hi, panels + 1)
    tot = 0.0
    for a, b in zip(edges[:-1], edges[1:]):
        u = 0.5 * (b - a) * x + 0.5 * (b + a)
        tot += 0.5 * (b - a) * np.sum(w * u ** (2 * m) * np.exp(-T * u * u))
    return tot


def test_F_at_zero():
    F = oracle.boys(16, 0.0)
    assert np.allclose(F, [1.0 / (2 * m + 1) for m in range(17)], rtol=1e-15, atol=0)


@pytest.mark.parametrize("T", [1e-8, 1e-3, 0.3, 1.0, 4.5, 12.0, 29.99, 30.0, 30.01, 45.0, 120.0, 1e4])
def test_F0_erf(T):
    ref = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    assert oracle.boys(0, T)[0] == pytest.approx(ref, rel=2e-15)


@pytest.mark.parametrize("T", [0.0, 0.05, 0.7, 2.0, 9.0, 17.5, 29.5, 30.5, 38.0, 60.0])
def test_Fm_quadrature(T):
    F = oracle.boys(12, T)
    for m in range(13):
        ref = quad_u(m, T)
        assert F[m] == pytest.approx(ref, rel=1e-13, abs=1e-300), (m, T)


def test_Fm_asymptote():
    T = 400.0
    F = oracle.boys(10, T)
    for m in range(11):
        asym = math.prod(range(2 * m - 1, 0, -2)) / 2 ** (m + 1) * math.sqrt(math.pi / T ** (2 * m + 1))
        assert F[m] == pytest.approx(asym, rel=1e-14)


def test_F_recursion_consistency():
    """F_m = (2T F_{m+1} + e^{-T}) / (2m+1) must hold on both sides of the switch."""
    for T in (5.0, 29.999, 30.0, 31.0, 80.0):
        F = oracle.boys(9, T)
        for m in range(9):
            assert F[m] == pytest.approx((2 * T * F[m + 1] + math.exp(-T)) / (2 * m + 1), rel=1e-13)


@pytest.mark.parametrize("T,kappa", [(0.0, 0.1), (0.4, 0.05), (3.0, 0.13), (25.0, 0.01), (31.0, 0.3),
                                     (200.0, 0.12), (7.0, 0.9999)])
def test_G_is_truncated_integral(T, kappa):
    G = oracle.gboys(8, T, kappa)
    F = oracle.boys(8, T)
    for m in range(9):
        ref = quad_u(m, T, lo=math.sqrt(kappa), hi=1.0)
        # G is a difference of two terms of size ~F_m(T): FP64 cancellation error scales with F_m(T)
        assert G[m] == pytest.approx(ref, rel=1e-12, abs=2e-15 * F[m]), (m, T, kappa)


def test_G_limits():
    # omega -> 0 (kappa -> 0): Coulomb; omega -> infinity (kappa -> 1): zero
    assert np.allclose(oracle.gboys(6, 2.0, 0.0), oracle.boys(6, 2.0), rtol=0, atol=0)
    assert np.all(np.abs(oracle.gboys(6, 2.0, 1.0)) < 1e-15)
