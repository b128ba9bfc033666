"""The identity behind the FP32 Boys step of the mixed-precision build, checked on the CPU.

The FP32 passes evaluate the attenuated Boys function G_m(T) = F_m(T) - kappa^{m+1/2} F_m(kappa T)
(paper Sec. 2, the erfc-screened kernel) as
    G_m = 1/2 T^{-a} (Gamma(a, kappa T) - Gamma(a, T)),  a = m + 1/2,
with both upper incomplete gamma functions from Gamma(1/2, x) = sqrt(pi) erfc(sqrt x) and the
upward recursion Gamma(a + 1, x) = a Gamma(a, x) + x^a e^{-x} (all terms positive), and accept the
result only where the subtracted term is at most 1/64 of the other.  Here: the identity against
the oracle's G_m (written as the difference of Boys functions) where that difference is itself
accurate, and the recursion carried out in FP32 arithmetic (numpy float32) against a 40-digit
evaluation of the incomplete gammas, on the accepted cases: relative error below 1e-5, below
2e-6 where kappa T < 20 (beyond that G_m < e^{-20} of the Schwarz bound)."""
import numpy as np
import pytest

import oracle

mp = pytest.importorskip("mpmath")
erfc = pytest.importorskip("scipy.special").erfc
gammaincc = pytest.importorskip("scipy.special").gammaincc
gamma = pytest.importorskip("scipy.special").gamma


def g_identity(mmax, T, kap):
    a = np.arange(mmax + 1) + 0.5
    return 0.5 * T ** (-a) * gamma(a) * (gammaincc(a, kap * T) - gammaincc(a, T))


def test_identity_matches_oracle():
    rng = np.random.default_rng(3)
    for _ in range(300):
        T = float(np.exp(rng.uniform(np.log(2.0), np.log(40.0))))
        kap = float(rng.uniform(0.01, 0.6))
        ref = oracle.gboys(8, T, kap)
        got = g_identity(8, T, kap)
        # both sides are differences of two FP64 numbers: agreement to the larger one's rounding
        assert np.allclose(got, ref, rtol=1e-8, atol=1e-14 * oracle.boys(8, T)[0])


def fp32_recursion(T, kap, Lt):
    f = np.float32
    Tf, sk = f(T), f(np.sqrt(kap))
    kapf = sk * sk
    kT = kapf * Tf
    yT = f(1.0 / np.sqrt(Tf))
    invT, c0 = yT * yT, f(0.886226925) * yT
    A, B = c0 * f(erfc(np.sqrt(kT))), c0 * f(erfc(np.sqrt(Tf)))
    hk, h1 = f(0.5) * f(np.exp(-kT)), f(0.5) * f(np.exp(-Tf))
    ok = bool(B <= A * f(1 / 64)) and bool(A <= f(1e30))
    G, kp = [A - B], sk
    for m in range(Lt):
        a = f(m + 0.5)
        A = (a * A + kp * hk) * invT
        B = (a * B + h1) * invT
        kp = kp * kapf
        ok = ok and bool(B <= A * f(1 / 64)) and bool(A <= f(1e30))
        G.append(A - B)
    return ok, np.array(G, dtype=np.float64)


def test_fp32_recursion_accuracy_on_accepted_cases():
    mp.mp.dps = 40
    rng = np.random.default_rng(0)
    accepted = 0
    for _ in range(600):
        T = float(np.exp(rng.uniform(np.log(0.01), np.log(2000.0))))
        rho = float(np.exp(rng.uniform(np.log(0.02), np.log(20.0))))
        kap = 0.11 ** 2 / (0.11 ** 2 + rho)
        if kap * T >= 60.0:
            continue
        Lt = int(rng.integers(0, 9))
        ok, G = fp32_recursion(T, kap, Lt)
        if not ok:
            continue
        accepted += 1
        Tm, km = mp.mpf(T), mp.mpf(kap)
        for m in range(Lt + 1):
            a = m + mp.mpf(1) / 2
            ref = float(mp.mpf(1) / 2 * Tm ** (-a) * (mp.gammainc(a, km * Tm) - mp.gammainc(a, Tm)))
            rel = abs(G[m] - ref) / abs(ref)
            assert rel <= (2e-6 if kap * T < 20.0 else 1e-5), (T, kap, m, rel)
    assert accepted > 150


def test_declined_near_zero_T():
    """T near 0 overflows the recursion; the check declines it (FP64 set-up instead)."""
    for T in (0.0, 1e-30, 1e-6, 0.05):
        ok, _ = fp32_recursion(T, 0.1, 8)
        assert not ok
