"""Pins of the oracle's integrals.

* primitive (ss|ss) against the closed form with F_0 through erf (erfc kernel and the
  omega -> 0 Coulomb limit), and omega -> infinity giving zero;
* p and d primitives against finite-difference derivatives of that closed form:
  (x - A_x) g = (1/2a) dg/dA_x and (x - A_x)^2 g = (1/4a^2) d^2g/dA_x^2 + (1/2a) g;
* every primitive class up to (dd|dd) against brute-force quadrature (no Boys function,
  no recurrence: tests/bruteforce.py);
* contracted, normalised spherical shell quartets against brute-force quadrature;
* eight-fold permutational symmetry (paper Sec. 3.1), the Schwarz inequality (Eq.
  schwarz), translation invariance and axis-permutation covariance.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from tests import bruteforce as bf
from paper_2009_03559_gb300 import inputs

OMEGA = 0.11
RNG = np.random.default_rng(12345)


def rand_geom(spread=1.5):
    return RNG.uniform(-spread, spread, (4, 3))


@pytest.mark.parametrize("omega", [OMEGA, 0.0, 0.5])
def test_ssss_closed_form(omega):
    for _ in range(20):
        C = rand_geom(2.0)
        al = RNG.uniform(0.1, 8.0, 4)
        v = oracle.prim_cart([0, 0, 0, 0], al, C, omega)[0, 0, 0, 0]
        ref = bf.ssss_closed(*C, *al, omega)
        assert v == pytest.approx(ref, rel=1e-13, abs=1e-16)


def test_large_omega_vanishes():
    C = rand_geom(1.0)
    al = [0.5, 0.7, 0.9, 1.1]
    coul = oracle.prim_cart([1, 1, 1, 1], al, C, 0.0)
    big = oracle.prim_cart([1, 1, 1, 1], al, C, 1e5)
    assert np.abs(big).max() < 1e-6 * np.abs(coul).max()


# ---------------------------------------------------------------- finite differences

def _f_shift(C, al, omega, shifts):
    Cs = C.copy()
    for (t, ax), h in shifts:
        Cs[t, ax] += h
    return bf.ssss_closed(*Cs, *al, omega)


def _deriv(C, al, omega, vars_, h=2e-3):
    """Mixed derivative d/dv1 d/dv2 ... (order <= 2) by central differences + Richardson."""
    def D(hh):
        if len(vars_) == 0:
            return _f_shift(C, al, omega, [])
        if len(vars_) == 1:
            v = vars_[0]
            return (_f_shift(C, al, omega, [(v, hh)]) - _f_shift(C, al, omega, [(v, -hh)])) / (2 * hh)
        v1, v2 = vars_
        if v1 == v2:
            return (_f_shift(C, al, omega, [(v1, hh)]) - 2 * _f_shift(C, al, omega, [])
                    + _f_shift(C, al, omega, [(v1, -hh)])) / (hh * hh)
        return (_f_shift(C, al, omega, [(v1, hh), (v2, hh)]) - _f_shift(C, al, omega, [(v1, hh), (v2, -hh)])
                - _f_shift(C, al, omega, [(v1, -hh), (v2, hh)]) + _f_shift(C, al, omega, [(v1, -hh), (v2, -hh)])) / (4 * hh * hh)
    d1, d2, d3 = D(h), D(h / 2), D(h / 4)
    r1 = (4 * d2 - d1) / 3
    r2 = (4 * d3 - d2) / 3
    return (16 * r2 - r1) / 15


def _fd_value(ls, comps, al, C, omega):
    """Expand the monomial prefactors into derivative operators on the s-type closed form."""
    # each centre contributes a list of (coefficient, [vars]) terms
    per_centre = []
    for t, (l, e) in enumerate(zip(ls, comps)):
        a = al[t]
        terms = [(1.0, [])]
        for ax in range(3):
            n = e[ax]
            if n == 0:
                continue
            if n == 1:
                new = [(1.0 / (2 * a), [(t, ax)])]
            else:  # n == 2
                new = [(1.0 / (4 * a * a), [(t, ax), (t, ax)]), (1.0 / (2 * a), [])]
            terms = [(c1 * c2, v1 + v2) for c1, v1 in terms for c2, v2 in new]
        per_centre.append(terms)
    total = 0.0
    for combo in itertools.product(*per_centre):
        coef = math.prod(c for c, _ in combo)
        vars_ = sum((v for _, v in combo), [])
        assert len(vars_) <= 2
        total += coef * _deriv(C, al, omega, vars_)
    return total


FD_CASES = [
    (1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1),
    (1, 0, 1, 0), (1, 1, 0, 0), (0, 0, 1, 1), (0, 1, 0, 1), (1, 0, 0, 1),
    (2, 0, 0, 0), (0, 2, 0, 0), (0, 0, 2, 0), (0, 0, 0, 2),
]


@pytest.mark.parametrize("ls", FD_CASES)
def test_finite_difference_p_d(ls):
    C = rand_geom(1.2)
    al = RNG.uniform(0.3, 2.5, 4)
    got = oracle.prim_cart(list(ls), al, C, OMEGA)
    comps = [bf.cart_list(l) for l in ls]
    scale = np.abs(got).max()
    for idx in itertools.product(*[range(len(c)) for c in comps]):
        cc = [comps[t][idx[t]] for t in range(4)]
        ref = _fd_value(ls, cc, al, C, OMEGA)
        assert abs(got[idx] - ref) <= 2e-8 * scale, (ls, cc, got[idx], ref)


# ---------------------------------------------------------------- brute force

BF_CLASSES = [(0, 0, 0, 0), (1, 0, 0, 0), (1, 1, 1, 1), (2, 0, 1, 0), (2, 1, 0, 2), (2, 2, 1, 1),
              (0, 2, 2, 0), (2, 2, 2, 2)]


@pytest.mark.parametrize("ls", BF_CLASSES)
def test_primitive_bruteforce(ls):
    C = rand_geom(1.5)
    al = RNG.uniform(0.2, 3.0, 4)
    got = oracle.prim_cart(list(ls), al, C, OMEGA)
    ref = bf.prim_cart_bf(ls, al, C, OMEGA)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-11 * scale


def _tiny_diamond():
    s = inputs.diamond_system(3, seed=77)
    B = oracle.Basis(s)
    shells = []
    for I in range(s.n_shells):
        a0 = int(s.shell_atom[I])
        off = 3 * I
        shells.append((int(s.shell_l[I]), s.xyz[a0], s.alpha[off:off + 3], s.coef[off:off + 3]))
    return s, B, shells


@pytest.mark.parametrize("q", [(0, 2, 5, 7), (4, 2, 9, 3), (4, 9, 14, 12), (4, 4, 9, 9), (14, 9, 4, 13)])
def test_contracted_bruteforce(q):
    s, B, shells = _tiny_diamond()
    got = B.quartet(*q)
    ref = bf.contracted_quartet_bf([shells[i] for i in q], s.omega)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-10 * max(scale, 1e-3)


def test_normalisation_unit_overlap():
    s, B, shells = _tiny_diamond()
    nrm, w = B.norms()
    for I, (l, A, al, co) in enumerate(shells):
        for m in range(2 * l + 1):
            wts = w[3 * I:3 * I + 3]
            ov = bf.self_overlap(l, m, al, wts) * nrm[I, m] ** 2
            assert ov == pytest.approx(1.0, rel=1e-13)


# ---------------------------------------------------------------- structure

def test_eightfold_symmetry():
    s, B, shells = _tiny_diamond()
    n = s.n_shells
    for _ in range(30):
        I, J, K, L = RNG.integers(0, n, 4)
        v = B.quartet(I, J, K, L)
        perms = {
            (J, I, K, L): v.transpose(1, 0, 2, 3),
            (I, J, L, K): v.transpose(0, 1, 3, 2),
            (J, I, L, K): v.transpose(1, 0, 3, 2),
            (K, L, I, J): v.transpose(2, 3, 0, 1),
            (L, K, I, J): v.transpose(3, 2, 0, 1),
            (K, L, J, I): v.transpose(2, 3, 1, 0),
            (L, K, J, I): v.transpose(3, 2, 1, 0),
        }
        scale = max(np.abs(v).max(), 1e-30)
        for key, exp in perms.items():
            assert np.abs(B.quartet(*key) - exp).max() <= 1e-13 * scale


def test_schwarz_inequality_all_functions():
    s, B, shells = _tiny_diamond()
    n = s.n_shells
    diag = {}
    for I in range(n):
        for J in range(n):
            d = B.quartet(I, J, I, J)
            ni, nj = d.shape[0], d.shape[1]
            diag[(I, J)] = np.array([[d[a, b, a, b] for b in range(nj)] for a in range(ni)])
            assert np.all(diag[(I, J)] >= -1e-15)  # the erfc kernel is positive definite
    for _ in range(40):
        I, J, K, L = RNG.integers(0, n, 4)
        v = B.quartet(I, J, K, L)
        bound = np.sqrt(diag[(I, J)][:, :, None, None] * diag[(K, L)][None, None, :, :])
        assert np.all(np.abs(v) <= bound * (1 + 1e-12) + 1e-300)


def test_translation_invariance():
    s = inputs.diamond_system(3, seed=78)
    B = oracle.Basis(s)
    s2 = inputs.diamond_system(3, seed=78)
    s2.xyz = s2.xyz + np.array([3.1, -7.2, 0.45])
    B2 = oracle.Basis(s2)
    for q in [(0, 4, 5, 9), (4, 9, 14, 4), (2, 3, 12, 13)]:
        a, b = B.quartet(*q), B2.quartet(*q)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_axis_permutation_covariance():
    """Cyclic x->y->z relabelling of all coordinates permutes p components."""
    s = inputs.cluster_system(4, seed=79)
    B = oracle.Basis(s)
    s2 = inputs.cluster_system(4, seed=79)
    s2.xyz = s.xyz[:, [2, 0, 1]]  # new (x,y,z) = old (z,x,y): old x is new y
    B2 = oracle.Basis(s2)
    perm = [1, 2, 0]  # old component c lives at new index perm[c]
    for q in [(1, 3, 5, 7), (1, 1, 3, 3), (0, 3, 5, 6)]:
        a = B.quartet(*q)
        b = B2.quartet(*q)
        idx = [perm if int(s.shell_l[x]) == 1 else [0] for x in q]
        b_back = b[np.ix_(*idx)]
        assert np.abs(a - b_back).max() <= 1e-12 * np.abs(a).max()
