"""Brute-force numerical integrals used to pin the oracle (test helper).

Nothing here uses a Boys function or a recurrence.  The attenuated kernel is written
as a Gaussian integral,

    erfc(omega r) / r = (2 / sqrt(pi)) * int_omega^inf exp(-t^2 r^2) dt,

so for Cartesian Gaussian primitives the six-dimensional integral becomes, for each t,
a product over x, y, z of two-dimensional integrals of a polynomial times a Gaussian in
(x, x').  Those are done exactly by Gauss-Hermite quadrature after an affine change of
variables (Cholesky factor of the 2x2 quadratic form); the t integral is done by
composite Gauss-Legendre quadrature in s = omega / t on (0, 1].

Basis functions are built from their definition: chi = N * S_m(r - A) * sum_k c_k
n_l(alpha_k) exp(-alpha_k |r - A|^2), with N from a Gauss-Hermite self-overlap.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np

# spherical polynomials S_m as {(i, j, k): coefficient}
SPH = {
    0: [{(0, 0, 0): 1.0}],
    1: [{(1, 0, 0): 1.0}, {(0, 1, 0): 1.0}, {(0, 0, 1): 1.0}],
    2: [
        {(1, 1, 0): 1.0},                                   # xy
        {(0, 1, 1): 1.0},                                   # yz
        {(2, 0, 0): -1.0, (0, 2, 0): -1.0, (0, 0, 2): 2.0},  # 3z^2 - r^2
        {(1, 0, 1): 1.0},                                   # xz
        {(2, 0, 0): 1.0, (0, 2, 0): -1.0},                  # x^2 - y^2
    ],
}


def dfact(n):
    return math.prod(range(n, 0, -2)) if n > 0 else 1


def prim_norm(alpha, l):
    return (2 * alpha / math.pi) ** 0.75 * (4 * alpha) ** (l / 2) / math.sqrt(dfact(2 * l - 1))


@lru_cache(maxsize=None)
def _gh(n):
    return np.polynomial.hermite.hermgauss(n)


def self_overlap(l, m, alphas, weights):
    """int (S_m(r) R(r))^2 d^3r by Gauss-Hermite, R = sum_k w_k exp(-alpha_k r^2)."""
    x, w = _gh(12)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    W = w[:, None, None] * w[None, :, None] * w[None, None, :]
    tot = 0.0
    for ak, wk in zip(alphas, weights):
        for al, wl in zip(alphas, weights):
            g = ak + al
            s = 1.0 / math.sqrt(g)
            poly = sum(c * (X * s) ** i * (Y * s) ** j * (Z * s) ** k for (i, j, k), c in SPH[l][m].items())
            tot += wk * wl * s ** 3 * np.sum(W * poly * poly)
    return tot


def contracted_functions(l, alphas, coefs):
    """(weights per primitive, [N_m]) of the normalised spherical functions of a shell."""
    wts = [c * prim_norm(a, l) for a, c in zip(alphas, coefs)]
    norms = [1.0 / math.sqrt(self_overlap(l, m, alphas, wts)) for m in range(2 * l + 1)]
    return wts, norms


def _s_grid(omega, n_panels=48, npts=24):
    """Nodes/weights in s on (0,1] for t = omega/s; graded towards s = 0."""
    x, w = np.polynomial.legendre.leggauss(npts)
    edges = np.concatenate([[0.0], np.geomspace(1e-5, 1.0, n_panels)])
    S, Wt = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        S.append(0.5 * (b - a) * x + 0.5 * (b + a))
        Wt.append(0.5 * (b - a) * w)
    return np.concatenate(S), np.concatenate(Wt)


def axis_integrals(t, a, A, b, B, c, C, d, D, lmax=2):
    """I[t, i, j, k, l] = int int (x-A)^i (x-B)^j e^{-a(x-A)^2 - b(x-B)^2} e^{-t^2 (x-x')^2}
    (x'-C)^k (x'-D)^l e^{-c(x'-C)^2 - d(x'-D)^2} dx dx'  for i,j,k,l <= lmax."""
    gx, gw = _gh(8)
    nt = t.shape[0]
    t2 = t * t
    M11 = a + b + t2
    M22 = c + d + t2
    M12 = -t2
    h1 = a * A + b * B
    h2 = c * C + d * D
    const = a * A * A + b * B * B + c * C * C + d * D * D
    det = M11 * M22 - M12 * M12
    z1 = (M22 * h1 - M12 * h2) / det
    z2 = (M11 * h2 - M12 * h1) / det
    cmin = const - (h1 * z1 + h2 * z2)
    # Cholesky of M: L = [[l11, 0], [l21, l22]]; z = z0 + L^{-T} y
    l11 = np.sqrt(M11)
    l21 = M12 / l11
    l22 = np.sqrt(M22 - l21 * l21)
    Y1, Y2 = np.meshgrid(gx, gx, indexing="ij")
    Wn = (gw[:, None] * gw[None, :]).ravel()
    y1 = Y1.ravel()[None, :]
    y2 = Y2.ravel()[None, :]
    # L^{-T} = [[1/l11, -l21/(l11 l22)], [0, 1/l22]]
    x = z1[:, None] + y1 / l11[:, None] - y2 * (l21 / (l11 * l22))[:, None]
    xp = z2[:, None] + y2 / l22[:, None]
    pref = np.exp(-cmin) / (l11 * l22)
    n = lmax + 1
    pa = np.stack([(x - A) ** i for i in range(n)], 1)   # [t, i, node]
    pb = np.stack([(x - B) ** i for i in range(n)], 1)
    pc = np.stack([(xp - C) ** i for i in range(n)], 1)
    pd = np.stack([(xp - D) ** i for i in range(n)], 1)
    I = np.einsum("tin,tjn,tkn,tln,n->tijkl", pa, pb, pc, pd, Wn, optimize=True)
    return I * pref[:, None, None, None, None]


def prim_cart_bf(ls, alphas, centres, omega, n_panels=48, npts=24):
    """Primitive Cartesian [ab|cd] (weight 1) for the erfc kernel, all components."""
    s, ws = _s_grid(omega, n_panels, npts)
    t = omega / s
    jac = ws * omega / (s * s) * (2.0 / math.sqrt(math.pi))
    a, b, c, d = alphas
    C4 = np.asarray(centres, dtype=float).reshape(4, 3)
    Ix = [axis_integrals(t, a, C4[0, k], b, C4[1, k], c, C4[2, k], d, C4[3, k]) for k in range(3)]
    comps = [cart_list(l) for l in ls]
    out = np.zeros(tuple(len(cl) for cl in comps))
    for ia, ea in enumerate(comps[0]):
        for ib, eb in enumerate(comps[1]):
            for ic, ec in enumerate(comps[2]):
                for id_, ed in enumerate(comps[3]):
                    prod = jac.copy()
                    for k in range(3):
                        prod = prod * Ix[k][:, ea[k], eb[k], ec[k], ed[k]]
                    out[ia, ib, ic, id_] = prod.sum()
    return out


def cart_list(l):
    return [(i, j, l - i - j) for i in range(l, -1, -1) for j in range(l - i, -1, -1)]


def contracted_quartet_bf(shells, omega, n_panels=48, npts=24):
    """Normalised spherical (IJ|KL) for four shells given as (l, centre, alphas, coefs)."""
    s, ws = _s_grid(omega, n_panels, npts)
    t = omega / s
    jac = ws * omega / (s * s) * (2.0 / math.sqrt(math.pi))
    info = []
    for (l, A, al, co) in shells:
        wts, norms = contracted_functions(l, al, co)
        info.append((l, np.asarray(A, float), list(al), wts, norms))
    nsph = [2 * x[0] + 1 for x in info]
    out = np.zeros(nsph)
    # Cartesian (raw monomial) contracted integrals, then spherical combination
    cart = {}
    for ka, (aa, wa) in enumerate(zip(info[0][2], info[0][3])):
        for kb, (ab, wb) in enumerate(zip(info[1][2], info[1][3])):
            for kc, (ac, wc) in enumerate(zip(info[2][2], info[2][3])):
                for kd, (ad, wd) in enumerate(zip(info[3][2], info[3][3])):
                    Ix = [axis_integrals(t, aa, info[0][1][k], ab, info[1][1][k], ac, info[2][1][k],
                                         ad, info[3][1][k]) for k in range(3)]
                    wt = wa * wb * wc * wd
                    for ea in cart_list(info[0][0]):
                        for eb in cart_list(info[1][0]):
                            for ec in cart_list(info[2][0]):
                                for ed in cart_list(info[3][0]):
                                    prod = jac.copy()
                                    for k in range(3):
                                        prod = prod * Ix[k][:, ea[k], eb[k], ec[k], ed[k]]
                                    key = (ea, eb, ec, ed)
                                    cart[key] = cart.get(key, 0.0) + wt * prod.sum()
    for m0 in range(nsph[0]):
        for m1 in range(nsph[1]):
            for m2 in range(nsph[2]):
                for m3 in range(nsph[3]):
                    v = 0.0
                    for e0, c0 in SPH[info[0][0]][m0].items():
                        for e1, c1 in SPH[info[1][0]][m1].items():
                            for e2, c2 in SPH[info[2][0]][m2].items():
                                for e3, c3 in SPH[info[3][0]][m3].items():
                                    v += c0 * c1 * c2 * c3 * cart[(e0, e1, e2, e3)]
                    out[m0, m1, m2, m3] = v * info[0][4][m0] * info[1][4][m1] * info[2][4][m2] * info[3][4][m3]
    return out


def ssss_closed(A, B, C, D, a, b, c, d, omega):
    """Closed-form primitive (ss|ss) for erfc(omega r)/r (omega = 0: Coulomb), F_0 via erf."""
    A, B, C, D = (np.asarray(v, float) for v in (A, B, C, D))
    p, q = a + b, c + d
    P = (a * A + b * B) / p
    Q = (c * C + d * D) / q
    rho = p * q / (p + q)
    T = rho * float(np.dot(P - Q, P - Q))

    def F0(x):
        if x < 1e-12:
            return 1.0 - x / 3.0
        return 0.5 * math.sqrt(math.pi / x) * math.erf(math.sqrt(x))

    kab = math.exp(-a * b / p * float(np.dot(A - B, A - B)))
    kcd = math.exp(-c * d / q * float(np.dot(C - D, C - D)))
    g = F0(T)
    if omega > 0:
        kap = omega * omega / (omega * omega + rho)
        g -= math.sqrt(kap) * F0(kap * T)
    return 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * kab * kcd * g
