"""Oracle for the NAO2GTO fit (paper Sec. "NAO2GTO scheme", the GTO expansion of a radial
function, the residual sum of squares and Algorithm 1).  TEST INFRASTRUCTURE ONLY (like the
rest of oracle/): the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs use it;
the CUDA library never imports or calls it and shares no code with it.  Plain NumPy, FP64,
one restart at a time.

What is fitted (paper, NAO2GTO scheme):
    chi(r) = sum_m D_m r^l exp(-alpha_m r^2),  m = 1..M,
    err(alpha, D) = sum_i (chi(r_i)/r_i^l - phi(r_i)/r_i^l)^2
                  = sum_i (sum_m D_m exp(-alpha_m r_i^2) - y_i)^2,   y_i = phi(r_i) / r_i^l,
with the constraint alpha_m >= alpha_min (0.1 in the paper).  Grid: r_i = i h, i = 1..n_r.

Algorithm 1, in its order: for iter = 1..N, (1) a constrained genetic algorithm gives an
initial alpha and D, (2) a constrained local minimisation refines them, (3) err is
evaluated, (4) the pair is kept if iter = 1 or err < best_err.

The paper names the two searches but prints neither; the readings here are these.
(1) Real-coded genetic algorithm on u_m = ln alpha_m in [ln alpha_min, ln alpha_max]:
    population P, G generations, individuals kept with sorted genes; fitness = err at the
    variable-projection D (for fixed alpha, D solves the normal equations of the linear
    least-squares problem, with a relative ridge 1e-12 on the diagonal); elitism (the best
    individual survives), binary tournaments (the second contestant wins only when its
    fitness is below the first's by more than a relative 1e-12), blend crossover
    c = a + w (b - a) with w uniform in [-0.25, 1.25), mutation of each gene with probability
    0.1 by a uniform step in [-0.5, 0.5), reflection at the box and sorting.
(2) Trust-region search over (alpha, D) in Levenberg-Marquardt form: the step solves
    (H + lambda diag H) delta = -g with H = J^T J and g = J^T res.  The bound is kept by
    projection: an exponent sitting on alpha_min whose gradient points out of the feasible set
    is held (its row and column of the system become those of the identity, its gradient
    component zero), and the trial point is projected onto alpha >= alpha_min.  (Reflecting
    the trial point at the bound, as the trust-region-reflective method does, stalled short
    of an active bound in this form.)  A trial point is accepted if it lowers err by more than
    a relative 1e-12 (lambda / 3), otherwise lambda x 4; the search stops after a relative
    decrease below 1e-10, at lambda > 1e10, or after max_iter trial steps.  The linear solves
    are direct (the systems are 2M x 2M, M <= 6).
Random draws: U(c) = (SplitMix64 output c of the run's seed >> 11) / 2^53, SplitMix64 as
published by Steele, Lea and Flood (2014): output c (0-based) of seed s is
mix(s + (c + 1) * 0x9E3779B97F4A7C15 mod 2^64).  Counter of slot k of individual j in
generation g (0 = the initial population) of restart q: ((q (G + 1) + g) P + j) S + k,
S = 4 + 2M slots (two tournaments of two draws, M blend weights, M mutation draws; the
initial population uses the first M).
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1
RIDGE = 1e-12
TIE = 1e-12
CONV = 1e-10
LAMBDA0 = 1e-3
LAMBDA_MAX = 1e10
P_MUT = 0.1
MUT_STEP = 0.5


# ---------------------------------------------------------------------------
# Counter-based draws (SplitMix64, Steele-Lea-Flood 2014)
# ---------------------------------------------------------------------------
def splitmix64(seed: int, counter: int) -> int:
    """Output number `counter` (0-based) of SplitMix64 started from `seed`."""
    z = (seed + (counter + 1) * GOLDEN_GAMMA) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def uniform(seed: int, counter: int) -> float:
    """A double in [0, 1) from the top 53 bits."""
    return (splitmix64(seed, counter) >> 11) * (1.0 / 9007199254740992.0)


def counter(q: int, g: int, j: int, k: int, G: int, P: int, M: int) -> int:
    return ((q * (G + 1) + g) * P + j) * (4 + 2 * M) + k


# ---------------------------------------------------------------------------
# The residual and its pieces
# ---------------------------------------------------------------------------
def grid(n_r: int, h: float) -> np.ndarray:
    return h * np.arange(1, n_r + 1, dtype=np.float64)


def targets(phi: np.ndarray, l: int, h: float) -> np.ndarray:
    """y_i = phi(r_i) / r_i^l."""
    r = grid(phi.shape[-1], h)
    return phi / r ** l


def gaussians(alpha: np.ndarray, r: np.ndarray) -> np.ndarray:
    """E[i, m] = exp(-alpha_m r_i^2)."""
    return np.exp(-np.outer(r * r, alpha))


def err(alpha, D, y, r) -> float:
    """The paper's residual sum of squares."""
    res = gaussians(np.asarray(alpha, float), r) @ np.asarray(D, float) - y
    return float(res @ res)


def project(alpha, y, r):
    """Variable projection: for fixed alpha, D from (A + RIDGE diag A) D = b with
    A = E^T E, b = E^T y; returns (D, err(alpha, D)).  A failed factorisation gives D = 0."""
    E = gaussians(np.asarray(alpha, float), r)
    A = E.T @ E
    b = E.T @ y
    A = A + RIDGE * np.diag(np.diag(A))
    try:
        L = np.linalg.cholesky(A)
    except np.linalg.LinAlgError:
        D = np.zeros(len(alpha))
        return D, err(alpha, D, y, r)
    D = np.linalg.solve(L.T, np.linalg.solve(L, b))
    return D, err(alpha, D, y, r)


def jacobian(alpha, D, r):
    """d res_i / d alpha_m = -D_m r_i^2 exp(-alpha_m r_i^2);  d res_i / d D_m = exp(...)."""
    E = gaussians(np.asarray(alpha, float), r)
    return np.hstack([-(r * r)[:, None] * E * np.asarray(D, float)[None, :], E])


# ---------------------------------------------------------------------------
# (1) constrained genetic algorithm
# ---------------------------------------------------------------------------
def _better(fa: float, fb: float) -> bool:
    """fa beats fb by more than the tie window."""
    return fa < fb * (1.0 - TIE)


def _best_index(fit) -> int:
    b = 0
    for j in range(1, len(fit)):
        if _better(fit[j], fit[b]):
            b = j
    return b


def _reflect_box(c: float, lo: float, hi: float) -> float:
    if c < lo:
        c = 2.0 * lo - c
    if c > hi:
        c = 2.0 * hi - c
    return min(max(c, lo), hi)


def genetic(q: int, y, r, M: int, P: int, G: int, alpha_min: float, alpha_max: float, seed: int,
            history=None):
    """Returns (alpha, D, fitness) of the best individual after G generations; `history`, if a
    list, receives per generation the genes and the best fitness."""
    lo, hi = math.log(alpha_min), math.log(alpha_max)
    pop = np.empty((P, M))
    fit = np.empty(P)
    for j in range(P):
        u = [lo + uniform(seed, counter(q, 0, j, m, G, P, M)) * (hi - lo) for m in range(M)]
        pop[j] = np.sort(u)
        fit[j] = project(np.exp(pop[j]), y, r)[1]
    if history is not None:
        history.append({"genes": pop.copy(), "best": float(fit[_best_index(fit)])})
    for g in range(1, G + 1):
        new = np.empty_like(pop)
        nfit = np.empty_like(fit)
        e = _best_index(fit)
        new[0], nfit[0] = pop[e], fit[e]
        for j in range(1, P):
            U = [uniform(seed, counter(q, g, j, k, G, P, M)) for k in range(4 + 2 * M)]

            def tournament(u1, u2):
                i1 = min(int(u1 * P), P - 1)
                i2 = min(int(u2 * P), P - 1)
                return i2 if _better(fit[i2], fit[i1]) else i1

            a = pop[tournament(U[0], U[1])]
            b = pop[tournament(U[2], U[3])]
            child = np.empty(M)
            for m in range(M):
                w = -0.25 + 1.5 * U[4 + m]
                c = a[m] + w * (b[m] - a[m])
                v = U[4 + M + m]
                if v < P_MUT:
                    c = c + MUT_STEP * (2.0 * (v / P_MUT) - 1.0)
                child[m] = _reflect_box(c, lo, hi)
            new[j] = np.sort(child)
            nfit[j] = project(np.exp(new[j]), y, r)[1]
        pop, fit = new, nfit
        if history is not None:
            history.append({"genes": pop.copy(), "best": float(fit[_best_index(fit)])})
    e = _best_index(fit)
    alpha = np.exp(pop[e])
    D, f = project(alpha, y, r)
    return alpha, D, f


# ---------------------------------------------------------------------------
# (2) constrained local minimal search
# ---------------------------------------------------------------------------
def local_search(alpha, D, y, r, alpha_min: float, max_iter: int):
    """Returns (alpha, D, err, trial steps taken)."""
    M = len(alpha)
    x = np.concatenate([np.asarray(alpha, float), np.asarray(D, float)])
    E = err(x[:M], x[M:], y, r)
    lam = LAMBDA0
    H = g = None
    it = 0
    while it < max_iter:
        if H is None:
            J = jacobian(x[:M], x[M:], r)
            res = gaussians(x[:M], r) @ x[M:] - y
            H = J.T @ J
            g = J.T @ res
        it += 1
        dH = np.diag(H)
        floor = 1e-12 * max(float(dH.max()), 0.0)
        A = H + lam * np.diag(np.maximum(dH, floor))
        gg = g.copy()
        for m in range(M):  # exponents held at the bound
            if x[m] <= alpha_min and g[m] > 0.0:
                A[m, :] = 0.0
                A[:, m] = 0.0
                A[m, m] = 1.0
                gg[m] = 0.0
        try:
            L = np.linalg.cholesky(A)
        except np.linalg.LinAlgError:
            lam *= 4.0
            if lam > LAMBDA_MAX:
                break
            continue
        delta = -np.linalg.solve(L.T, np.linalg.solve(L, gg))
        xt = x + delta
        xt[:M] = np.maximum(xt[:M], alpha_min)  # projection onto the feasible set
        Et = err(xt[:M], xt[M:], y, r)
        if Et < E * (1.0 - TIE):
            conv = (E - Et) <= CONV * E
            x, E = xt, Et
            lam = max(lam / 3.0, 1e-12)
            H = None
            if conv:
                break
        else:
            lam *= 4.0
            if lam > LAMBDA_MAX:
                break
    order = np.argsort(x[:M], kind="stable")
    return x[:M][order], x[M:][order], E, it


# ---------------------------------------------------------------------------
# Algorithm 1
# ---------------------------------------------------------------------------
def fit(phi, l: int, h: float, M: int, N: int, P: int, G: int, max_iter: int,
        alpha_min: float = 0.1, alpha_max: float = 1000.0, seed: int = 0, fun: int = 0,
        restarts=None):
    """Algorithm 1 for one radial function (index `fun` in a set of functions, which fixes
    the restart numbers q = fun N + iter).  Returns a dict with the best alpha, D, err and the
    per-restart results; `restarts` limits the loop to the given iterations."""
    r = grid(len(phi), h)
    y = targets(np.asarray(phi, float), l, h)
    its = range(N) if restarts is None else restarts
    per = []
    best = None
    for it in its:
        q = fun * N + it
        a0, d0, _ = genetic(q, y, r, M, P, G, alpha_min, alpha_max, seed)
        a, d, e, steps = local_search(a0, d0, y, r, alpha_min, max_iter)
        per.append({"alpha": a, "D": d, "err": e, "steps": steps, "ga_alpha": a0, "ga_D": d0})
        if best is None or e < best["err"]:
            best = {"alpha": a, "D": d, "err": e, "iter": it}
    return {"best": best, "restarts": per}
