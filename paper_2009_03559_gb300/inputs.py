"""Seeded synthetic inputs shaped like the paper's Si64 benchmark systems.

The paper benchmarks bulk silicon with 64 atoms per cell, an SZ basis (s and p
shells: 128 shells, 256 functions) and a DZP basis (2s 2p 1d: 320 shells, 832
functions) (Sec. "Results and discussion", figure table of Si64 shell counts).
Its real numerical orbitals and pseudopotentials are not available, so these
generators draw systems of the same shapes from seeded random numbers:

* ``cluster``: atoms on a cubic lattice (spacing ``h``) with uniform jitter,
  one s and one p shell per atom (SZ-like).
* ``diamond``: conventional 8-site diamond cells (lattice constant ``a``) with
  uniform jitter, shells s, s, p, p, d per atom (DZP-like, spherical d).

Every shell is a contraction of ``nprim`` primitives whose exponents are
log-uniform in a range and sorted in descending order; the raw contraction
weights are uniform in [0.1, 1).  Normalisation is NOT done here: each consumer
(the CPU oracle and the CUDA library) normalises the raw weights itself.

The density matrix is P = C C^T with C an orthonormal block (Q factor of the
Householder QR of a seeded standard-normal matrix), optionally set to zero
between functions whose atoms are further apart than a truncation radius.

This module holds no integral arithmetic; it only produces arrays.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

# angular momentum -> number of spherical functions (2l+1)
N_SPH = {0: 1, 1: 3, 2: 5}

OMEGA_HSE = 0.11  # bohr^-1, HSE06 range-separation parameter


@dataclass
class System:
    """One molecule/cluster: atoms, raw contracted shells and screening options."""

    name: str
    xyz: np.ndarray            # (n_atoms, 3) float64, bohr
    shell_atom: np.ndarray     # (n_shells,) int32
    shell_l: np.ndarray        # (n_shells,) int32, 0..2
    shell_nprim: np.ndarray    # (n_shells,) int32
    alpha: np.ndarray          # (sum nprim,) float64, bohr^-2
    coef: np.ndarray           # (sum nprim,) float64, raw weights (unnormalised)
    omega: float = OMEGA_HSE
    tau: float = 1e-10         # Schwarz threshold
    rcut: float = 0.0          # orbital cutoff radius (bohr); <= 0 means none
    seed: int = 0
    kind: str = ""
    rng_state: dict = field(default=None, repr=False)  # generator state after the basis draws

    @property
    def n_atoms(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_shells(self) -> int:
        return int(self.shell_l.shape[0])

    @property
    def shell_nbf(self) -> np.ndarray:
        return np.array([N_SPH[int(l)] for l in self.shell_l], dtype=np.int32)

    @property
    def shell_offset(self) -> np.ndarray:
        nb = self.shell_nbf
        return np.concatenate([[0], np.cumsum(nb)[:-1]]).astype(np.int64)

    @property
    def n_bf(self) -> int:
        return int(self.shell_nbf.sum())

    @property
    def bf_atom(self) -> np.ndarray:
        return np.repeat(self.shell_atom, self.shell_nbf).astype(np.int32)

    def basis_arrays(self):
        """Contiguous arrays in the order the C interfaces take them."""
        return (
            np.ascontiguousarray(self.xyz, dtype=np.float64),
            np.ascontiguousarray(self.shell_atom, dtype=np.int32),
            np.ascontiguousarray(self.shell_l, dtype=np.int32),
            np.ascontiguousarray(self.shell_nprim, dtype=np.int32),
            np.ascontiguousarray(self.alpha, dtype=np.float64),
            np.ascontiguousarray(self.coef, dtype=np.float64),
        )


def _site_block_cubic(n_atoms: int):
    """First n sites, lexicographic (i, j, k), of the smallest m^3 block holding n."""
    m = 1
    while m ** 3 < n_atoms:
        m += 1
    sites = [(i, j, k) for i in range(m) for j in range(m) for k in range(m)]
    return np.array(sites[:n_atoms], dtype=np.float64)


_DIAMOND_BASIS = np.array(
    [
        [0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0],
        [0.25, 0.25, 0.25], [0.25, 0.75, 0.75], [0.75, 0.25, 0.75], [0.75, 0.75, 0.25],
    ]
)


def _site_block_diamond(n_atoms: int):
    """First n sites, lexicographic (i, j, k, basis), of the smallest m^3 cell block."""
    m = 1
    while 8 * m ** 3 < n_atoms:
        m += 1
    sites = []
    for i in range(m):
        for j in range(m):
            for k in range(m):
                for b in range(8):
                    sites.append(np.array([i, j, k], dtype=np.float64) + _DIAMOND_BASIS[b])
    return np.array(sites[:n_atoms])


def _draw_shells(rng, n_atoms, shell_ls, nprim, alpha_lo, alpha_hi):
    shell_atom, shell_l, shell_nprim, alpha, coef = [], [], [], [], []
    for a in range(n_atoms):
        for l in shell_ls:
            ex = np.exp(rng.uniform(math.log(alpha_lo), math.log(alpha_hi), nprim))
            ex = np.sort(ex)[::-1]
            c = rng.uniform(0.1, 1.0, nprim)
            shell_atom.append(a)
            shell_l.append(l)
            shell_nprim.append(nprim)
            alpha.extend(ex.tolist())
            coef.extend(c.tolist())
    return (
        np.array(shell_atom, dtype=np.int32),
        np.array(shell_l, dtype=np.int32),
        np.array(shell_nprim, dtype=np.int32),
        np.array(alpha, dtype=np.float64),
        np.array(coef, dtype=np.float64),
    )


def cluster_system(n_atoms: int, seed: int, h: float = 2.5, jitter: float = 0.3,
                   alpha_range=(0.1, 20.0), nprim: int = 3, tau: float = 1e-10,
                   rcut: float = 0.0, omega: float = OMEGA_HSE) -> System:
    """Jittered cubic cluster; one s and one p shell per atom."""
    rng = np.random.default_rng(seed)
    xyz = h * _site_block_cubic(n_atoms) + rng.uniform(-jitter, jitter, (n_atoms, 3))
    sa, sl, sn, al, co = _draw_shells(rng, n_atoms, (0, 1), nprim, *alpha_range)
    return System(f"cluster{n_atoms}", xyz, sa, sl, sn, al, co, omega=omega, tau=tau,
                  rcut=rcut, seed=seed, kind="cluster", rng_state=rng.bit_generator.state)


def diamond_system(n_atoms: int, seed: int, a: float = 10.26, jitter: float = 0.05,
                   alpha_range=(0.08, 8.0), nprim: int = 3, tau: float = 1e-8,
                   rcut: float = 6.0, omega: float = OMEGA_HSE) -> System:
    """Jittered diamond-lattice piece; shells s, s, p, p, d (spherical) per atom."""
    rng = np.random.default_rng(seed)
    xyz = a * _site_block_diamond(n_atoms) + rng.uniform(-jitter, jitter, (n_atoms, 3))
    sa, sl, sn, al, co = _draw_shells(rng, n_atoms, (0, 0, 1, 1, 2), nprim, *alpha_range)
    return System(f"diamond{n_atoms}", xyz, sa, sl, sn, al, co, omega=omega, tau=tau,
                  rcut=rcut, seed=seed, kind="diamond", rng_state=rng.bit_generator.state)


def density_matrix(system: System, seed: int | None = None, truncate_bohr: float | None = None,
                   n_occ: int | None = None) -> np.ndarray:
    """P = C C^T, C = Q factor of a seeded N(0,1) matrix (n_bf x n_occ).

    With ``seed=None`` the generator continues from the state left after the basis
    draws of ``system`` (one seed per system); otherwise a fresh generator with that
    seed is used (one seed per request).  ``truncate_bohr`` zeroes P between
    functions on atoms further apart than that distance.
    """
    if seed is None:
        rng = np.random.default_rng()
        rng.bit_generator.state = system.rng_state
    else:
        rng = np.random.default_rng(seed)
    n = system.n_bf
    k = n // 2 if n_occ is None else n_occ
    g = rng.standard_normal((n, k))
    c, _ = np.linalg.qr(g)
    p = c @ c.T
    p = 0.5 * (p + p.T)
    if truncate_bohr is not None:
        ba = system.bf_atom
        d = np.linalg.norm(system.xyz[:, None, :] - system.xyz[None, :, :], axis=-1)
        far = d[ba][:, ba] > truncate_bohr
        p[far] = 0.0
    return np.ascontiguousarray(p)


# ---------------------------------------------------------------------------
# The five workloads (seed = 1000 * config index + system index)
# ---------------------------------------------------------------------------

def config0():
    """16-atom s,p cluster, 64 functions, tau 1e-10, no cutoff; P from a 64x32 block."""
    s = cluster_system(16, seed=0, tau=1e-10, rcut=0.0)
    return s, density_matrix(s)


def config1(n_atoms: int = 64):
    """Diamond piece (64 atoms = 2x2x2 cells at a=10.26), DZP-like, tau 1e-8, r_c 6,
    P truncated beyond 10 bohr."""
    s = diamond_system(n_atoms, seed=1000, tau=1e-8, rcut=6.0)
    return s, density_matrix(s, truncate_bohr=10.0)


def config2_systems(n_systems: int = 32, n_lo: int = 8, n_hi: int = 128):
    """Batch of independent systems; atom count uniform in [n_lo, n_hi], generator by coin."""
    meta = np.random.default_rng(2999)
    out = []
    for i in range(n_systems):
        n = int(meta.integers(n_lo, n_hi + 1))
        coin = int(meta.integers(0, 2))
        seed = 2000 + i
        if coin == 0:
            s = cluster_system(n, seed=seed, tau=1e-10, rcut=0.0)
            p = density_matrix(s)
        else:
            s = diamond_system(n, seed=seed, tau=1e-8, rcut=6.0)
            p = density_matrix(s, truncate_bohr=10.0)
        out.append((s, p))
    return out


def config3(n_atoms: int = 216):
    """Diamond 3x3x3 cells (216 atoms, 2808 functions), truncated P, mixed precision."""
    s = diamond_system(n_atoms, seed=3000, tau=1e-8, rcut=6.0)
    return s, density_matrix(s, truncate_bohr=10.0)


def config4_requests(n_requests: int = 2000, rate_per_s: float = 50.0, pool: int = 64,
                     n_lo: int = 16, n_hi: int = 512):
    """Serving stream: Poisson arrivals, systems drawn from a seeded pool of `pool`
    systems with log-uniform atom counts; each request carries its own P seed."""
    meta = np.random.default_rng(4999)
    systems = []
    for i in range(pool):
        n = int(round(math.exp(meta.uniform(math.log(n_lo), math.log(n_hi)))))
        coin = int(meta.integers(0, 2))
        seed = 4000 + i
        if coin == 0:
            systems.append(("cluster", n, seed))
        else:
            systems.append(("diamond", n, seed))
    gaps = meta.exponential(1.0 / rate_per_s, n_requests)
    t = np.cumsum(gaps)
    which = meta.integers(0, pool, n_requests)
    reqs = [(float(t[r]), int(which[r]), 100000 + r) for r in range(n_requests)]
    return systems, reqs


def make_system(kind: str, n_atoms: int, seed: int) -> System:
    if kind == "cluster":
        return cluster_system(n_atoms, seed=seed, tau=1e-10, rcut=0.0)
    return diamond_system(n_atoms, seed=seed, tau=1e-8, rcut=6.0)


def truncation_for(kind: str):
    return None if kind == "cluster" else 10.0


# ---------------------------------------------------------------------------
# Periodic images (the lattice sums of Eq. vx): a home cell, its lattice, and a real-space
# density P^R between functions of the home cell and of the cell shifted by R.
# ---------------------------------------------------------------------------

@dataclass
class PeriodicSystem:
    """Home cell (``cell``: a System whose atoms lie in the home cell) and the lattice
    (rows of ``lattice`` are the three cell vectors, bohr)."""

    cell: System
    lattice: np.ndarray

    def shift(self, n) -> np.ndarray:
        return np.asarray(n, dtype=np.float64) @ self.lattice


def periodic_diamond(cells=(1, 1, 1), seed: int = 5000, a: float = 10.26, jitter: float = 0.05,
                     spacing: float | None = None, tau: float = 1e-8, rcut: float = 6.0) -> PeriodicSystem:
    """Diamond crystal: the home cell holds cells[0] x cells[1] x cells[2] conventional
    8-atom cells (DZP-like shells as ``diamond_system``); lattice vectors are the home
    cell's edges.  ``spacing`` (bohr) replaces the edge length of the lattice (not the atom
    positions): a large spacing isolates the images."""
    n = 8 * int(np.prod(cells))
    rng = np.random.default_rng(seed)
    sites = []
    for i in range(cells[0]):
        for j in range(cells[1]):
            for k in range(cells[2]):
                for b in range(8):
                    sites.append(np.array([i, j, k], dtype=np.float64) + _DIAMOND_BASIS[b])
    xyz = a * np.array(sites) + rng.uniform(-jitter, jitter, (n, 3))
    sa, sl, sn, al, co = _draw_shells(rng, n, (0, 0, 1, 1, 2), 3, 0.08, 8.0)
    cell = System(f"pdiamond{n}", xyz, sa, sl, sn, al, co, tau=tau, rcut=rcut, seed=seed, kind="diamond",
                  rng_state=rng.bit_generator.state)
    edge = np.array(cells, dtype=np.float64) * (a if spacing is None else spacing)
    return PeriodicSystem(cell, np.diag(edge))


def image_system(ps: PeriodicSystem, cell_list) -> System:
    """The home cell's shells repeated in every cell of ``cell_list`` (cell-major order:
    all shells of cell_list[0], then of cell_list[1], ...), the same exponents and weights."""
    c = ps.cell
    n_at = c.n_atoms
    xyz = np.concatenate([c.xyz + ps.shift(n) for n in cell_list])
    k = len(cell_list)
    shell_atom = np.concatenate([c.shell_atom + i * n_at for i in range(k)]).astype(np.int32)
    return System(f"{c.name}x{k}", xyz, shell_atom, np.tile(c.shell_l, k), np.tile(c.shell_nprim, k),
                  np.tile(c.alpha, k), np.tile(c.coef, k), omega=c.omega, tau=c.tau, rcut=c.rcut,
                  seed=c.seed, kind=c.kind)


def periodic_density(ps: PeriodicSystem, r_cells: int, seed: int, truncate_bohr: float = 10.0,
                     decay_bohr: float = 3.0) -> dict:
    """Synthetic real-space density blocks P^R (n_bf x n_bf) for the cells R with every
    |R_i| <= r_cells: N(0,1) values damped by exp(-d/decay_bohr), d the distance between
    the two functions' atoms, zero beyond truncate_bohr, symmetrised so that
    P^{-R} = (P^R)^T.  A stand-in for the Brillouin-zone integral of the paper's P^N."""
    rng = np.random.default_rng(seed)
    c = ps.cell
    ba = c.bf_atom
    cells = [(i, j, k) for i in range(-r_cells, r_cells + 1) for j in range(-r_cells, r_cells + 1)
             for k in range(-r_cells, r_cells + 1)]
    raw = {}
    for R in cells:
        d = np.linalg.norm(c.xyz[ba][:, None, :] - (c.xyz[ba] + ps.shift(R))[None, :, :], axis=-1)
        m = rng.standard_normal((c.n_bf, c.n_bf)) * np.exp(-d / decay_bohr)
        m[d > truncate_bohr] = 0.0
        raw[R] = m
    P = {}
    for R in cells:
        mR = tuple(-x for x in R)
        P[R] = 0.5 * (raw[R] + raw[mR].T)
    return P


def periodic_sc(a: float = 6.0, seed: int = 5100, jitter: float = 0.3, tau: float = 1e-10,
                rcut: float = 3.5, spacing: float | None = None, shells=(0, 1)) -> PeriodicSystem:
    """Simple cubic crystal with one atom per cell (by default s and p shells, as
    ``cluster_system``; ``shells`` lists the angular momenta): the smallest periodic case.
    ``spacing`` replaces the lattice constant of the images."""
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(-jitter, jitter, (1, 3))
    sa, sl, sn, al, co = _draw_shells(rng, 1, tuple(shells), 3, 0.1, 20.0)
    cell = System("psc1", xyz, sa, sl, sn, al, co, tau=tau, rcut=rcut, seed=seed, kind="cluster",
                  rng_state=rng.bit_generator.state)
    return PeriodicSystem(cell, np.eye(3) * (a if spacing is None else spacing))


# ---------------------------------------------------------------------------
# Synthetic numerical radial functions for the NAO -> GTO fit
# ---------------------------------------------------------------------------
@dataclass
class RadialSet:
    """Radial functions phi(r_i) on the grid r_i = i h (i = 1..n_r), one row per function."""
    phi: np.ndarray    # (n_fun, n_r)
    l: np.ndarray      # (n_fun,) angular momenta
    h: float
    r_cut: float
    zeta: np.ndarray   # the Slater exponents they were drawn with
    seed: int


def confined_slater(l: int, zeta: float, r: np.ndarray, r_cut: float) -> np.ndarray:
    """r^l exp(-zeta r) (1 - (r / r_cut)^2)^2 inside r_cut, exactly zero beyond: a stand-in for a
    numerical atomic orbital (strictly confined, value and slope zero at the confining radius)."""
    x = np.clip(r / r_cut, 0.0, 1.0)
    f = r ** l * np.exp(-zeta * r) * (1.0 - x * x) ** 2
    return np.where(r < r_cut, f, 0.0)


def nao_set(n_elements: int = 4, seed: int = 6000, r_cut: float = 6.0, n_r: int = 512) -> RadialSet:
    """DZP-like radial sets (2s, 2p, 1d per element: 5 functions each), Slater exponents
    log-uniform per element (first zeta in [1.2, 2.4], second zeta 0.45-0.65 of it, d in
    [0.9, 1.8]), normalised so that sum_i phi_i^2 r_i^2 h = 1."""
    rng = np.random.default_rng(seed)
    h = r_cut / n_r
    r = h * np.arange(1, n_r + 1, dtype=np.float64)
    rows, ls, zs = [], [], []
    for _ in range(n_elements):
        for l in (0, 1):
            z1 = float(np.exp(rng.uniform(np.log(1.2), np.log(2.4))))
            z2 = z1 * float(rng.uniform(0.45, 0.65))
            for z in (z1, z2):
                rows.append(confined_slater(l, z, r, r_cut))
                ls.append(l)
                zs.append(z)
        z = float(np.exp(rng.uniform(np.log(0.9), np.log(1.8))))
        rows.append(confined_slater(2, z, r, r_cut))
        ls.append(2)
        zs.append(z)
    phi = np.array(rows)
    phi /= np.sqrt((phi * phi * (r * r)[None, :]).sum(axis=1) * h)[:, None]
    return RadialSet(phi, np.array(ls, dtype=np.int32), h, r_cut, np.array(zs), seed)
