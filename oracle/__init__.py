"""CPU oracle for the screened HSE exact-exchange build (plain C, FP64, OpenMP).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  The CUDA library never imports, links or calls it, and it
shares no code with that library.  See ``hfx_oracle.c`` for the definitions it follows
(exchange matrix Eq. vx, Schwarz screening Eq. schwarz, eight-fold symmetry, the
Cartesian-to-spherical step; Obara-Saika / Head-Gordon-Pople recurrences with the
erfc-attenuated Boys function).

Every function here is pinned by ``tests/test_oracle_*.py`` against things other
than itself: Gauss-Legendre quadrature of the Boys integrals, the closed-form (ss|ss)
integral, finite-difference derivatives of that closed form (p and d primitives),
brute-force numerical quadrature of the six-dimensional integral, the Schwarz
inequality, eight-fold symmetry, symmetry and semi-definiteness of K, and agreement
of the plain and symmetric loops.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hfx_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhfx_oracle.so")
_lib = None
_lock = threading.Lock()

MAXSPH = 5
NSPH = {0: 1, 1: 3, 2: 5}
NCART = {0: 1, 1: 3, 2: 6}
# quartet classes: pair classes ss, ps, pp, ds, dp, dd -> index hi*(hi+1)/2 + lo
PAIR_CLASSES = ["ss", "ps", "pp", "ds", "dp", "dd"]
QUARTET_CLASSES = [f"({PAIR_CLASSES[hi]}|{PAIR_CLASSES[lo]})" for hi in range(6) for lo in range(hi + 1)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math, OpenMP) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            up = ctypes.POINTER(ctypes.c_ubyte)
            lp = ctypes.POINTER(ctypes.c_longlong)
            vp = ctypes.c_void_p
            L.ora_boys.argtypes = [ctypes.c_int, ctypes.c_double, dp]
            L.ora_boys.restype = None
            L.ora_gboys.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
            L.ora_gboys.restype = None
            L.ora_basis_new.argtypes = [ctypes.c_int, dp, ctypes.c_int, ip, ip, ip, dp, dp]
            L.ora_basis_new.restype = vp
            L.ora_basis_free.argtypes = [vp]
            L.ora_basis_free.restype = None
            L.ora_n_bf.argtypes = [vp]
            L.ora_n_bf.restype = ctypes.c_int
            L.ora_basis_export.argtypes = [vp, dp, dp]
            L.ora_basis_export.restype = None
            L.ora_quartet.argtypes = [vp, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, dp]
            L.ora_quartet.restype = ctypes.c_int
            L.ora_prim_cart.argtypes = [ip, dp, dp, ctypes.c_double, dp]
            L.ora_prim_cart.restype = ctypes.c_int
            L.ora_screen_new.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int]
            L.ora_screen_new.restype = vp
            L.ora_screen_free.argtypes = [vp]
            L.ora_screen_free.restype = None
            L.ora_screen_export.argtypes = [vp, dp, up, up, dp]
            L.ora_screen_export.restype = None
            L.ora_count_quartets.argtypes = [vp, lp]
            L.ora_count_quartets.restype = None
            L.ora_build_K.argtypes = [vp, dp, ctypes.c_int, ctypes.c_int, dp]
            L.ora_build_K.restype = ctypes.c_double
            L.ora_build_K_dens.argtypes = [vp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
            L.ora_build_K_dens.restype = ctypes.c_double
            L.ora_build_K_dist.argtypes = [vp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp]
            L.ora_build_K_dist.restype = ctypes.c_double
            L.ora_dist_estimate.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.ora_dist_estimate.restype = ctypes.c_double
            L.ora_screen_export_dist.argtypes = [vp, dp, dp]
            L.ora_screen_export_dist.restype = None
            L.ora_K_block.argtypes = [vp, dp, ctypes.c_int, ctypes.c_int, dp]
            L.ora_K_block.restype = ctypes.c_int
            L.ora_trace_PK.argtypes = [ctypes.c_int, dp, dp]
            L.ora_trace_PK.restype = ctypes.c_double
            L.ora_eval_quartets.argtypes = [vp, ctypes.c_longlong, ip, ctypes.c_int]
            L.ora_eval_quartets.restype = ctypes.c_double
            L.ora_max_threads.argtypes = []
            L.ora_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def boys(mmax: int, T: float) -> np.ndarray:
    """F_m(T), m = 0..mmax."""
    out = np.zeros(mmax + 1)
    lib().ora_boys(mmax, float(T), _dp(out))
    return out


def gboys(mmax: int, T: float, kappa: float) -> np.ndarray:
    """G_m(T) = F_m(T) - kappa^{m+1/2} F_m(kappa T), m = 0..mmax."""
    out = np.zeros(mmax + 1)
    lib().ora_gboys(mmax, float(T), float(kappa), _dp(out))
    return out


def prim_cart(ls, alphas, centres, omega: float) -> np.ndarray:
    """Unnormalised primitive Cartesian [ab|cd] (weight 1), shape (nca, ncb, ncc, ncd)."""
    l4 = np.ascontiguousarray(ls, dtype=np.int32)
    a4 = np.ascontiguousarray(alphas, dtype=np.float64)
    c12 = np.ascontiguousarray(np.asarray(centres, dtype=np.float64).reshape(12))
    shape = tuple(NCART[int(l)] for l in ls)
    out = np.zeros(int(np.prod(shape)))
    rc = lib().ora_prim_cart(_ip(l4), _dp(a4), _dp(c12), float(omega), _dp(out))
    if rc != 0:
        raise ValueError("bad angular momentum")
    return out.reshape(shape)


class Basis:
    """A normalised contracted basis built from a generator ``System``."""

    def __init__(self, system):
        self.system = system
        xyz, sa, sl, sn, al, co = system.basis_arrays()
        self._keep = (xyz, sa, sl, sn, al, co)
        h = lib().ora_basis_new(int(xyz.shape[0]), _dp(xyz), int(sl.shape[0]), _ip(sa), _ip(sl),
                                _ip(sn), _dp(al), _dp(co))
        if not h:
            raise ValueError("invalid basis")
        self.h = h
        self.n_bf = lib().ora_n_bf(h)
        self.n_shells = int(sl.shape[0])
        self.shell_l = sl
        self.bf_off = np.concatenate([[0], np.cumsum([NSPH[int(l)] for l in sl])]).astype(np.int64)

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.ora_basis_free(h)
            self.h = None

    def norms(self):
        """(N_{I,m} per shell [n_shells, 5], radial weights c_k n_l(alpha_k) per primitive)."""
        nrm = np.zeros(self.n_shells * MAXSPH)
        w = np.zeros(self._keep[4].shape[0])
        lib().ora_basis_export(self.h, _dp(nrm), _dp(w))
        return nrm.reshape(self.n_shells, MAXSPH), w

    def quartet(self, I, J, K, L, omega=None) -> np.ndarray:
        """Spherical normalised (IJ|KL), shape (2lI+1, 2lJ+1, 2lK+1, 2lL+1)."""
        om = self.system.omega if omega is None else omega
        shape = tuple(NSPH[int(self.shell_l[s])] for s in (I, J, K, L))
        out = np.zeros(int(np.prod(shape)))
        rc = lib().ora_quartet(self.h, float(om), int(I), int(J), int(K), int(L), _dp(out))
        if rc != 0:
            raise IndexError("shell index out of range")
        return out.reshape(shape)


class Screen:
    """Orbital-cutoff and Schwarz screening data of a basis (Sec. 3.1)."""

    def __init__(self, basis: Basis, omega=None, tau=None, rcut=None, nthreads: int = 0):
        s = basis.system
        self.basis = basis
        self.omega = s.omega if omega is None else omega
        self.tau = s.tau if tau is None else tau
        self.rcut = s.rcut if rcut is None else rcut
        self.h = lib().ora_screen_new(basis.h, float(self.omega), float(self.tau), float(self.rcut),
                                      int(nthreads))

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.ora_screen_free(h)
            self.h = None

    def export(self):
        n = self.basis.n_shells
        Q = np.zeros(n * n)
        cut = np.zeros(n * n, dtype=np.uint8)
        kept = np.zeros(n * n, dtype=np.uint8)
        qmax = np.zeros(1)
        lib().ora_screen_export(self.h, _dp(Q), cut.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                                kept.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), _dp(qmax))
        return Q.reshape(n, n), cut.reshape(n, n).astype(bool), kept.reshape(n, n).astype(bool), float(qmax[0])

    def count_quartets(self) -> np.ndarray:
        """Kept canonical quartets per class (21 entries) and the total (entry 21)."""
        out = np.zeros(22, dtype=np.int64)
        lib().ora_count_quartets(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
        return out

    def build_K(self, P: np.ndarray, mode: str = "sym", nthreads: int = 0):
        """K and E_K = tr(PK).  mode 'plain' = four-fold definition loop, 'sym' = canonical."""
        n = self.basis.n_bf
        P = np.ascontiguousarray(P, dtype=np.float64)
        assert P.shape == (n, n)
        K = np.zeros((n, n))
        ek = lib().ora_build_K(self.h, _dp(P), 0 if mode == "plain" else 1, int(nthreads), _dp(K))
        return K, float(ek)

    def build_K_dens(self, P: np.ndarray, dens_tau: float, mode: str = "sym", nthreads: int = 0):
        """K and E_K with the density-weighted quartet test added to the keep rule:
        Q_IJ Q_KL max(|P| over the blocks (J,L), (J,K), (I,L), (I,K)) >= dens_tau.
        Also returns the block maxima of |P| (n_shells x n_shells)."""
        n = self.basis.n_bf
        P = np.ascontiguousarray(P, dtype=np.float64)
        assert P.shape == (n, n)
        K = np.zeros((n, n))
        ns = self.basis.n_shells
        pm = np.zeros(ns * ns)
        ek = lib().ora_build_K_dens(self.h, _dp(P), 0 if mode == "plain" else 1, int(nthreads),
                                    float(dens_tau), _dp(K), _dp(pm))
        return K, float(ek), pm.reshape(ns, ns)

    def build_K_dist(self, P: np.ndarray, dist_tau: float, mode: str = "sym", nthreads: int = 0):
        """K with the distance-aware quartet test (hfx_oracle.c, ora_build_K_dist)."""
        P = np.ascontiguousarray(P, dtype=np.float64)
        nb = self.basis.n_bf
        K = np.zeros((nb, nb))
        e = lib().ora_build_K_dist(self.h, _dp(P), 0 if mode == "plain" else 1, nthreads, float(dist_tau), _dp(K))
        return K, e

    def dist_estimate(self, I: int, J: int, K: int, L: int) -> float:
        """Q_IJ Q_KL exp(-kappa rho R^2) of the distance-aware test."""
        return lib().ora_dist_estimate(self.h, int(I), int(J), int(K), int(L))

    def export_dist(self):
        """Pair data of the distance-aware test: (n, n, 4) centre xyz and spread, (n, n) the
        smallest exponent sum."""
        ns = self.basis.n_shells
        pst = np.zeros(ns * ns * 4)
        pexp = np.zeros(ns * ns)
        lib().ora_screen_export_dist(self.h, _dp(pst), _dp(pexp))
        return pst.reshape(ns, ns, 4), pexp.reshape(ns, ns)

    def K_block(self, P: np.ndarray, I: int, Ks: int) -> np.ndarray:
        P = np.ascontiguousarray(P, dtype=np.float64)
        ni, nk = NSPH[int(self.basis.shell_l[I])], NSPH[int(self.basis.shell_l[Ks])]
        out = np.zeros(ni * nk)
        rc = lib().ora_K_block(self.h, _dp(P), int(I), int(Ks), _dp(out))
        if rc != 0:
            raise IndexError("shell index out of range")
        return out.reshape(ni, nk)

    def eval_quartets(self, ijkl: np.ndarray, nthreads: int = 0) -> float:
        q = np.ascontiguousarray(ijkl, dtype=np.int32)
        return float(lib().ora_eval_quartets(self.h, int(q.shape[0]), _ip(q), int(nthreads)))


def trace_PK(P: np.ndarray, K: np.ndarray) -> float:
    P = np.ascontiguousarray(P, dtype=np.float64)
    K = np.ascontiguousarray(K, dtype=np.float64)
    return float(lib().ora_trace_PK(int(P.shape[0]), _dp(P), _dp(K)))


def max_threads() -> int:
    return int(lib().ora_max_threads())
