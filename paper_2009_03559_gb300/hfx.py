"""Python binding of the C ABI in include/hfx.h (argument marshalling only).

Every step of the exchange build runs in the CUDA library ``_build/libhfx.so``; this
module loads it with ctypes and passes pointers.  There is no CPU path: if the library
or a CUDA device is missing, constructing ``HFX`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libhfx.so")

HFX_FP64, HFX_MIXED = 0, 1
HFX_SCHED_QUARTET, HFX_SCHED_PAIR, HFX_SCHED_DYNAMIC = 0, 1, 2
ERR_NAMES = {0: "OK", -1: "ARG", -2: "UNSUPPORTED_L", -3: "OOM", -4: "CUDA", -5: "STATE", -6: "TIMEOUT",
             -7: "ADMISSION"}
REQ_DONE, REQ_QUEUED, REQ_RUNNING = 0, 1, 2

PAIR_CLASSES = ["ss", "ps", "pp", "ds", "dp", "dd"]
QUARTET_CLASSES = [f"({PAIR_CLASSES[hi]}|{PAIR_CLASSES[lo]})" for hi in range(6) for lo in range(hi + 1)]
# spherical integrals per quartet of each class: product of (2l+1) over its four shells
_PAIR_SIZE = [1, 3, 9, 5, 15, 25]  # ss, ps, pp, ds, dp, dd
CLASS_SPH_SIZE = [_PAIR_SIZE[hi] * _PAIR_SIZE[lo] for hi in range(6) for lo in range(hi + 1)]
# quartet classes without d shells (bra and ket pair classes among ss, ps, pp)
SP_CLASS_MASK = sum(1 << (hi * (hi + 1) // 2 + lo) for hi in range(3) for lo in range(hi + 1))
ALL_CLASS_MASK = (1 << 21) - 1
FP32_CLASSES_DEFAULT = 0xFFFFF  # HFX_FP32_CLASSES_DEFAULT in include/hfx.h


class Options(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_double), ("schwarz_tau", ctypes.c_double), ("rcut_bohr", ctypes.c_double),
                ("prim_tau", ctypes.c_double), ("fp32_tau", ctypes.c_double), ("precision", ctypes.c_int),
                ("schedule", ctypes.c_int), ("skip_zero_p", ctypes.c_int), ("fp32_class_mask", ctypes.c_int),
                ("fp32_pmax_global", ctypes.c_int), ("reserved", ctypes.c_int * 1),
                ("density_tau", ctypes.c_double), ("dist_tau", ctypes.c_double)]


class NaoOptions(ctypes.Structure):
    _fields_ = [("n_gauss", ctypes.c_int), ("n_restarts", ctypes.c_int), ("population", ctypes.c_int),
                ("generations", ctypes.c_int), ("max_iter", ctypes.c_int), ("alpha_min", ctypes.c_double),
                ("alpha_max", ctypes.c_double), ("seed", ctypes.c_ulonglong)]


class ServerOptions(ctypes.Structure):
    _fields_ = [("hbm_budget_gb", ctypes.c_double), ("max_step_quartets", ctypes.c_double),
                ("max_inflight", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("precision", ctypes.c_int), ("reserved", ctypes.c_int * 5)]


class Result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32), ("system_id", ctypes.c_int32),
                ("step_size", ctypes.c_int32), ("pad", ctypes.c_int32), ("energy", ctypes.c_double),
                ("t_submit_ms", ctypes.c_double), ("t_admit_ms", ctypes.c_double), ("t_done_ms", ctypes.c_double),
                ("ms_step", ctypes.c_double), ("n_quartets", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("n_submitted", "n_done", "n_failed", "n_steps", "n_queued",
                                              "n_running", "quartets_done", "bytes_resident", "bytes_requests",
                                              "bytes_peak")] + \
               [("max_step_size", ctypes.c_int32), ("max_steps_inflight", ctypes.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("n_pairs_cutoff", ctypes.c_int64), ("n_pairs_kept", ctypes.c_int64),
                ("n_quartets", ctypes.c_int64), ("n_quartets_class", ctypes.c_int64 * 21),
                ("prim_quartets_class", ctypes.c_int64 * 21),
                ("quartets_evaluated_class", ctypes.c_int64 * 21),
                ("quartets_fp32_class", ctypes.c_int64 * 21), ("flops_fp32", ctypes.c_double),
                ("flops_fp64", ctypes.c_double), ("flops_class", ctypes.c_double * 21),
                ("group_size_class", ctypes.c_int32 * 21),
                ("ms_pairs", ctypes.c_double), ("ms_build", ctypes.c_double),
                ("ms_class", ctypes.c_double * 21), ("energy", ctypes.c_double),
                ("flops_recurrence", ctypes.c_double), ("special_evals", ctypes.c_double),
                ("streams_class", ctypes.c_int32 * 21), ("reserved_stats", ctypes.c_int32 * 1),
                ("flops_recurrence_class", ctypes.c_double * 21)]

    def as_dict(self):
        return {
            "n_pairs_cutoff": int(self.n_pairs_cutoff), "n_pairs_kept": int(self.n_pairs_kept),
            "n_quartets": int(self.n_quartets), "n_quartets_class": [int(x) for x in self.n_quartets_class],
            "prim_quartets_class": [int(x) for x in self.prim_quartets_class],
            "quartets_evaluated_class": [int(x) for x in self.quartets_evaluated_class],
            "quartets_fp32_class": [int(x) for x in self.quartets_fp32_class],
            "flops_fp32": float(self.flops_fp32),
            "flops_fp64": float(self.flops_fp64), "flops_class": [float(x) for x in self.flops_class],
            "group_size_class": [int(x) for x in self.group_size_class], "ms_pairs": float(self.ms_pairs),
            "ms_build": float(self.ms_build), "ms_class": [float(x) for x in self.ms_class],
            "energy": float(self.energy),
            "flops_recurrence": float(self.flops_recurrence), "special_evals": float(self.special_evals),
            "streams_class": [int(x) for x in self.streams_class],
            "flops_recurrence_class": [float(x) for x in self.flops_recurrence_class],
        }


class BatchStats(ctypes.Structure):
    _fields_ = [("n_quartets", ctypes.c_int64), ("ms_last", ctypes.c_double),
                ("group_size_class", ctypes.c_int32 * 21), ("chunk_class", ctypes.c_int32 * 21),
                ("tune_ms_class", ctypes.c_double * 21), ("tune_window_class", ctypes.c_int64 * 21),
                ("streams_class", ctypes.c_int32 * 21), ("tune_kept", ctypes.c_int32),
                ("tune_full_default_ms", ctypes.c_double), ("tune_full_tuned_ms", ctypes.c_double),
                ("branches", ctypes.c_int32), ("reserved_b", ctypes.c_int32 * 1)]

    def as_dict(self):
        return {"n_quartets": int(self.n_quartets), "ms_last": float(self.ms_last),
                "group_size_class": [int(x) for x in self.group_size_class],
                "chunk_class": [int(x) for x in self.chunk_class],
                "tune_ms_class": [float(x) for x in self.tune_ms_class],
                "tune_window_class": [int(x) for x in self.tune_window_class],
                "streams_class": [int(x) for x in self.streams_class], "tune_kept": int(self.tune_kept),
                "tune_full_default_ms": float(self.tune_full_default_ms),
                "tune_full_tuned_ms": float(self.tune_full_tuned_ms), "branches": int(self.branches)}


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libhfx.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    L.hfx_default_options.argtypes = [ctypes.POINTER(Options)]
    L.hfx_default_options.restype = None
    L.hfx_init_basis.argtypes = [ctypes.POINTER(vp), ctypes.c_int, dp, ctypes.c_int, ip, ip, ip, dp, dp,
                                 ctypes.POINTER(Options), vp]
    L.hfx_init_basis.restype = ctypes.c_int
    L.hfx_build_pairs.argtypes = [vp]
    L.hfx_build_pairs.restype = ctypes.c_int
    L.hfx_build_K.argtypes = [vp, vp, vp, ctypes.c_int]
    L.hfx_build_K.restype = ctypes.c_int
    L.hfx_build_K_host.argtypes = [vp, dp, dp]
    L.hfx_build_K_host.restype = ctypes.c_int
    L.hfx_energy_device.argtypes = [vp]
    L.hfx_energy_device.restype = vp
    L.hfx_energy.argtypes = [vp, dp]
    L.hfx_energy.restype = ctypes.c_int
    L.hfx_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    L.hfx_get_stats.restype = ctypes.c_int
    L.hfx_set_group_size.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.hfx_set_group_size.restype = ctypes.c_int
    L.hfx_debug_fail_alloc.argtypes = [ctypes.c_int]
    L.hfx_debug_fail_alloc.restype = ctypes.c_int
    L.hfx_measure_fp64_lane_cost.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.hfx_measure_fp64_lane_cost.restype = ctypes.c_int
    L.hfx_set_streams.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.hfx_set_streams.restype = ctypes.c_int
    L.hfx_set_timing.argtypes = [vp, ctypes.c_int]
    L.hfx_set_timing.restype = ctypes.c_int
    L.hfx_n_basis.argtypes = [vp]
    L.hfx_n_basis.restype = ctypes.c_int
    L.hfx_get_pairs.argtypes = [vp, ip, ip, dp, ctypes.c_int64]
    L.hfx_get_pairs.restype = ctypes.c_int64
    L.hfx_get_cta_busy.argtypes = [vp, dp, ctypes.c_int]
    L.hfx_get_cta_busy.restype = ctypes.c_int
    L.hfx_last_error.argtypes = [vp]
    L.hfx_last_error.restype = ctypes.c_char_p
    L.hfx_free.argtypes = [vp]
    L.hfx_free.restype = None
    pp = ctypes.POINTER(ctypes.c_void_p)
    L.hfx_batch_create.argtypes = [ctypes.POINTER(vp), pp, ctypes.c_int, vp]
    L.hfx_batch_create.restype = ctypes.c_int
    L.hfx_batch_tune.argtypes = [vp, pp, pp, ip]
    L.hfx_batch_tune.restype = ctypes.c_int
    L.hfx_batch_run.argtypes = [vp, pp, pp, ip]
    L.hfx_batch_run.restype = ctypes.c_int
    L.hfx_batch_set_branches.argtypes = [vp, ctypes.c_int]
    L.hfx_batch_set_branches.restype = ctypes.c_int
    L.hfx_batch_set_graph.argtypes = [vp, ctypes.c_int]
    L.hfx_batch_set_graph.restype = ctypes.c_int
    L.hfx_batch_set_tune_target.argtypes = [vp, ctypes.c_double]
    L.hfx_batch_set_tune_target.restype = ctypes.c_int
    L.hfx_batch_get_stats.argtypes = [vp, ctypes.POINTER(BatchStats)]
    L.hfx_batch_get_stats.restype = ctypes.c_int
    L.hfx_batch_free.argtypes = [vp]
    L.hfx_batch_free.restype = None
    L.hfx_build_K_batched.argtypes = [pp, pp, pp, ip, ctypes.c_int]
    L.hfx_build_K_batched.restype = ctypes.c_int
    L.hfx_energy_noalloc.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp, vp]
    L.hfx_energy_noalloc.restype = ctypes.c_int
    L.hfx_measure_fma_peak.argtypes = [dp, dp]
    L.hfx_measure_fma_peak.restype = ctypes.c_int
    L.hfx_build_K_part.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.hfx_build_K_part.restype = ctypes.c_int
    L.hfx_init_periodic.argtypes = [ctypes.POINTER(vp), ctypes.c_int, dp, dp, ctypes.c_int, ip, ip, ip, dp, dp,
                                    ctypes.POINTER(Options), vp]
    L.hfx_init_periodic.restype = ctypes.c_int
    L.hfx_periodic_cells.argtypes = [vp, ip, ctypes.c_int]
    L.hfx_periodic_cells.restype = ctypes.c_int
    L.hfx_build_K_periodic.argtypes = [vp, ctypes.c_int, ip, vp, ctypes.c_int, ip, vp]
    L.hfx_build_K_periodic.restype = ctypes.c_int
    i64p = ctypes.POINTER(ctypes.c_int64)
    L.hfx_part_range.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, i64p, i64p]
    L.hfx_part_range.restype = ctypes.c_int
    L.hfx_device_bytes.argtypes = [vp]
    L.hfx_device_bytes.restype = ctypes.c_int64
    u64p = ctypes.POINTER(ctypes.c_uint64)
    L.hfx_server_default_options.argtypes = [ctypes.POINTER(ServerOptions)]
    L.hfx_server_default_options.restype = None
    L.hfx_server_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ServerOptions)]
    L.hfx_server_create.restype = ctypes.c_int
    L.hfx_server_add_system.argtypes = [vp, vp, ip]
    L.hfx_server_add_system.restype = ctypes.c_int
    L.hfx_serve_submit.argtypes = [vp, ctypes.c_int, vp, vp, vp, u64p]
    L.hfx_serve_submit.restype = ctypes.c_int
    L.hfx_serve_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(Result)]
    L.hfx_serve_poll.restype = ctypes.c_int
    L.hfx_serve_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(Result)]
    L.hfx_serve_wait.restype = ctypes.c_int
    L.hfx_serve_release.argtypes = [vp, ctypes.c_uint64]
    L.hfx_serve_release.restype = ctypes.c_int
    L.hfx_serve_progress.argtypes = [vp]
    L.hfx_serve_progress.restype = ctypes.c_int
    L.hfx_serve_drain.argtypes = [vp, ctypes.c_double]
    L.hfx_serve_drain.restype = ctypes.c_int
    L.hfx_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    L.hfx_server_get_stats.restype = ctypes.c_int
    L.hfx_server_last_error.argtypes = [vp]
    L.hfx_server_last_error.restype = ctypes.c_char_p
    L.hfx_server_free.argtypes = [vp]
    L.hfx_server_free.restype = None
    nop = ctypes.POINTER(NaoOptions)
    L.hfx_nao_default_options.argtypes = [nop]
    L.hfx_nao_default_options.restype = None
    L.hfx_nao_fit.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, nop, vp, vp, vp, vp, vp, vp, vp,
                              vp, vp]
    L.hfx_nao_fit.restype = ctypes.c_int
    L.hfx_nao_genetic.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, nop, vp, vp, vp, vp]
    L.hfx_nao_genetic.restype = ctypes.c_int
    L.hfx_nao_local.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, nop, vp, vp, vp, vp, vp]
    L.hfx_nao_local.restype = ctypes.c_int
    L.hfx_nao_project.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                  vp, vp, vp, vp, vp]
    L.hfx_nao_project.restype = ctypes.c_int
    _lib = L
    return L


class HFXError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hfx error {code} ({ERR_NAMES.get(code, '?')}): {msg}")
        self.code = code


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def part_range(count, part, n_parts):
    """[q0, q1) of a list of `count` items owned by partition `part` of n_parts (C library)."""
    q0, q1 = ctypes.c_int64(), ctypes.c_int64()
    rc = load_library().hfx_part_range(int(count), int(part), int(n_parts), ctypes.byref(q0), ctypes.byref(q1))
    if rc != 0:
        raise HFXError(rc, "invalid partition")
    return q0.value, q1.value


def default_options() -> Options:
    o = Options()
    load_library().hfx_default_options(ctypes.byref(o))
    return o


def measure_fp64_lane_cost():
    """(ms with 32 active lanes, ms with 1 active lane) of the same FP64 FMA-chain kernel."""
    L = load_library()
    a, b = ctypes.c_double(), ctypes.c_double()
    rc = L.hfx_measure_fp64_lane_cost(ctypes.byref(a), ctypes.byref(b))
    if rc != 0:
        raise HFXError(rc, L.hfx_last_error(None).decode())
    return a.value, b.value


def measure_fma_peak():
    """(FP64 TFLOP/s, FP32 TFLOP/s) of the current device from an FMA-chain kernel."""
    a, b = ctypes.c_double(), ctypes.c_double()
    L = load_library()
    rc = L.hfx_measure_fma_peak(ctypes.byref(a), ctypes.byref(b))
    if rc != 0:
        raise HFXError(rc, L.hfx_last_error(None).decode())
    return a.value, b.value


def nao_options(**kw) -> NaoOptions:
    """hfx_nao_default_options, then the given fields (n_gauss, n_restarts, population,
    generations, max_iter, alpha_min, alpha_max, seed)."""
    o = NaoOptions()
    load_library().hfx_nao_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class NAOFit:
    """NAO -> GTO fit (paper Sec. "NAO2GTO scheme", Algorithm 1) of radial functions on the
    grid r_i = i h.  ``phi`` (n_fun x n_r) and ``l`` (n_fun) are uploaded once to torch CUDA
    tensors; every call runs in the CUDA library on ``stream`` (default: the current stream),
    so results are read on that stream or after synchronising it."""

    def __init__(self, phi, l, h, stream=None):
        import torch  # device memory and streams only
        if not torch.cuda.is_available():
            raise RuntimeError("the NAO fit needs a CUDA device; there is no CPU path")
        self.torch = torch
        self.L = load_library()
        self.phi = torch.as_tensor(np.ascontiguousarray(phi, dtype=np.float64)).cuda()
        self.l = torch.as_tensor(np.ascontiguousarray(l, dtype=np.int32)).cuda()
        self.n_fun, self.n_r = self.phi.shape
        self.h = float(h)
        self.stream = stream if stream is not None else torch.cuda.current_stream()

    def _rc(self, rc):
        if rc != 0:
            raise HFXError(rc, self.L.hfx_last_error(None).decode())

    def _z(self, *shape, dtype=None):
        return self.torch.zeros(*shape, dtype=dtype or self.torch.float64, device=self.phi.device)

    def fit(self, opt: NaoOptions):
        """Algorithm 1; returns a dict of torch CUDA tensors: best alpha, D (n_fun x M), err
        (n_fun) and per restart r_alpha, r_D, r_err, r_steps, r_ga_err."""
        M, N = opt.n_gauss, opt.n_restarts
        out = {"alpha": self._z(self.n_fun, M), "D": self._z(self.n_fun, M), "err": self._z(self.n_fun),
               "r_alpha": self._z(self.n_fun * N, M), "r_D": self._z(self.n_fun * N, M),
               "r_err": self._z(self.n_fun * N), "r_steps": self._z(self.n_fun * N, 2, dtype=self.torch.int32),
               "r_ga_err": self._z(self.n_fun * N)}
        self.fit_into(opt, out)
        return out

    def fit_into(self, opt: NaoOptions, out):
        """Algorithm 1 into preallocated tensors (the dict `fit` returns)."""
        p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
        self._rc(self.L.hfx_nao_fit(p(self.phi), p(self.l), self.n_fun, self.n_r, self.h, ctypes.byref(opt),
                                    p(out["alpha"]), p(out["D"]), p(out["err"]), p(out["r_alpha"]), p(out["r_D"]),
                                    p(out["r_err"]), p(out["r_steps"]), p(out["r_ga_err"]),
                                    ctypes.c_void_p(self.stream.cuda_stream)))

    def genetic(self, opt: NaoOptions):
        """The genetic step alone: per restart (alpha, D, err) of its best individual."""
        M, N = opt.n_gauss, opt.n_restarts
        a, d, e = self._z(self.n_fun * N, M), self._z(self.n_fun * N, M), self._z(self.n_fun * N)
        p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
        self._rc(self.L.hfx_nao_genetic(p(self.phi), p(self.l), self.n_fun, self.n_r, self.h, ctypes.byref(opt),
                                        p(a), p(d), p(e), ctypes.c_void_p(self.stream.cuda_stream)))
        return a, d, e

    def local(self, opt: NaoOptions, alpha, D):
        """The local search alone from per-restart starts (n_fun N x M arrays); returns
        (alpha, D, err, steps)."""
        M = opt.n_gauss
        a = self.torch.as_tensor(np.ascontiguousarray(alpha, dtype=np.float64)).reshape(-1, M).cuda().contiguous()
        d = self.torch.as_tensor(np.ascontiguousarray(D, dtype=np.float64)).reshape(-1, M).cuda().contiguous()
        if a.shape[0] != self.n_fun * opt.n_restarts or d.shape != a.shape:
            raise ValueError("local: one start (M exponents, M coefficients) per restart of every function")
        e = self._z(a.shape[0])
        st = self._z(a.shape[0], 2, dtype=self.torch.int32)
        p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
        self._rc(self.L.hfx_nao_local(p(self.phi), p(self.l), self.n_fun, self.n_r, self.h, ctypes.byref(opt),
                                      p(a), p(d), p(e), p(st), ctypes.c_void_p(self.stream.cuda_stream)))
        return a, d, e, st

    def project(self, M: int, fun_of_set, alpha):
        """Least-squares D and err for exponent sets (rows of alpha) of the given functions."""
        fs = self.torch.as_tensor(np.ascontiguousarray(fun_of_set, dtype=np.int32)).cuda()
        a = self.torch.as_tensor(np.ascontiguousarray(alpha, dtype=np.float64)).reshape(-1, M).cuda().contiguous()
        n = a.shape[0]
        d, e = self._z(n, M), self._z(n)
        p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
        self._rc(self.L.hfx_nao_project(p(self.phi), p(self.l), self.n_fun, self.n_r, self.h, M, n, p(fs), p(a),
                                        p(d), p(e), ctypes.c_void_p(self.stream.cuda_stream)))
        return d, e


class HFX:
    """One system: basis on the device, pair list, K builds.

    ``system`` is an ``inputs.System``; ``stream`` a torch.cuda.Stream (or None for the
    current stream).  ``build_K(P)`` takes and returns torch CUDA float64 tensors.
    """

    def __init__(self, system, stream=None, tau=None, rcut=None, omega=None, schedule=HFX_SCHED_DYNAMIC,
                 prim_tau=None, skip_zero_p=True, precision=HFX_FP64, fp32_tau=None, fp32_class_mask=None,
                 fp32_pmax_global=False, density_tau=0.0, dist_tau=0.0):
        import torch  # device memory and streams only
        if not torch.cuda.is_available():
            raise RuntimeError("HFX needs a CUDA device; there is no CPU path")
        self.torch = torch
        L = load_library()
        self.L = L
        self.system = system
        o = default_options()
        o.omega = system.omega if omega is None else omega
        o.schwarz_tau = system.tau if tau is None else tau
        o.rcut_bohr = system.rcut if rcut is None else rcut
        if prim_tau is not None:
            o.prim_tau = prim_tau
        o.schedule = schedule
        o.skip_zero_p = 1 if skip_zero_p else 0
        o.precision = precision
        if fp32_tau is not None:
            o.fp32_tau = fp32_tau
        if fp32_class_mask is not None:
            o.fp32_class_mask = fp32_class_mask
        o.fp32_pmax_global = 1 if fp32_pmax_global else 0
        o.density_tau = float(density_tau)
        o.dist_tau = float(dist_tau)
        self.options = o
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        xyz, sa, sl, sn, al, co = system.basis_arrays()
        self._host = (xyz, sa, sl, sn, al, co)
        h = ctypes.c_void_p()
        rc = L.hfx_init_basis(ctypes.byref(h), int(xyz.shape[0]), _dp(xyz), int(sl.shape[0]), _ip(sa), _ip(sl),
                              _ip(sn), _dp(al), _dp(co), ctypes.byref(o), ctypes.c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise HFXError(rc, L.hfx_last_error(None).decode())
        self.h = h
        self.n_bf = L.hfx_n_basis(h)
        self.pairs_built = False

    def _check(self, rc):
        if rc != 0:
            raise HFXError(rc, self.L.hfx_last_error(self.h).decode())

    def build_pairs(self):
        self._check(self.L.hfx_build_pairs(self.h))
        self.pairs_built = True
        return self

    def set_group_size(self, cls, gs):
        """Lanes per quartet for quartet class cls in later builds (0 = default)."""
        self._check(self.L.hfx_set_group_size(self.h, int(cls), int(gs)))

    def set_streams(self, cls, k):
        """Primitive quartets the warp kernel runs at a time for class cls (0 = default)."""
        self._check(self.L.hfx_set_streams(self.h, int(cls), int(k)))

    def set_timing(self, on=True):
        self._check(self.L.hfx_set_timing(self.h, 1 if on else 0))

    def build_K(self, P, K=None, part=0, n_parts=1):
        """K for the density P (torch float64 CUDA tensor, n x n, contiguous rows); with
        n_parts > 1 only partition `part` of the quartet list (the parts sum to K)."""
        torch = self.torch
        n = self.n_bf
        if not (P.is_cuda and P.dtype == torch.float64 and P.shape == (n, n) and P.stride(1) == 1):
            raise ValueError("P must be a float64 CUDA tensor of shape (n_bf, n_bf) with unit column stride")
        if K is None:
            K = torch.empty((n, n), dtype=torch.float64, device=P.device)
        ld = P.stride(0)
        if K.stride(0) != ld or K.stride(1) != 1:
            raise ValueError("K must have the same row stride as P")
        if n_parts == 1:
            self._check(self.L.hfx_build_K(self.h, ctypes.c_void_p(P.data_ptr()), ctypes.c_void_p(K.data_ptr()), ld))
        else:
            self._check(self.L.hfx_build_K_part(self.h, ctypes.c_void_p(P.data_ptr()),
                                                ctypes.c_void_p(K.data_ptr()), ld, int(part), int(n_parts)))
        return K

    def build_K_host(self, P: np.ndarray) -> np.ndarray:
        P = np.ascontiguousarray(P, dtype=np.float64)
        assert P.shape == (self.n_bf, self.n_bf)
        K = np.empty_like(P)
        self._check(self.L.hfx_build_K_host(self.h, _dp(P), _dp(K)))
        return K

    def energy(self) -> float:
        e = ctypes.c_double()
        self._check(self.L.hfx_energy(self.h, ctypes.byref(e)))
        return e.value

    def energy_device_ptr(self) -> int:
        return int(self.L.hfx_energy_device(self.h))

    def stats(self) -> dict:
        s = Stats()
        self._check(self.L.hfx_get_stats(self.h, ctypes.byref(s)))
        return s.as_dict()

    def pairs(self):
        n = self.stats()["n_pairs_kept"]
        a = np.zeros(max(n, 1), np.int32)
        b = np.zeros(max(n, 1), np.int32)
        q = np.zeros(max(n, 1))
        r = self.L.hfx_get_pairs(self.h, _ip(a), _ip(b), _dp(q), int(max(n, 1)))
        if r < 0:
            raise HFXError(int(r), self.L.hfx_last_error(self.h).decode())
        return a[:r], b[:r], q[:r]

    def device_bytes(self) -> int:
        return int(self.L.hfx_device_bytes(self.h))

    def sm_busy_ns(self, max_n=1024):
        out = np.zeros(max_n)
        r = self.L.hfx_get_cta_busy(self.h, _dp(out), max_n)
        self._check(0 if r >= 0 else r)
        return out[:r]

    def close(self):
        if getattr(self, "h", None):
            self.L.hfx_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Periodic(HFX):
    """Lattice sums of the exchange matrix for a crystal (``inputs.PeriodicSystem``): the home
    cell's basis with its images, list-IJ anchored in the home cell.  ``build_K(P_R, G_list)``
    takes density blocks {R: n_bf x n_bf array} and returns {G: K^G} (torch CUDA float64)."""

    def __init__(self, ps, stream=None, tau=None, rcut=None, omega=None):
        import torch  # device memory and streams only
        if not torch.cuda.is_available():
            raise RuntimeError("Periodic needs a CUDA device; there is no CPU path")
        self.torch = torch
        L = load_library()
        self.L = L
        system = ps.cell
        self.system = system
        o = default_options()
        o.omega = system.omega if omega is None else omega
        o.schwarz_tau = system.tau if tau is None else tau
        o.rcut_bohr = system.rcut if rcut is None else rcut
        self.options = o
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        xyz, sa, sl, sn, al, co = system.basis_arrays()
        lat = np.ascontiguousarray(ps.lattice, dtype=np.float64)
        self._host = (xyz, sa, sl, sn, al, co, lat)
        h = ctypes.c_void_p()
        rc = L.hfx_init_periodic(ctypes.byref(h), int(xyz.shape[0]), _dp(xyz), _dp(lat), int(sl.shape[0]), _ip(sa),
                                 _ip(sl), _ip(sn), _dp(al), _dp(co), ctypes.byref(o),
                                 ctypes.c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise HFXError(rc, L.hfx_last_error(None).decode())
        self.h = h
        self.n_bf = system.n_bf
        self.pairs_built = False

    def cells(self):
        n = self.L.hfx_periodic_cells(self.h, None, 0)
        self._check(0 if n >= 0 else n)
        out = np.zeros(3 * n, dtype=np.int32)
        self.L.hfx_periodic_cells(self.h, _ip(out), n)
        return out.reshape(n, 3)

    def build_K(self, P_R, G_list):
        torch = self.torch
        n = self.n_bf
        Rs = sorted(P_R)
        R_cells = np.ascontiguousarray(np.array(Rs, dtype=np.int32).reshape(-1, 3))
        P = torch.from_numpy(np.stack([np.asarray(P_R[R], dtype=np.float64) for R in Rs])).cuda()
        G = np.ascontiguousarray(np.array([tuple(g) for g in G_list], dtype=np.int32).reshape(-1, 3))
        K = torch.empty((len(G), n, n), dtype=torch.float64, device="cuda")
        with torch.cuda.stream(self.stream):
            self._check(self.L.hfx_build_K_periodic(self.h, len(Rs), _ip(R_cells), ctypes.c_void_p(P.data_ptr()),
                                                    len(G), _ip(G), ctypes.c_void_p(K.data_ptr())))
        self.stream.synchronize()
        return {tuple(int(x) for x in g): K[i] for i, g in enumerate(G)}


def _ptr_array(values):
    arr = (ctypes.c_void_p * len(values))(*[ctypes.c_void_p(int(v)) for v in values])
    return ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), arr


class Batch:
    """Batched K builds over several ``HFX`` contexts (one launch per angular class for all
    systems, captured once as a CUDA graph and replayed)."""

    def __init__(self, contexts, stream=None, graph=True):
        self.L = load_library()
        self.contexts = list(contexts)
        ptrs, self._keep = _ptr_array([c.h.value for c in self.contexts])
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        rc = self.L.hfx_batch_create(ctypes.byref(h), ptrs, len(self.contexts), st)
        if rc != 0:
            raise HFXError(rc, self.L.hfx_last_error(None).decode())
        self.h = h
        if not graph:
            self.L.hfx_batch_set_graph(h, 0)

    def _args(self, Ps, Ks):
        pP, kP = _ptr_array([P.data_ptr() for P in Ps])
        pK, kK = _ptr_array([K.data_ptr() for K in Ks])
        ld = (ctypes.c_int * len(Ps))(*[int(P.stride(0)) for P in Ps])
        return pP, pK, ctypes.cast(ld, ctypes.POINTER(ctypes.c_int)), (kP, kK, ld)

    def _check(self, rc):
        if rc != 0:
            raise HFXError(rc, self.L.hfx_last_error(None).decode())

    def set_branches(self, n):
        """Parallel branches the class launches are spread over (1..4)."""
        self._check(self.L.hfx_batch_set_branches(self.h, int(n)))

    def tune(self, Ps, Ks, target_ms=None):
        if target_ms is not None:
            self._check(self.L.hfx_batch_set_tune_target(self.h, ctypes.c_double(target_ms)))
        pP, pK, ld, keep = self._args(Ps, Ks)
        self._check(self.L.hfx_batch_tune(self.h, pP, pK, ld))

    def run(self, Ps, Ks):
        pP, pK, ld, keep = self._args(Ps, Ks)
        self._keep_run = keep
        self._check(self.L.hfx_batch_run(self.h, pP, pK, ld))

    def stats(self):
        s = BatchStats()
        self._check(self.L.hfx_batch_get_stats(self.h, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        if getattr(self, "h", None):
            self.L.hfx_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request loop with continuous batching over registered ``HFX`` contexts (the C
    server in hfx_batch.cu; this class only marshals arguments)."""

    def __init__(self, hbm_budget_gb=120.0, max_inflight=4, max_batch=16, precision=HFX_FP64,
                 max_step_quartets=None):
        self.L = load_library()
        o = ServerOptions()
        self.L.hfx_server_default_options(ctypes.byref(o))
        o.hbm_budget_gb = float(hbm_budget_gb)
        o.max_inflight = int(max_inflight)
        o.max_batch = int(max_batch)
        o.precision = int(precision)
        if max_step_quartets is not None:
            o.max_step_quartets = float(max_step_quartets)
        h = ctypes.c_void_p()
        rc = self.L.hfx_server_create(ctypes.byref(h), ctypes.byref(o))
        if rc != 0:
            raise HFXError(rc, self.L.hfx_last_error(None).decode())
        self.h = h
        self.contexts = []
        self._keep = {}

    def _check(self, rc):
        if rc < 0:
            raise HFXError(rc, self.L.hfx_server_last_error(self.h).decode())
        return rc

    def add_system(self, ctx) -> int:
        i = ctypes.c_int()
        self._check(self.L.hfx_server_add_system(self.h, ctx.h, ctypes.byref(i)))
        self.contexts.append(ctx)
        return i.value

    def submit(self, system_id, P, K_out, stream=None) -> int:
        """P, K_out: torch float64 tensors (CUDA, or pinned CPU), n x n contiguous.  They
        are kept alive here until the request's result has been read."""
        import torch
        t = ctypes.c_uint64()
        if stream is None and P.is_cuda:
            stream = torch.cuda.current_stream()
        st = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        self._check(self.L.hfx_serve_submit(self.h, int(system_id), ctypes.c_void_p(P.data_ptr()),
                                            ctypes.c_void_p(K_out.data_ptr()), st, ctypes.byref(t)))
        self._keep[t.value] = (P, K_out)
        return t.value

    def poll(self, ticket, release=False) -> dict:
        """State of a request; with release=True a finished request is also forgotten by
        the server (its ticket becomes unknown)."""
        r = Result()
        self._check(self.L.hfx_serve_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(r)))
        if r.status <= 0:
            self._keep.pop(ticket, None)
            if release:
                self.release(ticket)
        return r.as_dict()

    def wait(self, ticket, timeout_ms=-1.0, release=False) -> dict:
        r = Result()
        self._check(self.L.hfx_serve_wait(self.h, ctypes.c_uint64(ticket), ctypes.c_double(timeout_ms),
                                          ctypes.byref(r)))
        self._keep.pop(ticket, None)
        if release:
            self.release(ticket)
        return r.as_dict()

    def release(self, ticket):
        self._check(self.L.hfx_serve_release(self.h, ctypes.c_uint64(ticket)))

    def progress(self) -> int:
        return self._check(self.L.hfx_serve_progress(self.h))

    def drain(self, timeout_ms=-1.0):
        self._check(self.L.hfx_serve_drain(self.h, ctypes.c_double(timeout_ms)))

    def stats(self) -> dict:
        s = ServerStats()
        self._check(self.L.hfx_server_get_stats(self.h, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        if getattr(self, "h", None):
            self.L.hfx_server_free(self.h)
            self.h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
