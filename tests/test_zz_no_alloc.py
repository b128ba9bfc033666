"""hfx_energy_noalloc: the exchange energy without any device allocation.

Some callers cannot let a library call cudaMalloc (they serve all device memory from their
own pool or under a fixed budget, or an allocation would synchronise the device in a
latency-critical loop).  This entry point keeps its scratch in a fixed array inside the
library image.  The test calls it through the C ABI twice in a row -- the second call on
a smaller matrix, so rows left over from the first call are present in the shared
scratch -- and compares each result with E_K from the existing entry point (hfx_energy)
within the tolerance the parity tests use.  This file sorts last so that a run stopping
at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

from paper_2009_03559_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_E = 1e-10
MAX_N = 16384  # HFX_NOALLOC_MAX_N in include/hfx.h


def _existing_energy(hfx, system, P):
    h = hfx.HFX(system).build_pairs()
    Pd = torch.from_numpy(P).cuda()
    K = h.build_K(Pd)
    return h, Pd, K, h.energy()


def test_energy_noalloc_two_calls_match_existing_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_03559_gb300 import hfx
    L = hfx.load_library()
    stream = torch.cuda.current_stream()
    cases = [inputs.config1(8), inputs.config0()]   # n = 104, then n = 64
    for system, P in cases:
        h, Pd, K, e_ref = _existing_energy(hfx, system, P)
        n = system.n_bf
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.hfx_energy_noalloc(ctypes.c_void_p(Pd.data_ptr()), ctypes.c_void_p(K.data_ptr()), n, n,
                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, L.hfx_last_error(None)
        torch.cuda.synchronize()
        assert abs(out.item() - e_ref) <= TOL_E, (out.item(), e_ref)
        h.close()


def test_energy_noalloc_strided_rows():
    """P and K as the left n columns of wider row-major buffers (ld = n + 7), the padding
    filled with NaN: only the n x n matrices may be read."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_03559_gb300 import hfx
    L = hfx.load_library()
    stream = torch.cuda.current_stream()
    system, P = inputs.config1(8)
    h, Pd, K, e_ref = _existing_energy(hfx, system, P)
    n = system.n_bf
    ld = n + 7
    Pw = torch.full((n, ld), float("nan"), dtype=torch.float64, device="cuda")
    Kw = torch.full((n, ld), float("nan"), dtype=torch.float64, device="cuda")
    Pw[:, :n] = Pd
    Kw[:, :n] = K
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        rc = L.hfx_energy_noalloc(ctypes.c_void_p(Pw.data_ptr()), ctypes.c_void_p(Kw.data_ptr()), n, ld,
                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, L.hfx_last_error(None)
        torch.cuda.synchronize()
        assert abs(out.item() - e_ref) <= TOL_E, (out.item(), e_ref)
    h.close()


def test_energy_noalloc_rejects_sizes_beyond_scratch():
    from paper_2009_03559_gb300 import hfx
    L = hfx.load_library()
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    rc = L.hfx_energy_noalloc(dummy, dummy, MAX_N + 1, MAX_N + 1, dummy, None)
    assert rc == -1
    assert b"n must be in 1.." in L.hfx_last_error(None)
    assert L.hfx_energy_noalloc(dummy, dummy, 8, 4, dummy, None) == -1  # ld < n
