"""The C-ABI library builds, loads and exports every function declared in include/hfx.h;
host-side argument checks answer without a GPU.  No compute calls are made here."""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hfx.h")


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2009_03559_gb300 import build, hfx
    build.build()
    return hfx.load_library()


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hfx_[A-Za-z0-9_]+)\s*\(", txt)))


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("hfx_init_basis", "hfx_build_pairs", "hfx_build_K", "hfx_build_K_host", "hfx_free",
                     "hfx_last_error", "hfx_n_basis", "hfx_get_stats"):
        assert required in names


def test_every_declared_symbol_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_bad_l_rejected_on_host(lib):
    from paper_2009_03559_gb300 import hfx, inputs
    s = inputs.cluster_system(2, seed=1)
    xyz, sa, sl, sn, al, co = s.basis_arrays()
    sl = sl.copy()
    sl[0] = 3
    h = ctypes.c_void_p()
    rc = lib.hfx_init_basis(ctypes.byref(h), 2, hfx._dp(xyz), int(sl.shape[0]), hfx._ip(sa), hfx._ip(sl),
                            hfx._ip(sn), hfx._dp(al), hfx._dp(co), None, None)
    assert rc == -2
    assert b"angular momentum" in lib.hfx_last_error(None)
    assert not h.value


def test_null_and_empty_rejected(lib):
    h = ctypes.c_void_p()
    assert lib.hfx_init_basis(None, 1, None, 1, None, None, None, None, None, None, None) == -1
    assert lib.hfx_init_basis(ctypes.byref(h), 0, None, 0, None, None, None, None, None, None, None) == -1
    assert lib.hfx_build_pairs(None) == -1
    assert lib.hfx_build_K(None, None, None, 0) == -1
    assert lib.hfx_n_basis(None) == -1


def test_bad_exponent_rejected(lib):
    from paper_2009_03559_gb300 import hfx, inputs
    s = inputs.cluster_system(2, seed=1)
    xyz, sa, sl, sn, al, co = s.basis_arrays()
    al = al.copy()
    al[2] = -1.0
    h = ctypes.c_void_p()
    rc = lib.hfx_init_basis(ctypes.byref(h), 2, hfx._dp(xyz), int(sl.shape[0]), hfx._ip(sa), hfx._ip(sl),
                            hfx._ip(sn), hfx._dp(al), hfx._dp(co), None, None)
    assert rc == -1


def test_tables_regenerate_identically():
    """The committed recurrence tables are exactly what the generator writes."""
    import subprocess
    import sys
    gen = os.path.join(ROOT, "paper_2009_03559_gb300", "csrc", "gen_eri_tables.py")
    inc = os.path.join(ROOT, "paper_2009_03559_gb300", "csrc", "eri_tables.inc")
    out = subprocess.run([sys.executable, gen], check=True, capture_output=True, text=True).stdout
    assert out == open(inc).read()


def test_server_options_and_null_arguments_rejected_on_host(lib):
    """Server entry points check their arguments before any CUDA call."""
    import ctypes
    from paper_2009_03559_gb300 import hfx
    L = hfx.load_library()
    o = hfx.ServerOptions()
    L.hfx_server_default_options(ctypes.byref(o))
    assert (o.hbm_budget_gb, o.max_step_quartets, o.max_inflight, o.max_batch, o.precision) == (120.0, 1e7, 4, 16, 0)
    h = ctypes.c_void_p()
    for field, bad in (("hbm_budget_gb", 0.0), ("max_step_quartets", -1.0), ("max_inflight", 0), ("max_batch", 0),
                       ("precision", 7)):
        b = hfx.ServerOptions()
        L.hfx_server_default_options(ctypes.byref(b))
        setattr(b, field, bad)
        assert L.hfx_server_create(ctypes.byref(h), ctypes.byref(b)) == -1
    t = ctypes.c_uint64()
    r = hfx.Result()
    assert L.hfx_serve_submit(None, 0, None, None, None, ctypes.byref(t)) == -1
    assert L.hfx_serve_poll(None, 1, ctypes.byref(r)) == -1
    assert L.hfx_serve_wait(None, 1, ctypes.c_double(0.0), ctypes.byref(r)) == -1
    assert L.hfx_serve_drain(None, ctypes.c_double(0.0)) == -1
    assert L.hfx_server_add_system(None, None, None) == -1
    assert L.hfx_serve_release(None, 1) == -1


def test_bench_oracle_sample_is_canonical_and_kept():
    """The CPU-baseline sampler draws kept canonical quartets (I>=J, K>=L, pair IJ at or
    after pair KL in the kept list, Q_IJ Q_KL >= tau)."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_2009_03559_gb300 import inputs
    s, P = inputs.config1(8)
    S = oracle.Screen(oracle.Basis(s))
    smp = bench.oracle_sample(S, s, 3000)
    Q, cut, kept, qmax = S.export()
    assert smp.shape == (3000, 4)
    I, J, K, L = smp.T
    assert np.all(I >= J) and np.all(K >= L)
    assert np.all(kept[I, J]) and np.all(kept[K, L])
    assert np.all(Q[I, J] * Q[K, L] >= S.tau)


def test_header_compiles_as_c_and_host_calls_work(lib, tmp_path):
    """include/hfx.h is plain C: a C99 program using it compiles with warnings as errors,
    links against the library and its host-side calls answer without a GPU."""
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2009_03559_gb300 import hfx
    libdir = os.path.dirname(hfx.LIB_PATH)
    exe = str(tmp_path / "abi_from_c")
    src = os.path.join(ROOT, "tests", "c", "abi_from_c.c")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), src,
                        "-o", exe, "-L", libdir, "-lhfx", f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert "C ABI ok" in r.stdout


def test_nao_arguments_checked_on_host(lib):
    """The NAO-fit entry points reject bad sizes and options before any CUDA call."""
    from paper_2009_03559_gb300 import hfx
    o = hfx.nao_options()
    assert (o.n_gauss, o.n_restarts, o.population, o.generations, o.max_iter) == (3, 512, 32, 30, 100)
    assert o.alpha_min == 0.1 and o.alpha_max == 1000.0
    dummy = ctypes.c_void_p(16)  # never dereferenced: the checks fail first
    args = lambda: (dummy, dummy, 4, 512, 0.01, ctypes.byref(o), dummy, dummy, dummy, dummy, dummy, dummy,  # noqa
                    None, None, None)
    for field, bad in (("n_gauss", 0), ("n_gauss", 7), ("population", 1), ("population", 65),
                       ("n_restarts", 0), ("generations", -1), ("max_iter", -1), ("alpha_min", 0.0),
                       ("alpha_max", 0.05)):
        o = hfx.nao_options(**{field: bad})
        assert lib.hfx_nao_fit(*args()) == -1, field
    o = hfx.nao_options()
    assert lib.hfx_nao_fit(dummy, dummy, 4, 1025, 0.01, ctypes.byref(o), dummy, dummy, dummy, dummy, dummy, dummy,
                           None, None, None) == -1
    assert lib.hfx_nao_fit(dummy, dummy, 4, 512, 0.0, ctypes.byref(o), dummy, dummy, dummy, dummy, dummy, dummy,
                           None, None, None) == -1
    assert lib.hfx_nao_fit(None, dummy, 4, 512, 0.01, ctypes.byref(o), dummy, dummy, dummy, dummy, dummy, dummy,
                           None, None, None) == -1
    assert b"nao" in lib.hfx_last_error(None)
    assert lib.hfx_nao_project(dummy, dummy, 4, 512, 0.01, 3, 5, None, dummy, dummy, dummy, None) == -1
