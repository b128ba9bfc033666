"""Build the CUDA library libhfx.so for sm_103a, in-tree (paper_2009_03559_gb300/_build).

Steps: regenerate the recurrence tables if their generator changed, compile each
translation unit with nvcc in parallel, link a shared library.  No CMake.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libhfx.so")
INCLUDE = os.path.join(ROOT, "include")
SOURCES = ["hfx_api.cu", "hfx_eri.cu", "hfx_setup.cu", "hfx_batch.cu", "hfx_noalloc.cu", "hfx_nao.cu"]
HEADERS = ["hfx_internal.cuh", "eri_engine.cuh", "eri_tables.inc", "hfx_eri.h", "hfx_setup.h", "hfx_ctx.h"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _tables_current() -> bool:
    gen = os.path.join(CSRC, "gen_eri_tables.py")
    inc = os.path.join(CSRC, "eri_tables.inc")
    return os.path.exists(inc) and os.path.getmtime(inc) >= os.path.getmtime(gen)


def generate_tables() -> None:
    gen = os.path.join(CSRC, "gen_eri_tables.py")
    inc = os.path.join(CSRC, "eri_tables.inc")
    out = subprocess.run([sys.executable, gen], check=True, capture_output=True, text=True).stdout
    tmp = inc + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        f.write(out)
    os.replace(tmp, inc)


def _newest(paths) -> float:
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False,
          extra_flags=(), out_dir: str = BUILD) -> str:
    """Compile into out_dir/libhfx.so; extra_flags (e.g. -D tuning macros) go to nvcc."""
    lib_path = os.path.join(out_dir, "libhfx.so")
    os.makedirs(out_dir, exist_ok=True)
    if not _tables_current():
        generate_tables()
    deps = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "hfx.h"), __file__]
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= _newest(deps + srcs):
        return lib_path
    nv = nvcc()
    flags = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
             "--expt-relaxed-constexpr"]
    if ptxas_verbose:
        flags += ["-Xptxas", "-v"]
    flags += list(extra_flags)

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src).replace(".cu", ".o"))
        cmd = [nv] + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose or ptxas_verbose:
        for obj, err in results:
            if err:
                print(err, file=sys.stderr)
    objs = [o for o, _ in results]
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [nv, ARCH, "-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_verbose="--ptxas" in sys.argv))
