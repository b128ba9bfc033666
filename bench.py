#!/usr/bin/env python3
"""Benchmark of the screened HSE exchange build (one JSON line on rank 0).

Step = one K build (P on the device -> K and E_K ready) of the 64-atom DZP-like diamond
workload (832 functions, orbital cutoff 6 bohr, Schwarz tau 1e-8, P truncated beyond
10 bohr), plain FP64, through the C ABI.  value = screened quartets per second (whole
job).  L2 is flushed (256 MiB write) between timed steps; each step is timed with CUDA
events on the library's stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

N > 1 (torchrun): independent replicas of the same workload, one per GPU ("scaling":
"weak"); the K build has no exchange step between GPUs.  --impl reference times the
CPU oracle (the only other implementation: there is no reference code) on the host
cores for a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "HFX K-build ms & screened ERI quartets/s vs plain FP64; p50/p99 latency"
def workload_desc(s, mixed=False, fp32_classes="all"):
    prec = ("mixed precision (FP32 recurrences where Q*Q*max|P| < 1e-6, "
            f"{'all classes' if fp32_classes == 'all' else 's,p classes only'}; FP64 Boys and K)"
            if mixed else "plain FP64")
    return (f"diamond-{s.n_atoms} DZP-like: {s.n_atoms} atoms (a=10.26 bohr cells), {s.n_shells} shells "
            f"s,s,p,p,d, {s.n_bf} spherical functions, 3 primitives/shell, omega=0.11, r_c=6 bohr, "
            f"tau=1e-8, P truncated beyond 10 bohr; {prec}")


WORKLOAD = ("diamond-64 DZP-like: 64 atoms (2x2x2 cells, a=10.26 bohr), 320 shells s,s,p,p,d, "
            "832 spherical functions, 3 primitives/shell, omega=0.11, r_c=6 bohr, tau=1e-8, "
            "P truncated beyond 10 bohr; plain FP64")


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def reference_arm(args, ws, rank):
    """CPU oracle on the host cores, a bounded sample of the same workload per step."""
    if rank != 0:
        return
    import oracle
    from paper_2009_03559_gb300 import inputs
    s, P = inputs.config1(64)
    B = oracle.Basis(s)
    S = oracle.Screen(B)
    sample = oracle_sample(S, s, n=args.ref_sample)
    cores = oracle.max_threads()
    for _ in range(args.warmup):
        S.eval_quartets(sample)
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        S.eval_quartets(sample)
        t.append(time.perf_counter() - t0)
    qps = len(sample) * args.steps / sum(t)
    desc = (f"{len(sample)} canonical kept quartets drawn uniformly (seeded) from the workload, "
            f"integrals only (no digest), per step")
    line = {
        "metric": METRIC, "value": qps, "unit": "quartets/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(t) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "sample": desc},
        "cpu_baseline": {"value": qps, "unit": "quartets/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": qps, "unit": "quartets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def oracle_sample(S, s, n, seed=777):
    """Seeded uniform sample of kept canonical quartets (I>=J, K>=L, IJ>=KL)."""
    Q, cut, kept, qmax = S.export()
    ns = s.n_shells
    pairs = [(I, J) for I in range(ns) for J in range(I + 1) if kept[I, J]]
    q = np.array([Q[I, J] for I, J in pairs])
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        a, b = rng.integers(0, len(pairs), 2)
        if b > a:
            a, b = b, a
        if q[a] * q[b] >= S.tau:
            out.append(pairs[a] + pairs[b])
    return np.array(out, dtype=np.int32)


def cpu_baseline(args):
    import oracle
    from paper_2009_03559_gb300 import inputs
    s, P = inputs.config1(64)
    S = oracle.Screen(oracle.Basis(s))
    sample = oracle_sample(S, s, n=args.ref_sample)
    S.eval_quartets(sample[:2000])
    t0 = time.perf_counter()
    S.eval_quartets(sample)
    dt = time.perf_counter() - t0
    return {"value": len(sample) / dt, "unit": "quartets/s", "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{len(sample)} canonical kept quartets of the workload drawn uniformly (seeded), "
                      f"integrals only, {dt:.1f} s"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--ref-sample", type=int, default=60000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--atoms", type=int, default=64,
                    help="diamond piece size (64 = the benchmark workload; smaller for profiler captures)")
    ap.add_argument("--report", action="store_true", help="per-class table on stderr")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--fp32-classes", default="sp", choices=["all", "sp"])
    ap.add_argument("--fp32-tau", type=float, default=1e-6)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_info()

    if args.impl == "reference":
        reference_arm(args, ws, rank)
        return

    import torch
    pg = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
        pg = dist
    else:
        torch.cuda.set_device(0)
    from paper_2009_03559_gb300 import hfx, inputs

    s, P_np = inputs.config1(args.atoms)
    stream = torch.cuda.Stream()
    mixed = args.precision == "mixed"
    h = hfx.HFX(s, stream=stream, precision=hfx.HFX_MIXED if mixed else hfx.HFX_FP64,
                fp32_class_mask=((1 << 21) - 1) if args.fp32_classes == "all" else hfx.SP_CLASS_MASK,
                fp32_tau=args.fp32_tau)
    h.build_pairs()
    P = torch.from_numpy(P_np).cuda()
    K = torch.empty_like(P)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    n_q = h.stats()["n_quartets"]
    fp64_peak, fp32_peak = hfx.measure_fma_peak()

    # untimed warm-up (last one with per-class timing and counters for the roofline)
    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            h.set_timing(i == args.warmup - 1)
            h.build_K(P, K)
        st_timed = h.stats()
        h.set_timing(False)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            h.build_K(P, K)
            ev[i][1].record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ck = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if pg:
        t = torch.tensor([total_ms], device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        total_ms = float(t.item())
    energy = h.energy()

    # end-to-end through the host-buffer entry point (copies inside the timed region)
    e2e_t = []
    for i in range(args.e2e_steps):
        t0 = time.perf_counter()
        Kh = h.build_K_host(P_np)
        e2e_t.append(time.perf_counter() - t0)
    nbytes = 8 * s.n_bf * s.n_bf

    # roofline of the dominant kernel: the warp-cooperative FP64 kernel (classes with G=32)
    from paper_2009_03559_gb300.hfx import QUARTET_CLASSES
    ms_cls = st_timed["ms_class"]
    g32 = [c for c in range(21) if st_timed["group_size_class"][c] == 32 or mixed]
    flops_cls = st_timed["flops_class"]
    dom_ms = sum(ms_cls[c] for c in g32)
    dom_fl = sum(flops_cls[c] for c in g32)
    achieved = dom_fl / (dom_ms * 1e-3) / 1e12 if dom_ms > 0 else None
    launches_per_step = sum(1 for c in range(21) if st_timed["n_quartets_class"][c] > 0) + 3

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": n_q * args.steps * ws / (total_ms * 1e-3),
            "unit": "quartets/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps,
            "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if not mixed else "f64+f32",
            "data": "synthetic",
            "config": {"workload": workload_desc(s, mixed, args.fp32_classes), "n_bf": s.n_bf, "quartets_per_step": n_q,
                       "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas x{ws}",
                       "energy_E_K": energy},
            "e2e": {"value": n_q / float(np.median(e2e_t)) if e2e_t else None, "unit": "quartets/s",
                    "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
            "gpu_launches": launches_per_step * args.steps,
            "roofline": {"bound": "alu", "kernel": "eri_g32_kernel (FP64 classes with warp groups)",
                         "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": (achieved / fp64_peak) if achieved else None, "traffic": None,
                         "peak_source": "FP64 FMA-chain probe of this run (hfx_measure_fma_peak)"},
            "clocks": {"sm_mhz": ck["sm_mhz"], "sm_max_mhz": ck["sm_max_mhz"], "reasons": ck["reasons"]},
            "fp64_flops_per_step": st_timed["flops_fp64"],
            "fp32_flops_per_step": st_timed["flops_fp32"],
            "quartets_evaluated_per_step": sum(st_timed["quartets_evaluated_class"]),
            "quartets_fp32_per_step": sum(st_timed["quartets_fp32_class"]),
            "fp64_tflops_step": st_timed["flops_fp64"] / (total_ms / args.steps * 1e-3) / 1e12,
            "fp32_peak_tflops": fp32_peak,
            "class_ms": {QUARTET_CLASSES[c]: round(ms_cls[c], 3) for c in range(21)},
        }
        if args.report:
            print(f"{'class':9s} {'G':>2s} {'quartets':>11s} {'prims':>12s} {'ms':>9s} {'TF/s':>6s} {'frac':>5s}",
                  file=sys.stderr)
            for c in range(21):
                ms = ms_cls[c]
                fl = flops_cls[c]
                tf = fl / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
                print(f"{QUARTET_CLASSES[c]:9s} {st_timed['group_size_class'][c]:2d} "
                      f"{st_timed['n_quartets_class'][c]:11d} {st_timed['prim_quartets_class'][c]:12d} "
                      f"{ms:9.2f} {tf:6.3f} {tf / fp64_peak:5.2f}", file=sys.stderr)
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
