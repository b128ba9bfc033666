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

Other workloads (one JSON line each, rank 0, one GPU; reports beside the main line):
  --workload batch32     32 systems (8..128 atoms, cluster or diamond) in one batched,
                         autotuned build replayed from a CUDA graph, vs the same systems
                         built one by one (plain FP64)
  --workload diamond216  216-atom diamond (2808 functions): plain FP64 vs mixed precision
  --workload balance     the 64-atom build under the three work distributions (static bra-pair
                         split, Algorithm 2; static quartet split, Algorithm 3; dynamic
                         chunks): build time and the spread of busy time over the SMs
  --workload serve       request stream (Poisson arrivals, systems from a seeded pool)
                         through the continuous-batching server (mixed precision) vs the
                         same stream built one request at a time (plain FP64, FIFO)
  --workload nao2gto     the NAO -> GTO fit (Algorithm 1) of 20 synthetic confined radial
                         functions (4 DZP-like element sets), 3 Gaussians each, 512 restarts
                         per function (population 32, 30 generations, 100 local steps)
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
MASK_DESC = {"default": "every class but (dd|dd)", "sp": "s,p classes only", "all": "all classes"}


def class_mask(hfx, name):
    return {"default": hfx.FP32_CLASSES_DEFAULT, "sp": hfx.SP_CLASS_MASK, "all": hfx.ALL_CLASS_MASK}[name]


def workload_desc(s, mixed=False, fp32_classes="default"):
    prec = ("mixed precision (FP32 recurrences where Q*Q*max|P| < 1e-6, "
            f"{MASK_DESC[fp32_classes]}; FP32 Boys step where the incomplete-gamma difference is safe, else "
            f"FP64; FP64 HRR, spherical step and K)" if mixed else "plain FP64")
    return (f"diamond-{s.n_atoms} DZP-like: {s.n_atoms} atoms (a=10.26 bohr cells), {s.n_shells} shells "
            f"s,s,p,p,d, {s.n_bf} spherical functions, 3 primitives/shell, omega=0.11, r_c=6 bohr, "
            f"tau=1e-8, P truncated beyond 10 bohr; {prec}")


WORKLOAD = ("diamond-64 DZP-like: 64 atoms (2x2x2 cells, a=10.26 bohr), 320 shells s,s,p,p,d, "
            "832 spherical functions, 3 primitives/shell, omega=0.11, r_c=6 bohr, tau=1e-8, "
            "P truncated beyond 10 bohr; plain FP64")


def max_over_ranks(value, pg):
    """Maximum of a host float over the ranks of the default process group (CUDA tensor
    for NCCL, CPU tensor for gloo)."""
    import torch
    dev = "cuda" if pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


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
    """Seeded uniform sample of kept canonical quartets (I>=J, K>=L, IJ>=KL): pairs of
    kept shell pairs drawn uniformly, kept if their Schwarz product passes tau."""
    Q, cut, kept, qmax = S.export()
    I, J = np.nonzero(np.tril(kept))
    q = Q[I, J]
    rng = np.random.default_rng(seed)
    out = []
    got = 0
    while got < n:
        a = rng.integers(0, len(I), 4 * n)
        b = rng.integers(0, len(I), 4 * n)
        hi, lo = np.maximum(a, b), np.minimum(a, b)
        ok = q[hi] * q[lo] >= S.tau
        hi, lo = hi[ok], lo[ok]
        out.append(np.stack([I[hi], J[hi], I[lo], J[lo]], axis=1))
        got += len(hi)
    return np.ascontiguousarray(np.concatenate(out)[:n], dtype=np.int32)


def cpu_baseline(args):
    import oracle
    from paper_2009_03559_gb300 import inputs
    s, P = inputs.config1(64)
    S = oracle.Screen(oracle.Basis(s))
    sample = oracle_sample(S, s, n=args.cpu_sample)
    cores = oracle.max_threads()
    S.eval_quartets(sample[:2000])
    t0 = time.perf_counter()
    S.eval_quartets(sample)
    dt = time.perf_counter() - t0
    # the same oracle on one thread, on the first 1/cores of the sample (last: the oracle
    # keeps the thread count it was last given)
    one = sample[: max(2000, len(sample) // max(cores, 1))]
    t0 = time.perf_counter()
    S.eval_quartets(one, nthreads=1)
    dt1 = time.perf_counter() - t0
    return {"value": len(sample) / dt, "unit": "quartets/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(sample)} canonical kept quartets of the workload drawn uniformly (seeded), "
                      f"integrals only, {dt:.1f} s",
            "single_thread_value": len(one) / dt1}


def _evt(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_batch32(args, torch, hfx, inputs):
    """32 independent systems: one batched, autotuned build replayed from a CUDA graph vs
    the same systems built one by one through the single-system entry point."""
    systems = inputs.config2_systems()
    ctxs = [hfx.HFX(s).build_pairs() for s, P in systems]
    Ps = [torch.from_numpy(P).cuda() for s, P in systems]
    Ks = [torch.empty_like(P) for P in Ps]
    Ks1 = [torch.empty_like(P) for P in Ps]
    nq = sum(c.stats()["n_quartets"] for c in ctxs)
    torch.cuda.synchronize()
    a, b = _evt(torch)
    # one by one (plain single-system path), one pass after a small warm-up
    ctxs[11].build_K(Ps[11], Ks1[11])
    a.record()
    for c, P, K in zip(ctxs, Ps, Ks1):
        c.build_K(P, K)
    b.record()
    torch.cuda.synchronize()
    seq_ms = a.elapsed_time(b)
    e_seq = [c.energy() for c in ctxs]
    bt = hfx.Batch(ctxs)
    clocks = ClockSampler(0)
    clocks.start()
    a.record()
    bt.run(Ps, Ks)  # default per-class choices; graph capture and instantiation + first launch
    b.record()
    torch.cuda.synchronize()
    def_ms = a.elapsed_time(b)
    t0 = time.perf_counter()
    bt.tune(Ps, Ks)
    tune_s = time.perf_counter() - t0
    a.record()
    bt.run(Ps, Ks)  # tuned choices: new graph
    b.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    tuned_ms = a.elapsed_time(b)
    # the tuner keeps its choices only if they ran the whole batch faster than the defaults in
    # its own timed runs; the line reports the replay after tuning (whichever it kept)
    bat_ms = tuned_ms
    e_bat = [c.energy() for c in ctxs]
    dk = max(torch.abs(x - y).max().item() for x, y in zip(Ks, Ks1))
    st = bt.stats()
    print(json.dumps({
        "metric": METRIC, "workload": "batch32", "value": nq / (bat_ms * 1e-3), "unit": "quartets/s",
        "ms_per_step": bat_ms, "n_gpus": 1, "steps": 1, "warmup": 1, "higher_is_better": True,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "32 systems, atoms uniform in 8..128, cluster (s,p; tau 1e-10, no cutoff) or "
                               "diamond (s,s,p,p,d; tau 1e-8, r_c 6 bohr, P truncated beyond 10 bohr) by a "
                               "seeded coin; plain FP64",
                   "quartets": nq, "systems": [[s.kind, s.n_atoms, s.n_bf] for s, P in systems]},
        "one_by_one": {"ms": seq_ms, "quartets_per_s": nq / (seq_ms * 1e-3)},
        "batched_default_ms": def_ms, "batched_tuned_ms": tuned_ms,
        "speedup_vs_one_by_one": seq_ms / bat_ms,
        "tuner": {"seconds": tune_s, "group_size_class": st["group_size_class"], "chunk_class": st["chunk_class"],
                  "streams_class": st["streams_class"], "window_class": st["tune_window_class"],
                  "kept_tuned_choices": bool(st["tune_kept"]),
                  "whole_batch_default_ms": st["tune_full_default_ms"],
                  "whole_batch_tuned_ms": st["tune_full_tuned_ms"]},
        "max_abs_dK_batched_vs_single": dk,
        "max_abs_dE_batched_vs_single": max(abs(x - y) for x, y in zip(e_seq, e_bat)),
        "clocks": {"sm_mhz": ck["sm_mhz"], "sm_max_mhz": ck["sm_max_mhz"], "reasons": ck["reasons"]},
    }), flush=True)


def nao_flops(M, n_r, evals, jpasses, trials):
    """FP64 flops (FMA = 2) per grid point as the NAO kernels are written, times the passes:
    genetic fitness = Gaussians by recurrence (2M per pass, two passes), normal equations
    (M(M+1) + 2M) and residual (2M + 3); Jacobian pass 4M + 3 + 6 M(M+1)/2 + 4M; trial pass
    4M + 3.  exp() calls (3M per lane and pass) are not counted."""
    na = M * (M + 1) // 2
    fit = 2 * M + 2 * na + 2 * M + 2 * M + 2 * M + 3
    jac = 4 * M + 3 + 6 * na + 4 * M
    trial = 4 * M + 3
    return n_r * (evals * fit + jpasses * jac + trials * trial)


def run_nao(args, torch, hfx, inputs):
    """NAO -> GTO fit (paper Sec. "NAO2GTO scheme", Algorithm 1) of a DZP-like radial set."""
    rs = inputs.nao_set(4)
    o = hfx.nao_options()
    n_fun, n_r = rs.phi.shape
    M, N, P, G = o.n_gauss, o.n_restarts, o.population, o.generations
    stream = torch.cuda.Stream()
    F = hfx.NAOFit(rs.phi, rs.l, rs.h, stream=stream)
    out = F.fit(o)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            F.fit_into(o, out)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    evs = [_evt(torch) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(float(i))
            evs[i][0].record(stream)
            F.fit_into(o, out)
            evs[i][1].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in evs]
    # the genetic kernel alone (the dominant launch), timed the same way
    ga_evs = [_evt(torch) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(float(i))
            ga_evs[i][0].record(stream)
            F.genetic(o)
            ga_evs[i][1].record(stream)
    torch.cuda.synchronize()
    ga_ms = float(np.mean([a.elapsed_time(b) for a, b in ga_evs]))
    st = out["r_steps"].cpu().numpy()
    n_rs = n_fun * N
    evals = n_rs * (P + G * (P - 1) + 1)
    fl_ga = nao_flops(M, n_r, evals, 0, 0)
    fl_all = nao_flops(M, n_r, evals, int(st[:, 1].sum()), int(st[:, 0].sum()))
    fp64_peak, _ = hfx.measure_fma_peak()
    mean_ms = float(np.mean(ms))
    # e2e: host radial functions in, best fits out, through the public binding each step
    e2e_ms = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):  # the copies back are ordered after the fit
            Fh = hfx.NAOFit(rs.phi, rs.l, rs.h, stream=stream)
            res = Fh.fit(o)
            best = (res["alpha"].cpu(), res["D"].cpu(), res["err"].cpu())
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    h2d = rs.phi.nbytes + rs.l.astype(np.int32).nbytes
    d2h = sum(t.numel() * t.element_size() for t in best)
    # CPU oracle on a bounded sample of the same restarts
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import nao2gto as ON
        rng = np.random.default_rng(5)
        picks = [(int(f), int(it)) for f, it in zip(rng.integers(0, n_fun, 96), rng.integers(0, N, 96))]
        t0 = time.perf_counter()
        dev = []
        for f, it in picks:
            ref = ON.fit(rs.phi[f], int(rs.l[f]), rs.h, M=M, N=N, P=P, G=G, max_iter=o.max_iter,
                         alpha_min=o.alpha_min, alpha_max=o.alpha_max, seed=o.seed, fun=f, restarts=[it])
            q = f * N + it
            e_gpu = float(out["r_err"][q].item())
            dev.append(abs(e_gpu - ref["restarts"][0]["err"]) / ref["restarts"][0]["err"])
        dt = time.perf_counter() - t0
        cpu = {"value": len(picks) / dt, "unit": "restarts/s", "cores": 1, "kind": "oracle",
               "sample": f"{len(picks)} restarts of the workload drawn uniformly (seeded), {dt:.1f} s",
               "max_rel_err_diff_gpu_vs_oracle": max(dev)}
    err = out["err"].cpu().numpy()
    y2 = [float(((rs.phi[f] / (rs.h * np.arange(1, n_r + 1)) ** rs.l[f]) ** 2).sum()) for f in range(n_fun)]
    print(json.dumps({
        "metric": "NAO->GTO fit: Algorithm 1 restarts/s", "workload": "nao2gto",
        "value": n_rs / (mean_ms * 1e-3), "unit": "restarts/s", "ms_per_step": mean_ms,
        "p50_ms": float(np.median(ms)), "p99_ms": float(np.percentile(ms, 99)),
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{n_fun} confined Slater-type radial functions (4 elements x 2s 2p 1d), "
                               f"n_r {n_r} on (0, {rs.r_cut:g}] bohr; M {M}, N {N}, P {P}, G {G}, "
                               f"max_iter {o.max_iter}, alpha >= {o.alpha_min:g}",
                   "l2": "flushed between timed steps (256 MiB write)"},
        "e2e": {"value": n_rs / (float(np.median(e2e_ms)) * 1e-3), "unit": "restarts/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": 3 * args.steps,
        "roofline": {"bound": "alu", "kernel": "nao_genetic_kernel, CUDA events around each launch",
                     "achieved": fl_ga / (ga_ms * 1e-3) / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": fl_ga / (ga_ms * 1e-3) / 1e12 / fp64_peak, "traffic": None,
                     "flops": "per grid point as written (FMA = 2): Gaussian recurrence, normal equations, "
                              "residual; exp() calls apart", "peak_source": "FP64 FMA-chain probe of this run"},
        "genetic_ms": ga_ms, "whole_fit_tflops": fl_all / (mean_ms * 1e-3) / 1e12,
        "fit_rel_err": {"min": float(min(e / y for e, y in zip(err, y2))),
                        "max": float(max(e / y for e, y in zip(err, y2)))},
        "local_steps_mean": float(st[:, 0].mean()),
        "cpu_baseline": cpu,
        "clocks": {"sm_mhz": ck["sm_mhz"], "sm_max_mhz": ck["sm_max_mhz"], "reasons": ck["reasons"]},
    }), flush=True)


def run_diamond216(args, torch, hfx, inputs):
    """216-atom diamond: plain FP64 build vs mixed precision (FP32 recurrences for quartets
    with Q_IJ Q_KL max|P blocks| < fp32_tau)."""
    s, P_np = inputs.config3()
    P = torch.from_numpy(P_np).cuda()
    out = {}
    Ks = {}
    for name, prec, mask in (("fp64", hfx.HFX_FP64, None), ("mixed", hfx.HFX_MIXED, hfx.FP32_CLASSES_DEFAULT),
                             ("mixed_all", hfx.HFX_MIXED, hfx.ALL_CLASS_MASK)):
        h = hfx.HFX(s, precision=prec, fp32_class_mask=mask, fp32_tau=args.fp32_tau).build_pairs()
        h.set_timing(True)
        K = torch.empty_like(P)
        h.build_K(P, K)  # warm-up
        torch.cuda.synchronize()
        a, b = _evt(torch)
        a.record()
        h.build_K(P, K)
        b.record()
        torch.cuda.synchronize()
        st = h.stats()
        ms = a.elapsed_time(b)
        out[name] = {"ms": ms, "quartets_per_s": st["n_quartets"] / (ms * 1e-3), "energy": h.energy(),
                     "quartets_evaluated": sum(st["quartets_evaluated_class"]),
                     "quartets_fp32": sum(st["quartets_fp32_class"]),
                     "fp64_flops": st["flops_fp64"], "fp32_flops": st["flops_fp32"]}
        Ks[name] = K
        n_q = st["n_quartets"]
        h.close()
    for name in ("mixed", "mixed_all"):
        d = (Ks[name] - Ks["fp64"]).abs()
        out[name]["max_abs_dK_vs_fp64"] = d.max().item()
        out[name]["rms_dK_vs_fp64"] = float(torch.sqrt((d * d).mean()).item())
        out[name]["abs_dE_vs_fp64"] = abs(out[name]["energy"] - out["fp64"]["energy"])
    print(json.dumps({
        "metric": METRIC, "workload": "diamond216", "value": out["mixed"]["quartets_per_s"],
        "unit": "quartets/s", "ms_per_step": out["mixed"]["ms"], "n_gpus": 1, "steps": 1, "warmup": 1,
        "higher_is_better": True, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": workload_desc(s, True, "default"), "quartets": n_q, "fp32_tau": args.fp32_tau},
        "runs": out}), flush=True)


def run_balance(args, torch, hfx, inputs):
    """Load balance of the three distributions of a class launch's quartets over the SMs
    (the paper's pair vs quartet comparison, plus the dynamic counter): per schedule the
    K-build time and the per-SM busy time (sum of CTA lifetimes per SM, globaltimer)."""
    s, P_np = inputs.config1(args.atoms)
    P = torch.from_numpy(P_np).cuda()
    out = {}
    Kref = None
    for name, sch in (("pair_static", hfx.HFX_SCHED_PAIR), ("quartet_static", hfx.HFX_SCHED_QUARTET),
                      ("dynamic", hfx.HFX_SCHED_DYNAMIC)):
        h = hfx.HFX(s, schedule=sch).build_pairs()
        K = h.build_K(P)  # warm-up
        h.set_timing(True)
        h.build_K(P, K)
        st = h.stats()
        busy = h.sm_busy_ns()
        busy = busy[busy > 0]
        out[name] = {"ms": st["ms_build"], "sm_busy_mean_ms": float(busy.mean()) / 1e6,
                     "sm_busy_max_ms": float(busy.max()) / 1e6, "sm_busy_min_ms": float(busy.min()) / 1e6,
                     "imbalance_max_over_mean": float(busy.max() / busy.mean()),
                     "efficiency_mean_over_max": float(busy.mean() / busy.max()), "sms": int(busy.size)}
        if Kref is None:
            Kref = K.clone()
        out[name]["max_abs_dK_vs_pair_static"] = torch.abs(K - Kref).max().item()
        h.close()
    print(json.dumps({"metric": METRIC, "workload": "balance", "value": out["dynamic"]["ms"], "unit": "ms",
                      "higher_is_better": False, "n_gpus": 1, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": workload_desc(s)}, "schedules": out}), flush=True)


def run_serve(args, torch, hfx, inputs):
    """The request stream through the continuous-batching server (mixed precision) and,
    with the same arrivals, one request at a time through the plain FP64 single-system
    path (FIFO).  Latency = device completion - submission, split into the wait for
    admission (queueing) and admission -> completion (service)."""
    pool, reqs = inputs.config4_requests(n_requests=args.requests, rate_per_s=args.rate, n_hi=args.serve_max_atoms)
    used = sorted({w for _, w, _ in reqs})
    sysobj = {w: inputs.make_system(pool[w][0], pool[w][1], pool[w][2]) for w in used}
    P_dev = [torch.from_numpy(inputs.density_matrix(sysobj[w], seed=sd,
                                                    truncate_bohr=inputs.truncation_for(sysobj[w].kind))).cuda()
             for _, w, sd in reqs]
    K_srv = [torch.empty_like(P) for P in P_dev]
    K_one = [torch.empty_like(P) for P in P_dev]
    arrivals = [t for t, _, _ in reqs]
    # plain arm: FP64 contexts, one build at a time in arrival order
    plain = {w: hfx.HFX(sysobj[w]).build_pairs() for w in used}
    nq = {w: plain[w].stats()["n_quartets"] for w in used}
    plain[reqs[0][1]].build_K(P_dev[0], K_one[0])  # warm-up
    torch.cuda.synchronize()
    lat1, wait1, svc1, e_one, t0 = [], [], [], [], time.perf_counter()
    for i, (ta, w, sd) in enumerate(reqs):
        while time.perf_counter() - t0 < ta:
            time.sleep(1e-4)
        ts = time.perf_counter() - t0
        plain[w].build_K(P_dev[i], K_one[i])
        torch.cuda.synchronize()
        td = time.perf_counter() - t0
        lat1.append(1e3 * (td - ta))
        wait1.append(1e3 * (ts - ta))
        svc1.append(1e3 * (td - ts))
        e_one.append(plain[w].energy())
    span1 = time.perf_counter() - t0 - arrivals[0]
    # served arm
    srv = hfx.Server(hbm_budget_gb=120.0, max_inflight=4, max_batch=16, precision=hfx.HFX_MIXED)
    mixed_ctx = {w: hfx.HFX(sysobj[w], precision=hfx.HFX_MIXED).build_pairs() for w in used}
    sid = {w: srv.add_system(mixed_ctx[w]) for w in used}
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    tickets, t0 = [], time.perf_counter()
    for i, (ta, w, sd) in enumerate(reqs):
        while time.perf_counter() - t0 < ta:
            srv.progress()
            time.sleep(1e-4)
        tickets.append(srv.submit(sid[w], P_dev[i], K_srv[i]))
    srv.drain()
    ck = clocks.stop()
    res = [srv.poll(t, release=True) for t in tickets]
    st = srv.stats()
    lat2 = [r["t_done_ms"] - r["t_submit_ms"] for r in res]
    wait2 = [r["t_admit_ms"] - r["t_submit_ms"] for r in res]
    svc2 = [r["t_done_ms"] - r["t_admit_ms"] for r in res]
    span2 = (max(r["t_done_ms"] for r in res) - min(r["t_submit_ms"] for r in res)) * 1e-3
    total_q = sum(nq[w] for _, w, _ in reqs)
    dk = max(torch.abs(a - b).max().item() for a, b in zip(K_srv, K_one))
    de = max(abs(r["energy"] - e) for r, e in zip(res, e_one))
    pct = lambda v, q: float(np.percentile(v, q))
    offered = (len(reqs) - 1) / (arrivals[-1] - arrivals[0]) if len(reqs) > 1 else None
    arm = lambda lat, wait, svc, span: {
        "quartets_per_s": total_q / span, "requests_per_s": len(reqs) / span, "span_s": span,
        "latency_p50_ms": pct(lat, 50), "latency_p99_ms": pct(lat, 99),
        "queue_p50_ms": pct(wait, 50), "queue_p99_ms": pct(wait, 99),
        "service_p50_ms": pct(svc, 50), "service_p99_ms": pct(svc, 99)}
    served = arm(lat2, wait2, svc2, span2)
    served.update({"steps": st["n_steps"], "max_step_size": st["max_step_size"],
                   "max_steps_inflight": st["max_steps_inflight"], "bytes_peak": st["bytes_peak"]})
    print(json.dumps({
        "metric": METRIC, "workload": "serve", "value": served["quartets_per_s"], "unit": "quartets/s",
        "p50_ms": served["latency_p50_ms"], "p99_ms": served["latency_p99_ms"], "n_gpus": 1,
        "higher_is_better": True, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": f"{args.requests} requests of a Poisson stream at {args.rate:g} req/s offered, systems "
                               f"drawn from a seeded pool of 64 (atoms log-uniform in 16..{args.serve_max_atoms}, "
                               "cluster or diamond), fresh P per request; server: 4 stream slots, batches of "
                               "<= 16 and <= 1e7 quartets, 120 GB admission budget, mixed precision (FP32 below "
                               "1e-6, every class but (dd|dd))",
                   "requests": args.requests, "systems_used": len(used), "quartets": total_q,
                   "offered_requests_per_s": offered, "arrival_span_s": arrivals[-1] - arrivals[0],
                   "max_atoms": args.serve_max_atoms},
        "served_mixed": served,
        "one_at_a_time_fp64": arm(lat1, wait1, svc1, span1),
        "speedup_quartets_per_s": served["quartets_per_s"] / (total_q / span1),
        "max_abs_dK_served_mixed_vs_fp64": dk, "max_abs_dE_served_mixed_vs_fp64": de,
        "clocks": {"sm_mhz": ck["sm_mhz"], "sm_max_mhz": ck["sm_max_mhz"], "reasons": ck["reasons"]},
    }), flush=True)
    srv.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--ref-sample", type=int, default=2000000, help="quartets per oracle step (--impl reference)")
    ap.add_argument("--cpu-sample", type=int, default=5000000,
                    help="quartets of the CPU-oracle baseline on the main line (10-30 s of host work)")
    ap.add_argument("--workload", default="diamond64", choices=["diamond64", "batch32", "diamond216", "serve", "balance",
                                                              "nao2gto"])
    ap.add_argument("--requests", type=int, default=32, help="serve: requests of the stream to run")
    ap.add_argument("--rate", type=float, default=0.3, help="serve: offered Poisson rate (requests/s)")
    ap.add_argument("--serve-max-atoms", type=int, default=96, help="serve: largest system of the pool")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--atoms", type=int, default=64,
                    help="diamond piece size (64 = the benchmark workload; smaller for profiler captures)")
    ap.add_argument("--report", action="store_true", help="per-class table on stderr")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--fp32-classes", default="default", choices=["default", "all", "sp"])
    ap.add_argument("--fp32-tau", type=float, default=1e-6)
    ap.add_argument("--no-mixed", action="store_true", help="skip the same-run mixed-precision build")
    ap.add_argument("--dist-tau", type=float, default=0.0,
                    help="distance-aware screening threshold (0 = off, the benchmark setting)")
    ap.add_argument("--mixed-steps", type=int, default=5, help="timed mixed-precision builds in the main run")
    ap.add_argument("--density-tau", type=float, default=0.0,
                    help="density-weighted screening threshold (0 = off, the benchmark setting)")
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

    if args.workload != "diamond64":
        if rank == 0:
            {"batch32": run_batch32, "diamond216": run_diamond216, "serve": run_serve,
             "balance": run_balance, "nao2gto": run_nao}[args.workload](
                args, torch, hfx, inputs)
        if pg:
            pg.destroy_process_group()
        return

    s, P_np = inputs.config1(args.atoms)
    stream = torch.cuda.Stream()
    mixed = args.precision == "mixed"
    h = hfx.HFX(s, stream=stream, precision=hfx.HFX_MIXED if mixed else hfx.HFX_FP64,
                fp32_class_mask=class_mask(hfx, args.fp32_classes),
                fp32_tau=args.fp32_tau, density_tau=args.density_tau, dist_tau=args.dist_tau)
    h.build_pairs()
    ms_pairs = h.stats()["ms_pairs"]
    P = torch.from_numpy(P_np).cuda()
    K = torch.empty_like(P)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    n_q = h.stats()["n_quartets"]
    fp64_peak, fp32_peak = hfx.measure_fma_peak()
    lane_ms32, lane_ms1 = hfx.measure_fp64_lane_cost()

    def timed_builds(hh, KK, steps, warmup, sampler=None):
        """warm-up, then `steps` builds each bracketed by CUDA events on the library's
        stream (L2 flushed before each); per-class CUDA events and counters stay on"""
        hh.set_timing(True)
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                hh.build_K(P, KK)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if sampler:
            sampler.start()
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        cms, st = [], None
        with torch.cuda.stream(stream):
            for i in range(steps):
                flush.fill_(float(i))
                evs[i][0].record(stream)
                hh.build_K(P, KK)
                evs[i][1].record(stream)
                st = hh.stats()  # waits for this step (outside its events)
                cms.append(st["ms_class"])
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        ck = sampler.stop() if sampler else None
        return [a.elapsed_time(b) for a, b in evs], cms, st, ck

    clocks = ClockSampler(local)
    step_ms, class_ms, st_timed, ck = timed_builds(h, K, args.steps, args.warmup, clocks)
    total_ms = sum(step_ms)
    if pg:
        total_ms = max_over_ranks(total_ms, pg)
    energy = h.energy()

    # the mixed-precision build of the same workload in the same run (the metric's
    # comparison against plain FP64): time, throughput and errors against the FP64 K
    mixed_obj = None
    if not mixed and not args.no_mixed and not args.density_tau and not args.dist_tau:
        hm = hfx.HFX(s, stream=stream, precision=hfx.HFX_MIXED, fp32_tau=args.fp32_tau).build_pairs()
        Km = torch.empty_like(P)
        m_ms, _, st_m, _ = timed_builds(hm, Km, args.mixed_steps, 2)
        d = (Km - K).abs()
        m_med = float(np.median(m_ms))
        mixed_obj = {
            "ms_per_step": float(np.mean(m_ms)), "p50_ms": m_med, "p99_ms": float(np.percentile(m_ms, 99)),
            "steps": args.mixed_steps, "quartets_per_s": n_q / (np.mean(m_ms) * 1e-3),
            "speedup_vs_fp64": (total_ms / args.steps) / float(np.mean(m_ms)),
            "quartets_fp32": int(sum(st_m["quartets_fp32_class"])),
            "quartets_evaluated": int(sum(st_m["quartets_evaluated_class"])),
            "max_abs_dK_vs_fp64": d.max().item(), "rms_dK_vs_fp64": float(torch.sqrt((d * d).mean()).item()),
            "abs_dE_vs_fp64": abs(hm.energy() - energy), "fp32_tau": args.fp32_tau,
            "fp32_classes": MASK_DESC["default"],
        }
        hm.close()

    # end-to-end through the host-buffer entry point (copies inside the timed region)
    e2e_t = []
    for i in range(args.e2e_steps):
        t0 = time.perf_counter()
        Kh = h.build_K_host(P_np)
        e2e_t.append(time.perf_counter() - t0)
    nbytes = 8 * s.n_bf * s.n_bf

    # roofline of the dominant kernel: the warp-group kernel (the classes it runs), from the
    # CUDA events around each class launch over the timed steps
    from paper_2009_03559_gb300.hfx import QUARTET_CLASSES
    ms_cls = [float(np.mean([c[k] for c in class_ms])) for k in range(21)]
    g32 = [c for c in range(21) if st_timed["group_size_class"][c] == 32]
    dom_ms = sum(ms_cls[c] for c in g32)
    prim_c = st_timed["prim_quartets_class"]
    # algorithmic flops: vertical recurrence + contraction per primitive quartet, horizontal
    # recurrence + spherical step + digest per quartet (the Boys evaluations are counted
    # apart, as special-function evaluations)
    rec_fl = sum(st_timed["flops_recurrence_class"][c] for c in g32)
    set_fl = sum(st_timed["flops_class"][c] for c in g32)   # the same plus the primitive set-up
    f32 = st_timed["flops_fp32"] if mixed else 0.0
    ach = lambda fl: (fl - f32 + f32 * (fp64_peak / fp32_peak)) / (dom_ms * 1e-3) / 1e12 if dom_ms > 0 else None
    achieved, achieved_all = ach(rec_fl), ach(set_fl)
    boys_per_s = sum(prim_c[c] * (2 if s.omega > 0 else 1) for c in g32) / (dom_ms * 1e-3) if dom_ms > 0 else None
    # kernel launches per step: class launches (two per class taking FP32 under mixed precision)
    # + density-block maxima + K = A + A^T + two E_K reduction kernels
    n_cls = sum(1 for c in range(21) if st_timed["n_quartets_class"][c] > 0)
    launches_per_step = n_cls + (sum(1 for c in range(21) if st_timed["n_quartets_class"][c] > 0 and
                                     (hfx.FP32_CLASSES_DEFAULT >> c) & 1) if mixed else 0) + 4

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
            "config": {"workload": workload_desc(s, mixed, args.fp32_classes)
                                   + (f"; density-weighted screening {args.density_tau:g}" if args.density_tau else "")
                                   + (f"; distance-aware screening {args.dist_tau:g}" if args.dist_tau else ""),
                       "n_bf": s.n_bf, "quartets_per_step": n_q,
                       "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas x{ws}",
                       "energy_E_K": energy},
            "pair_build_ms": ms_pairs,
            "e2e": {"value": n_q / float(np.median(e2e_t)) if e2e_t else None, "unit": "quartets/s",
                    "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
            "gpu_launches": launches_per_step * args.steps,
            "roofline": {"bound": "alu", "kernel": "eri_g32_kernel (the classes run one quartet per warp), CUDA "
                                                   "events around each class launch over the timed steps",
                         "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": (achieved / fp64_peak) if achieved else None,
                         "flops": "vertical recurrence + contraction per evaluated primitive quartet, horizontal "
                                  "recurrence + spherical step + digest per evaluated quartet (operation counts "
                                  "of the generated tables); Boys evaluations counted apart"
                                  + ("; FP32 flops counted at the FP64/FP32 peak ratio" if mixed else ""),
                         "traffic": None,
                         "traffic_note": "not taken in this run; ncu on one 16-atom launch of this kernel "
                                         "(dp|dp): 1.43 MB read + 0.34 MB written, L2 hit rate 99%",
                         "peak_source": "FP64 FMA-chain probe of this run (hfx_measure_fma_peak)",
                         "with_setup": {"achieved": achieved_all, "frac": (achieved_all / fp64_peak) if achieved_all
                                        else None, "flops": "the same plus the primitive set-up as written "
                                                            "(Boys Taylor chains included)"},
                         "boys_evals_per_s": boys_per_s},
            "clocks": {"sm_mhz": ck["sm_mhz"], "sm_max_mhz": ck["sm_max_mhz"], "reasons": ck["reasons"]},
            "fp64_flops_per_step": st_timed["flops_fp64"],
            "fp32_flops_per_step": st_timed["flops_fp32"],
            "recurrence_flops_per_step": st_timed["flops_recurrence"],
            "quartets_evaluated_per_step": sum(st_timed["quartets_evaluated_class"]),
            # class mixes compare on these: primitive quartets and spherical integrals per second
            "prim_quartets_per_s": sum(st_timed["prim_quartets_class"]) / (total_ms / args.steps * 1e-3),
            "sph_integrals_per_s": sum(q * n for q, n in zip(st_timed["n_quartets_class"], hfx.CLASS_SPH_SIZE))
                                   / (total_ms / args.steps * 1e-3),
            "quartets_fp32_per_step": sum(st_timed["quartets_fp32_class"]),
            "fp64_tflops_step": st_timed["flops_fp64"] / (total_ms / args.steps * 1e-3) / 1e12,
            "fp32_peak_tflops": fp32_peak,
            "fp64_lane_cost": {"ms_32_active_lanes": lane_ms32, "ms_1_active_lane": lane_ms1,
                               "note": "the same FP64 warp instructions with 1 or 32 active lanes"},
            "class_ms": {QUARTET_CLASSES[c]: round(ms_cls[c], 3) for c in range(21)},
        }
        if mixed_obj:
            line["mixed"] = mixed_obj
        if args.report:
            print(f"{'class':9s} {'G':>2s} {'k':>2s} {'quartets':>11s} {'prims':>12s} {'ms':>9s} {'TF/s':>6s} "
                  f"{'frac':>5s}", file=sys.stderr)
            for c in range(21):
                ms = ms_cls[c]
                fl = st_timed["flops_recurrence_class"][c]
                tf = fl / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
                print(f"{QUARTET_CLASSES[c]:9s} {st_timed['group_size_class'][c]:2d} {st_timed['streams_class'][c]:2d} "
                      f"{st_timed['n_quartets_class'][c]:11d} {prim_c[c]:12d} "
                      f"{ms:9.2f} {tf:6.3f} {tf / fp64_peak:5.2f}", file=sys.stderr)
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
