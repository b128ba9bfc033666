"""The request loop (continuous batching over resident systems), through the C ABI.

Each result must be the same alone and in a mix of concurrent requests (the only
difference allowed is the order of the FP64 atomic additions into K: 1e-12), equal to the
single-system build, and, for one small system, to the FP64 oracle within 1e-10.
"""
import numpy as np
import pytest

import oracle
from paper_2009_03559_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_ORDER = 1e-12


@pytest.fixture(scope="module")
def hfx_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_03559_gb300 import hfx
    return hfx


SYSTEMS = [("diamond", 32), ("cluster", 8), ("diamond", 12), ("cluster", 20), ("diamond", 5), ("diamond", 16)]


def make_systems():
    return [inputs.make_system(kind, n, seed=9100 + i) for i, (kind, n) in enumerate(SYSTEMS)]


def density(s, seed):
    return inputs.density_matrix(s, seed=seed, truncate_bohr=inputs.truncation_for(s.kind))


def request_list(systems):
    """(system index, P seed) pairs: every system twice, the big one first."""
    out = []
    for rep in range(2):
        for i in range(len(systems)):
            out.append((i, 500 + 10 * i + rep))
    return out


def run_alone(hfx, systems, reqs, **kw):
    res = {}
    for i, seed in reqs:
        srv = hfx.Server(**kw)
        c = hfx.HFX(systems[i], precision=kw.get("precision", 0)).build_pairs()
        sid = srv.add_system(c)
        P = torch.from_numpy(density(systems[i], seed)).cuda()
        K = torch.empty_like(P)
        t = srv.submit(sid, P, K)
        r = srv.wait(t)
        assert r["status"] == 0 and r["step_size"] == 1
        res[(i, seed)] = (K.cpu().numpy(), r["energy"])
        srv.close()
        c.close()
    return res


@pytest.mark.parametrize("precision", [0, 1])
def test_alone_equals_mix(hfx_mod, precision):
    systems = make_systems()
    reqs = request_list(systems)
    kw = dict(max_inflight=2, max_batch=4, precision=precision, max_step_quartets=1e12)
    alone = run_alone(hfx_mod, systems, reqs, **kw)
    srv = hfx_mod.Server(**kw)
    ctxs = [hfx_mod.HFX(s, precision=precision).build_pairs() for s in systems]
    ids = [srv.add_system(c) for c in ctxs]
    Ps = [torch.from_numpy(density(systems[i], seed)).cuda() for i, seed in reqs]
    Ks = [torch.empty_like(P) for P in Ps]
    torch.cuda.synchronize()
    tickets = [srv.submit(ids[i], P, K) for (i, seed), P, K in zip(reqs, Ps, Ks)]
    results = [srv.wait(t, timeout_ms=600000) for t in tickets]
    st = srv.stats()
    assert st["n_done"] == len(reqs) and st["n_failed"] == 0
    assert st["max_step_size"] > 1, st        # requests were batched
    assert st["max_steps_inflight"] == 2, st  # and steps overlapped on the device
    assert st["bytes_peak"] <= 120e9
    for (i, seed), K, r in zip(reqs, Ks, results):
        Ka, ea = alone[(i, seed)]
        assert r["status"] == 0
        assert np.abs(K.cpu().numpy() - Ka).max() <= TOL_ORDER
        assert abs(r["energy"] - ea) <= TOL_ORDER
        assert r["t_submit_ms"] <= r["t_admit_ms"] <= r["t_done_ms"] + 1.0
    # the same requests through the single-system entry point
    tol = 1e-12 if precision == 0 else 1e-7
    for (i, seed), K in zip(reqs[:len(systems)], Ks):
        h = hfx_mod.HFX(systems[i]).build_pairs()
        Kr = h.build_K(torch.from_numpy(density(systems[i], seed)).cuda())
        assert torch.abs(K - Kr).max().item() <= tol
    srv.close()


def test_served_result_matches_oracle(hfx_mod):
    s = inputs.make_system("diamond", 5, seed=9104)
    P = density(s, 77)
    srv = hfx_mod.Server()
    c = hfx_mod.HFX(s).build_pairs()
    sid = srv.add_system(c)
    Pd = torch.from_numpy(P).cuda()
    K = torch.empty_like(Pd)
    r = srv.wait(srv.submit(sid, Pd, K))
    Ko, eo = oracle.Screen(oracle.Basis(s)).build_K(P, "sym")
    assert np.abs(K.cpu().numpy() - Ko).max() <= 1e-10
    assert abs(r["energy"] - eo) <= 1e-10


def test_pinned_host_buffers_and_pageable_refused(hfx_mod):
    s = inputs.make_system("cluster", 12, seed=9200)
    P = density(s, 3)
    srv = hfx_mod.Server()
    c = hfx_mod.HFX(s).build_pairs()
    sid = srv.add_system(c)
    Ph = torch.from_numpy(P).pin_memory()
    Kh = torch.empty_like(Ph).pin_memory()
    r = srv.wait(srv.submit(sid, Ph, Kh))
    Kd = c.build_K(torch.from_numpy(P).cuda()).cpu().numpy()
    assert np.abs(Kh.numpy() - Kd).max() <= TOL_ORDER
    with pytest.raises(hfx_mod.HFXError) as ei:
        srv.submit(sid, torch.from_numpy(P.copy()), Kh)   # pageable P
    assert ei.value.code == -1


def test_memory_admission(hfx_mod):
    """A budget that holds one request at a time: requests wait for memory, all finish,
    the peak stays within the budget; a request larger than the budget is refused."""
    small = inputs.make_system("diamond", 16, seed=9300)
    big = inputs.make_system("diamond", 64, seed=9301)
    probe = hfx_mod.Server(max_inflight=2, max_batch=4)
    cs = hfx_mod.HFX(small).build_pairs()
    cb = hfx_mod.HFX(big).build_pairs()
    probe.add_system(cs)
    resident_small = probe.stats()["bytes_resident"]
    probe.close()
    n = small.n_bf
    req_bytes = 2 * ((n * n * 8 + 255) // 256 * 256) + (small.n_shells ** 2 * 8 + 255) // 256 * 256 + 256
    budget = resident_small + 1.5 * req_bytes
    srv = hfx_mod.Server(hbm_budget_gb=budget / 1e9, max_inflight=2, max_batch=4)
    sid = srv.add_system(cs)
    with pytest.raises(hfx_mod.HFXError) as ei:   # the big system alone exceeds the budget
        srv.add_system(cb)
    assert ei.value.code == -7
    Ps = [torch.from_numpy(density(small, 40 + k)).cuda() for k in range(5)]
    Ks = [torch.empty_like(P) for P in Ps]
    tickets = [srv.submit(sid, P, K) for P, K in zip(Ps, Ks)]
    res = [srv.wait(t, timeout_ms=600000) for t in tickets]
    st = srv.stats()
    assert all(r["status"] == 0 and r["step_size"] == 1 for r in res)
    assert st["max_steps_inflight"] == 1 and st["bytes_peak"] <= budget
    for P, K in zip(Ps, Ks):
        assert torch.abs(K - cs.build_K(P)).max().item() <= TOL_ORDER


def test_wait_timeout_then_completion(hfx_mod):
    s = inputs.make_system("diamond", 64, seed=9400)
    srv = hfx_mod.Server()
    c = hfx_mod.HFX(s).build_pairs()
    sid = srv.add_system(c)
    P = torch.from_numpy(density(s, 5)).cuda()
    K = torch.empty_like(P)
    t = srv.submit(sid, P, K)
    with pytest.raises(hfx_mod.HFXError) as ei:
        srv.wait(t, timeout_ms=0.0)
    assert ei.value.code == -6
    assert srv.poll(t)["status"] in (1, 2)
    with pytest.raises(hfx_mod.HFXError) as ei:   # not finished: cannot be released
        srv.release(t)
    assert ei.value.code == -5
    r = srv.wait(t, release=True)
    assert r["status"] == 0 and np.isfinite(r["energy"])
    with pytest.raises(hfx_mod.HFXError):         # released: the ticket is gone
        srv.poll(t)


def test_step_quartet_limit(hfx_mod):
    """With a step limit below every system's quartet count, each step holds one request."""
    s = inputs.make_system("cluster", 8, seed=9500)
    srv = hfx_mod.Server(max_inflight=1, max_batch=16, max_step_quartets=1.0)
    c = hfx_mod.HFX(s).build_pairs()
    sid = srv.add_system(c)
    Ps = [torch.from_numpy(density(s, 60 + k)).cuda() for k in range(4)]
    Ks = [torch.empty_like(P) for P in Ps]
    res = [srv.wait(t) for t in [srv.submit(sid, P, K) for P, K in zip(Ps, Ks)]]
    assert all(r["status"] == 0 and r["step_size"] == 1 for r in res)
    assert srv.stats()["max_step_size"] == 1
