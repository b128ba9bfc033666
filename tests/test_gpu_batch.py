"""Batched K builds: systems of different kinds and sizes in one launch per class, run
through a captured CUDA graph; every system's K must equal its single-system build and
the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2009_03559_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hfx_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_03559_gb300 import hfx
    return hfx


def small_batch():
    out = []
    for i, (kind, n) in enumerate([("cluster", 8), ("diamond", 12), ("cluster", 20), ("diamond", 5),
                                   ("cluster", 1), ("diamond", 16)]):
        s = inputs.make_system(kind, n, seed=9000 + i)
        P = inputs.density_matrix(s, truncate_bohr=inputs.truncation_for(kind))
        out.append((s, P))
    return out


def single(hfx, s, P, **kw):
    h = hfx.HFX(s, **kw).build_pairs()
    K = h.build_K(torch.from_numpy(P).cuda())
    torch.cuda.synchronize()
    return K.cpu().numpy(), h.energy()


@pytest.mark.parametrize("graph", [True, False])
def test_batch_equals_single_and_oracle(hfx_mod, graph):
    systems = small_batch()
    ctxs = [hfx_mod.HFX(s).build_pairs() for s, P in systems]
    Ps = [torch.from_numpy(P).cuda() for s, P in systems]
    Ks = [torch.empty_like(P) for P in Ps]
    b = hfx_mod.Batch(ctxs, graph=graph)
    for rep in range(2):       # capture, then replay
        b.run(Ps, Ks)
        torch.cuda.synchronize()
        for (s, P), c, K in zip(systems, ctxs, Ks):
            Kr, er = single(hfx_mod, s, P)
            assert np.abs(K.cpu().numpy() - Kr).max() <= 1e-12
            assert abs(c.energy() - er) <= 1e-12
    for idx in (0, 1):
        s, P = systems[idx]
        Ko, eo = oracle.Screen(oracle.Basis(s)).build_K(P, "sym")
        assert np.abs(Ks[idx].cpu().numpy() - Ko).max() <= 1e-10
        assert abs(ctxs[idx].energy() - eo) <= 1e-10


def test_graph_replay_with_new_buffers(hfx_mod):
    systems = small_batch()
    ctxs = [hfx_mod.HFX(s).build_pairs() for s, P in systems]
    b = hfx_mod.Batch(ctxs)
    Ps = [torch.from_numpy(P).cuda() for s, P in systems]
    Ks = [torch.empty_like(P) for P in Ps]
    b.run(Ps, Ks)
    # fresh densities in fresh buffers: the same graph, refreshed pointer table
    P2 = [inputs.density_matrix(s, seed=77 + i, truncate_bohr=inputs.truncation_for(s.kind))
          for i, (s, P) in enumerate(systems)]
    Ps2 = [torch.from_numpy(P).cuda() for P in P2]
    Ks2 = [torch.empty_like(P) for P in Ps2]
    b.run(Ps2, Ks2)
    torch.cuda.synchronize()
    for (s, _), P, K in zip(systems, P2, Ks2):
        Kr, er = single(hfx_mod, s, P)
        assert np.abs(K.cpu().numpy() - Kr).max() <= 1e-12


def test_tuned_batch_mixed_precision(hfx_mod):
    systems = small_batch()
    ctxs = [hfx_mod.HFX(s, precision=hfx_mod.HFX_MIXED).build_pairs() for s, P in systems]
    b = hfx_mod.Batch(ctxs)
    Ps = [torch.from_numpy(P).cuda() for s, P in systems]
    Ks = [torch.empty_like(P) for P in Ps]
    b.tune(Ps, Ks)
    b.run(Ps, Ks)
    torch.cuda.synchronize()
    st = b.stats()
    assert st["n_quartets"] > 0 and set(st["group_size_class"]) <= {1, 32}
    for (s, P), K in zip(systems, Ks):
        Kr, er = single(hfx_mod, s, P)
        assert np.abs(K.cpu().numpy() - Kr).max() <= 1e-7


def test_tuner_fp64_and_one_shot(hfx_mod):
    systems = small_batch()
    ctxs = [hfx_mod.HFX(s).build_pairs() for s, P in systems]
    b = hfx_mod.Batch(ctxs)
    Ps = [torch.from_numpy(P).cuda() for s, P in systems]
    Ks = [torch.empty_like(P) for P in Ps]
    b.tune(Ps, Ks)
    b.run(Ps, Ks)
    torch.cuda.synchronize()
    st = b.stats()
    assert set(st["group_size_class"]) <= {1, 32}
    K1 = [K.clone() for K in Ks]
    L = hfx_mod.load_library()
    pP, pK, ld, keep = b._args(Ps, Ks)
    pc, keepc = hfx_mod._ptr_array([c.h.value for c in ctxs])
    assert L.hfx_build_K_batched(pc, pP, pK, ld, len(ctxs)) == 0
    torch.cuda.synchronize()
    for a, c in zip(K1, Ks):
        assert torch.abs(a - c).max().item() <= 1e-12
