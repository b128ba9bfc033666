"""Parity at full size for the two largest workloads, on outputs the oracle computes one
by one (tests/golden/make_golden.py: oracle K blocks, one shell pair at a time, and
per-class counts of kept quartets):

* the 216-atom diamond (2808 functions), plain FP64 (K blocks within 1e-10) and mixed
  precision (K blocks within 1e-7; E_K within 1e-7 of the FP64 build, whose own E_K is
  pinned by the smaller parity tests);
* the 32-system batch (8..128 atoms) in one batched build replayed from a CUDA graph,
  the launch configuration bench.py times for it (K blocks of every system within 1e-10);
* the first 96 sites of the 216-atom generator, small enough for a full oracle K
  (tests/golden/oracle_diamond96.json): E_K of the FP64 build within 1e-10 and of the
  mixed-precision build within 1e-7 of the oracle's, K blocks likewise.
The stored 216-atom blocks cover every pair of shell types (s, p, d) x (s, p, d), so every
quartet class contributes to them.
"""
import json
import os

import numpy as np
import pytest

from paper_2009_03559_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.fullsize]
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def hfx_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_03559_gb300 import hfx
    return hfx


def block_errors(s, K, blocks):
    off, nb = s.shell_offset, s.shell_nbf
    errs = []
    for b in blocks:
        I, J = b["I"], b["J"]
        errs.append(np.abs(K[off[I]:off[I] + nb[I], off[J]:off[J] + nb[J]] - np.array(b["K"])))
    flat = np.concatenate([e.ravel() for e in errs])
    return float(flat.max()), float(np.sqrt((flat ** 2).mean()))


def test_diamond216_fp64_and_mixed(hfx_mod):
    g = json.load(open(os.path.join(GOLD, "oracle_diamond216.json")))["systems"][0]
    s, P = inputs.config3()
    assert s.n_bf == g["n_bf"]
    Pd = torch.from_numpy(P).cuda()
    out = {}
    for name, prec in (("fp64", hfx_mod.HFX_FP64), ("mixed", hfx_mod.HFX_MIXED)):
        h = hfx_mod.HFX(s, precision=prec).build_pairs()
        st = h.stats()
        assert st["n_quartets"] == g["n_quartets"]
        assert st["n_quartets_class"] == g["n_quartets_class"]
        K = h.build_K(Pd)
        torch.cuda.synchronize()
        out[name] = (K.cpu().numpy(), h.energy())
        h.close()
    mx, rms = block_errors(s, out["fp64"][0], g["blocks"])
    assert mx <= 1e-10, (mx, rms)
    mx, rms = block_errors(s, out["mixed"][0], g["blocks"])
    dE = abs(out["mixed"][1] - out["fp64"][1])
    print(f"diamond216 mixed: max|dK| blocks {mx:.2e} rms {rms:.2e}, |dE| vs FP64 {dE:.2e}")
    assert mx <= 1e-7 and dE <= 1e-7
    assert np.array_equal(out["fp64"][0], out["fp64"][0].T)


def test_diamond96_energy_against_full_oracle(hfx_mod):
    g = json.load(open(os.path.join(GOLD, "oracle_diamond96.json")))
    s, P = inputs.config3(96)
    assert s.n_bf == g["n_bf"] and s.seed == g["seed"]
    Pd = torch.from_numpy(P).cuda()
    for name, prec, tol in (("fp64", hfx_mod.HFX_FP64, 1e-10), ("mixed", hfx_mod.HFX_MIXED, 1e-7)):
        h = hfx_mod.HFX(s, precision=prec).build_pairs()
        st = h.stats()
        assert st["n_quartets"] == g["n_quartets"]
        assert st["n_quartets_class"] == g["n_quartets_class"]
        K = h.build_K(Pd)
        torch.cuda.synchronize()
        Kh = K.cpu().numpy()
        e = h.energy()
        mx, rms = block_errors(s, Kh, g["blocks"])
        print(f"diamond96 {name}: |dE| vs oracle {abs(e - g['E_K']):.2e}, max|dK| blocks {mx:.2e}")
        assert abs(e - g["E_K"]) <= tol
        assert mx <= tol
        h.close()


def test_batch32_graph(hfx_mod):
    g = json.load(open(os.path.join(GOLD, "oracle_batch32.json")))["systems"]
    systems = inputs.config2_systems()
    ctxs = [hfx_mod.HFX(s).build_pairs() for s, P in systems]
    for c, gs in zip(ctxs, g):
        st = c.stats()
        assert st["n_quartets"] == gs["n_quartets"] and st["n_quartets_class"] == gs["n_quartets_class"]
    Ps = [torch.from_numpy(P).cuda() for s, P in systems]
    Ks = [torch.empty_like(P) for P in Ps]
    b = hfx_mod.Batch(ctxs)
    b.run(Ps, Ks)
    torch.cuda.synchronize()
    worst = 0.0
    for (s, P), K, gs in zip(systems, Ks, g):
        Kh = K.cpu().numpy()
        mx, rms = block_errors(s, Kh, gs["blocks"])
        worst = max(worst, mx)
        assert np.array_equal(Kh, Kh.T)
    print(f"batch32: max|dK| over sampled blocks of 32 systems {worst:.2e}")
    assert worst <= 1e-10
