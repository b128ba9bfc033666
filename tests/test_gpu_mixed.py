"""Mixed precision: FP32 set-up (incomplete-gamma Boys step, FP64 for the primitive quartets it
declines), recurrences and contraction for quartets with Q_IJ Q_KL max|P blocks| < 1e-6; FP64
HRR, spherical step and K accumulation.  Tolerance against the FP64 oracle: max |dK| <= 1e-7 and
|dE_K| <= 1e-7 Hartree (the number the target statement fixes for this path).  The class masks
checked: the default (every class but (dd|dd)), s,p classes only, and all classes (on the small
cases, where it still meets the tolerance).  Shells of 5 and 6 primitives run the primitive
loops in several chunks of 96 (the deferred FP64 set-ups are flushed per chunk)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2009_03559_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-7
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def hfx_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_03559_gb300 import hfx
    return hfx


def build(hfx, s, P, **kw):
    h = hfx.HFX(s, **kw).build_pairs()
    h.set_timing(True)
    K = h.build_K(torch.from_numpy(P).cuda()).cpu().numpy()
    return h, K, h.energy()


def oracle_K(s, P):
    S = oracle.Screen(oracle.Basis(s))
    return S.build_K(P, "sym")


@pytest.mark.parametrize("mask", ["all", "sp", "default"])
@pytest.mark.parametrize("case", ["cluster16", "diamond8", "diamond16"])
def test_mixed_against_oracle(hfx_mod, case, mask):
    s, P = {"cluster16": inputs.config0, "diamond8": lambda: inputs.config1(8),
            "diamond16": lambda: inputs.config1(16)}[case]()
    m = {"all": hfx_mod.ALL_CLASS_MASK, "sp": hfx_mod.SP_CLASS_MASK, "default": hfx_mod.FP32_CLASSES_DEFAULT}[mask]
    h, K, e = build(hfx_mod, s, P, precision=hfx_mod.HFX_MIXED, fp32_class_mask=m)
    Ko, eo = oracle_K(s, P)
    st = h.stats()
    assert sum(st["quartets_fp32_class"]) > 0
    dk = np.abs(K - Ko)
    print(f"{case} {mask}: fp32 quartets {sum(st['quartets_fp32_class'])}/{sum(st['quartets_evaluated_class'])} "
          f"max|dK| {dk.max():.2e} rms {np.sqrt((dk ** 2).mean()):.2e} |dE| {abs(e - eo):.2e}")
    assert dk.max() <= TOL
    assert abs(e - eo) <= TOL
    assert np.array_equal(K, K.T)


def test_mixed_with_zero_threshold_is_fp64(hfx_mod):
    s, P = inputs.config1(8)
    h1, K1, e1 = build(hfx_mod, s, P, precision=hfx_mod.HFX_MIXED, fp32_tau=0.0)
    h2, K2, e2 = build(hfx_mod, s, P)
    assert sum(h1.stats()["quartets_fp32_class"]) == 0
    assert np.abs(K1 - K2).max() <= 1e-12


def test_mixed_diamond64_full_size(hfx_mod):
    """64-atom diamond (832 functions): E_K and sampled K blocks against stored oracle values."""
    path = os.path.join(GOLD, "oracle_diamond64.json")
    g = json.load(open(path))
    s, P = inputs.config1(64)
    h, K, e = build(hfx_mod, s, P, precision=hfx_mod.HFX_MIXED)
    off, nb = s.shell_offset, s.shell_nbf
    worst = 0.0
    for b in g["blocks"]:
        I, J = b["I"], b["J"]
        worst = max(worst, float(np.abs(K[off[I]:off[I] + nb[I], off[J]:off[J] + nb[J]] - np.array(b["K"])).max()))
    print(f"diamond64 mixed: |dE| {abs(e - g['E_K']):.2e} max|dK| over sampled blocks {worst:.2e}")
    assert worst <= TOL
    assert abs(e - g["E_K"]) <= TOL


@pytest.mark.parametrize("case", ["cluster16", "diamond16"])
def test_mixed_global_pmax(hfx_mod, case):
    """The FP32 test with the whole-matrix max|P| instead of the quartet's four blocks:
    never more FP32 quartets than the per-quartet test, and within the same tolerance."""
    s, P = {"cluster16": inputs.config0, "diamond16": lambda: inputs.config1(16)}[case]()
    m = (1 << 21) - 1
    hq, Kq, eq = build(hfx_mod, s, P, precision=hfx_mod.HFX_MIXED, fp32_class_mask=m)
    hg, Kg, eg = build(hfx_mod, s, P, precision=hfx_mod.HFX_MIXED, fp32_class_mask=m, fp32_pmax_global=True)
    Ko, eo = oracle_K(s, P)
    nq = sum(hq.stats()["quartets_fp32_class"])
    ng = sum(hg.stats()["quartets_fp32_class"])
    print(f"{case}: fp32 quartets per-quartet Pmax {nq}, global Pmax {ng}; "
          f"max|dK| {np.abs(Kg - Ko).max():.2e} |dE| {abs(eg - eo):.2e}")
    assert 0 < ng <= nq
    assert np.abs(Kg - Ko).max() <= TOL and abs(eg - eo) <= TOL


@pytest.mark.parametrize("kind,nprim", [("diamond", 5), ("cluster", 6)])
def test_many_primitives(hfx_mod, kind, nprim):
    """More than 96 primitive quartets per quartet (up to 25 x 25 or 36 x 36): FP64 and mixed
    builds against the oracle."""
    if kind == "diamond":
        s = inputs.diamond_system(4, seed=71, nprim=nprim, tau=1e-8, rcut=6.0)
        P = inputs.density_matrix(s, truncate_bohr=10.0)
    else:
        s = inputs.cluster_system(8, seed=72, nprim=nprim, h=5.0, tau=1e-10, rcut=0.0)
        P = inputs.density_matrix(s)
    Ko, eo = oracle_K(s, P)
    h, K, e = build(hfx_mod, s, P)
    assert np.abs(K - Ko).max() <= 1e-10 and abs(e - eo) <= 1e-10
    h, K, e = build(hfx_mod, s, P, precision=hfx_mod.HFX_MIXED)
    st = h.stats()
    assert sum(st["quartets_fp32_class"]) > 0
    assert np.abs(K - Ko).max() <= TOL and abs(e - eo) <= TOL


def test_thread_kernel_fp32_pass(hfx_mod):
    """The thread kernel's FP32 pass (run when a caller fixes the low classes to one quartet per
    thread): FP32 set-up with deferred FP64 set-ups per lane, against the oracle."""
    s, P = inputs.config1(8)
    Ko, eo = oracle_K(s, P)
    h = hfx_mod.HFX(s, precision=hfx_mod.HFX_MIXED).build_pairs()
    h.set_timing(True)  # the per-class counters
    for c in (0, 1, 2, 3, 4, 6, 7, 10, 15):
        h.set_group_size(c, 1)
    K = h.build_K(torch.from_numpy(P).cuda()).cpu().numpy()
    st = h.stats()
    assert sum(st["quartets_fp32_class"][c] for c in (0, 1, 2, 3, 4, 6, 7, 10, 15)) > 0
    assert np.abs(K - Ko).max() <= TOL and abs(h.energy() - eo) <= TOL
