"""Allocation failures, injected on the host (hfx_debug_fail_alloc makes the k-th context
allocation fail as an out-of-memory error would; the GPU itself sees no fault): the entry
point reports HFX_ERR_OOM with its message, releases what it held, and the next call on a
fresh or the same context works and gives the same K."""
import pytest

from paper_2009_03559_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hfx_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_03559_gb300 import hfx
    return hfx


def test_init_reports_oom_and_recovers(hfx_mod):
    L = hfx_mod.load_library()
    s, P = inputs.config1(4)
    for k in (1, 3, 9):
        assert L.hfx_debug_fail_alloc(k) == 0
        with pytest.raises(hfx_mod.HFXError) as ei:
            hfx_mod.HFX(s)
        assert ei.value.code == -3 and "injected" in str(ei.value)
    assert L.hfx_debug_fail_alloc(0) == 0
    h = hfx_mod.HFX(s).build_pairs()
    assert h.stats()["n_quartets"] > 0
    h.close()


def test_pair_build_reports_oom_and_the_context_stays_usable(hfx_mod):
    L = hfx_mod.load_library()
    s, P = inputs.config1(4)
    ref = hfx_mod.HFX(s).build_pairs()
    Kref = ref.build_K(torch.from_numpy(P).cuda())
    h = hfx_mod.HFX(s)
    for k in (1, 4, 12):
        assert L.hfx_debug_fail_alloc(k) == 0
        with pytest.raises(hfx_mod.HFXError) as ei:
            h.build_pairs()
        assert ei.value.code == -3
    L.hfx_debug_fail_alloc(0)
    h.build_pairs()
    K = h.build_K(torch.from_numpy(P).cuda())
    assert torch.abs(K - Kref).max().item() <= 1e-13  # atomic accumulation order aside
    h.close()
    ref.close()
