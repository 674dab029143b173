"""fcc_plan_bases_noalloc: basis construction that makes no device allocation.

It is meant for callers that must not call cudaMalloc / cudaFree while they
run (either may synchronise the whole device; some hosts own all device memory
through their own pool).  Its results must equal what fcc_plan_create builds,
on consecutive calls that reuse the library's one static scratch array.
This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2204_13622_gb300 import binding
    return binding


def _same(a, b, rel=1e-12):
    a, b = np.asarray(a), np.asarray(b)
    assert a.shape == b.shape
    scale = max(np.abs(b).max(), 1e-300)
    assert np.abs(a - b).max() <= rel * scale


def _check_against_plan(B, N, L, den, res):
    plan = B.Plan(2, 16000.0, N, den, tau_max=L)
    info, se, so, Pe, Po, Ue, Uo = res
    for k in ("I", "Q", "K", "K_even", "K_odd", "center"):
        assert info[k] == plan.info[k], k
    pse, pso = plan.singular_values()
    _same(se, pse)
    _same(so, pso)
    for got, ref in zip((Pe, Po, Ue, Uo), plan.bases()):
        _same(got, ref, rel=1e-10)
    plan.close()


@pytest.mark.parametrize("N,L,den", [(512, 5, 4), (1024, 12, 8)])
def test_noalloc_matches_plan_create_twice(B, N, L, den):
    first = B.plan_bases_noalloc(2, 16000.0, N, den, tau_max=L)
    second = B.plan_bases_noalloc(2, 16000.0, N, den, tau_max=L)
    _check_against_plan(B, N, L, den, first)
    _check_against_plan(B, N, L, den, second)


def test_noalloc_after_a_different_grid(B):
    # the static array keeps the previous call's contents; a smaller grid in
    # between must not leak into the next result
    B.plan_bases_noalloc(2, 16000.0, 1024, 8, tau_max=12)
    small = B.plan_bases_noalloc(2, 16000.0, 64, 4, tau_max=2)
    _check_against_plan(B, 64, 2, 4, small)
    again = B.plan_bases_noalloc(2, 16000.0, 512, 4, tau_max=5)
    _check_against_plan(B, 512, 5, 4, again)


def test_noalloc_rejects_grids_beyond_the_static_array(B):
    desc = B.PlanDesc(2, None, 16000.0, 4096, 343.0, 63.0, 4, 0, 0.999, 0, 0)
    info = B.PlanInfo()
    st = B.lib().fcc_plan_bases_noalloc(ctypes.byref(desc), ctypes.byref(info), None, None, None, None,
                                       None, None, None)
    assert st == 2  # FCC_ERR_UNSUPPORTED
    assert "static array" in B.lib().fcc_last_error().decode()


def test_noalloc_calls_leave_device_memory_unchanged(B):
    # the first call on the device may load the library's device code, which
    # allocates the static array; after it, calls must not change the amount of
    # free device memory (no cudaMalloc, no library workspace, no torch tensor)
    B.plan_bases_noalloc(2, 16000.0, 512, 4, tau_max=5)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    torch_bytes0 = torch.cuda.memory_allocated()
    for N, L, den in [(512, 5, 4), (1024, 12, 8), (256, 3, 4), (512, 5, 4)]:
        B.plan_bases_noalloc(2, 16000.0, N, den, tau_max=L)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
    assert torch.cuda.memory_allocated() == torch_bytes0
