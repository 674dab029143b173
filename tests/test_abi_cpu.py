"""Host-side checks of the C ABI that need no GPU: the library loads and
exports every function include/*.h declares, and the binding agrees."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2204_13622_gb300 import binding
    return binding.lib()


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, h)).read(), flags=re.S)
            names |= set(re.findall(r"\b(fcc_[a-z_]+)\s*\(", txt))
    return sorted(names)


def test_header_lists_every_binding_export():
    from paper_2204_13622_gb300 import binding
    assert declared_functions() == sorted(binding.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    from paper_2204_13622_gb300 import binding
    for code in binding.STATUS:
        s = lib.fcc_status_string(code).decode()
        assert s and s != "unknown status"
    assert lib.fcc_status_string(99).decode() == "unknown status"


def test_null_arguments_rejected_without_gpu(lib):
    from paper_2204_13622_gb300 import binding
    assert lib.fcc_plan_create(None, None) == 1
    assert lib.fcc_tdoa(None, None, 0, None, None, None, None, None, None) == 1
    assert lib.fcc_plan_info(None, None) == 1
    lib.fcc_plan_destroy(None)  # no-op
    d = binding.PlanDesc(1, None, 16000.0, 512, 343.0, 3.0, 4, 0, 0.999, 0, 0)
    h = ctypes.c_void_p()
    assert lib.fcc_plan_create(ctypes.byref(d), ctypes.byref(h)) == 1  # n_mics < 2
    d = binding.PlanDesc(4, None, 16000.0, 500, 343.0, 3.0, 4, 0, 0.999, 0, 0)
    assert lib.fcc_plan_create(ctypes.byref(d), ctypes.byref(h)) == 1  # N not a power of two
    assert "power of two" in lib.fcc_last_error().decode()
    # DoA search entry points
    assert lib.fcc_doa_create(None, None, None, 4, ctypes.byref(h)) == 1 and not h.value
    assert lib.fcc_doa_search(None, None, 0, None, None, None) == 1
    assert lib.fcc_doa_workspace(None, 10, None) == 1
    assert lib.fcc_tdoa_doa(None, None, 0, None, None, None, None, None, 0, None) == 1
    lib.fcc_doa_destroy(None)  # no-op
    # STFT front-end entry points
    T = ctypes.c_longlong()
    assert lib.fcc_stft_frames(None, 10, 4, ctypes.byref(T)) == 1
    assert lib.fcc_stft(None, None, 0, 0, 1, None, None) == 1
    assert lib.fcc_pcm_workspace(None, 10, 4, None) == 1
    assert lib.fcc_tdoa_pcm(None, None, 0, 0, 1, None, None, None, None, 0, None) == 1
    assert lib.fcc_tdoa_pcm_host(None, None, 0, 0, 1, None, None, None, None) == 1


def test_debug_hooks_validate_arguments(lib):
    assert lib.fcc_debug_set(99, 0) == 1
    assert lib.fcc_debug_set(0, 10) == 1          # wait bound below 1000 cycles
    assert lib.fcc_debug_set(1, -1) == 1
    assert lib.fcc_debug_set(0, 5000) == 0
    assert lib.fcc_debug_set(0, 0) == 0           # back to the default bound
    assert lib.fcc_debug_set(2, 0) == 0


def test_no_cpu_fallback_without_a_gpu(lib):
    # a valid plan on a machine with no GPU fails with FCC_ERR_CUDA and leaves
    # no handle: nothing in the library computes on the host instead
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2204_13622_gb300 import binding
    d = binding.PlanDesc(4, None, 16000.0, 512, 343.0, 3.0, 4, 0, 0.999, 0, 0)
    h = ctypes.c_void_p()
    assert lib.fcc_plan_create(ctypes.byref(d), ctypes.byref(h)) == 4 and not h.value
    with pytest.raises(binding.FccError) as e:
        binding.Plan(4, 16000.0, 512, 4, tau_max=3, device=0)
    assert e.value.status == 4


def test_remaining_entry_points_reject_null_arguments(lib):
    # every entry point not covered above answers FCC_ERR_INVALID_ARG (1) to a
    # null handle or output before it touches a device; destroy(NULL) is a no-op
    N = None
    h = ctypes.c_void_p()
    d = ctypes.c_double
    calls = [
        lambda: lib.fcc_plan_taus(N, N),
        lambda: lib.fcc_plan_singular_values(N, N, N, N, N),
        lambda: lib.fcc_plan_bases(N, N, N, N, N),
        lambda: lib.fcc_tdoa_host(N, N, 0, N, N, N, N),
        lambda: lib.fcc_gcc_tdoa(N, N, 0, N, N, N, N),
        lambda: lib.fcc_plan_sync(N, N),
        lambda: lib.fcc_plan_geometry(N, N),
        lambda: lib.fcc_plan_autotune(N, N, 0, 1, N),
        lambda: lib.fcc_smooth_workspace(N, 10, N),
        lambda: lib.fcc_tdoa_smoothed(N, N, 0, d(0.5), N, N, 0, N, N, N, N, N, N),
        lambda: lib.fcc_batch_create(N, N, 0, 0, 0, N, ctypes.byref(h)),
        lambda: lib.fcc_batch_info(N, N),
        lambda: lib.fcc_batch_array_info(N, 0, N),
        lambda: lib.fcc_batch_bind(N, N, N, N, N, N),
        lambda: lib.fcc_batch_run(N, N),
        lambda: lib.fcc_batch_sync(N, N),
        lambda: lib.fcc_mlp_create(16, 128, N, d(0.1), N, 0, N),
        lambda: lib.fcc_mlp_get_state(N, N, N, N, N),
        lambda: lib.fcc_mlp_set_state(N, N, N, N, 0),
        lambda: lib.fcc_mlp_gradient(N, N, N, N, 10, N, N, N),
        lambda: lib.fcc_mlp_train_step(N, N, N, N, 10, ctypes.c_float(0.1), N, N),
        lambda: lib.fcc_mlp_infer(N, N, N, 10, ctypes.c_float(0.5), N, N, N, N),
        lambda: lib.fcc_tdoa_learned(N, N, N, 10, ctypes.c_float(0.5), N, N, N, N, N, N, N),
        lambda: lib.fcc_mlp_sync(N, N),
        lambda: lib.fcc_plan_bases_noalloc(N, N, N, N, N, N, N, N, N),
    ]
    for i, call in enumerate(calls):
        assert call() == 1, i
    assert not h.value
    lib.fcc_batch_destroy(N)
    lib.fcc_mlp_destroy(N)
